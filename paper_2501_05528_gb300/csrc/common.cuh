// Shared host/device helpers of the tblr library (status handling, problem
// checks, kernel-matrix entry functors).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tblr.h"

namespace tblr {

// Record a formatted message for tblr_last_error() (thread-local).
void set_error(const char *fmt, ...);

// Validated, derived view of a tblr_problem.
struct Prob {
  int d, kernel, k, p, e, r, ell, s3, precision, nearfield;
  bool tagged, selfadjoint;  // sketch mode and the self-adjoint flag
  int zrule;                 // TBLR_Z_PROJECT or TBLR_Z_MINRATIO
  int64_t n, b, C;  // C = ell * r
  int grid[3];
  double lo[3], hi[3];
};

// Fills `out` from `in`; returns TBLR_OK or TBLR_EINVAL (message set).
int check_problem(const tblr_problem *in, Prob *out);
int check_layout(const Prob &P, const tblr_layout *lay);

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Returns TBLR_ECUDA (message set) if the last launch failed.
int launch_status(const char *what);

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace tblr

#define TBLR_TRY(call)                 \
  do {                                 \
    int st_ = (call);                  \
    if (st_ != TBLR_OK) return st_;    \
  } while (0)

#define TBLR_CUDA(call)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      tblr::set_error("%s:%d: %s failed: %s", __FILE__, __LINE__, #call,             \
                      cudaGetErrorString(e_));                                       \
      return TBLR_ECUDA;                                                             \
    }                                                                                \
  } while (0)

#define TBLR_REQUIRE(cond, ...)          \
  do {                                   \
    if (!(cond)) {                       \
      tblr::set_error(__VA_ARGS__);      \
      return TBLR_EINVAL;                \
    }                                    \
  } while (0)

namespace tblr {

// ---------------------------------------------------------------- operators
// Entry functors give A(p, q) for box-major positions p (row) and q (column).

// §7.1: A_pq = log|x_p - x_q| = 0.5 log(|x_p - x_q|^2), zero diagonal.
struct Laplace2D {
  const double *x, *y;
  __device__ __forceinline__ double operator()(int64_t p, int64_t q) const {
    if (p == q) return 0.0;
    double dx = x[p] - x[q], dy = y[p] - y[q];
    return 0.5 * log(dx * dx + dy * dy);
  }
};

// A_pq = 1 / (4 pi |x_p - x_q|), zero diagonal.
struct Laplace3D {
  const double *x, *y, *z;
  __device__ __forceinline__ double operator()(int64_t p, int64_t q) const {
    if (p == q) return 0.0;
    double dx = x[p] - x[q], dy = y[p] - y[q], dz = z[p] - z[q];
    return 0.07957747154594767 * rsqrt(dx * dx + dy * dy + dz * dz);  // 1/(4 pi)
  }
};

// Explicit matrix in original point order, row-major; `adjoint` reads A^T.
struct Dense {
  const double *a;
  const int32_t *perm;
  int64_t n;
  int adjoint;
  __device__ __forceinline__ double operator()(int64_t p, int64_t q) const {
    int64_t i = perm[p], j = perm[q];
    return adjoint ? a[j * n + i] : a[i * n + j];
  }
};

// Dispatch a callable templated on the entry functor for the problem's kernel.
template <class F>
int with_operator(const Prob &P, const tblr_layout *lay, const double *dense, int adjoint, F &&f) {
  const int64_t n = P.n;
  switch (P.kernel) {
    case TBLR_KERNEL_LAPLACE2D:
      return f(Laplace2D{lay->pts, lay->pts + n});
    case TBLR_KERNEL_LAPLACE3D:
      return f(Laplace3D{lay->pts, lay->pts + n, lay->pts + 2 * n});
    case TBLR_KERNEL_DENSE:
      TBLR_REQUIRE(dense != nullptr, "dense operator needs the matrix");
      return f(Dense{dense, lay->perm, n, adjoint});
  }
  set_error("unknown kernel %d", P.kernel);
  return TBLR_EINVAL;
}

inline bool symmetric_kernel(int kernel) {
  return kernel == TBLR_KERNEL_LAPLACE2D || kernel == TBLR_KERNEL_LAPLACE3D;
}

// Warp reductions.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// The boxes whose columns enter B_ij (§6.1): every box of colour(j) for the
// paper's identity probe, or j alone for the exact discrepancy block.  The
// whole block scans the colours (a ballot per warp, then the warps' counts in
// order), writes the set in ascending box order to shared memory and returns
// its size.  Every thread of the block must call it (blockDim.x a multiple of 32).
__device__ __forceinline__ int block_probe_set(int j, int mode, const int32_t *__restrict__ colour,
                                               int b, int *set) {
  __shared__ int wcount[32];
  if (mode == TBLR_NEARFIELD_EXACT) {
    if (threadIdx.x == 0) set[0] = j;
    __syncthreads();
    return 1;
  }
  const int g = colour[j];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int base = 0;
  for (int x0 = 0; x0 < b; x0 += blockDim.x) {
    const int x = x0 + threadIdx.x;
    const bool hit = x < b && colour[x] == g;
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) wcount[w] = __popc(m);
    __syncthreads();
    int off = base, tot = 0;
    for (int v = 0; v < nw; ++v) {
      if (v < w) off += wcount[v];
      tot += wcount[v];
    }
    if (hit) set[off + __popc(m & ((1u << lane) - 1u))] = x;
    base += tot;
    __syncthreads();
  }
  return base;
}

}  // namespace tblr
