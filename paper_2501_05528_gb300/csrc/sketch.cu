// a2 (extended test matrices, §4.1 eq. extend_test_mat), the FP64 black-box
// apply Y = A X with A generated tile by tile, and a3 (sketch, Algorithm 2).
//
// FP64 apply design (GB300 runs DFMA at ~1.2 TFLOP/s, so the kernel is bound
// by the FP64 pipe, not by memory): a CTA owns BM = 16 rows of Y and up to
// 256 * CPT columns; each K step generates the BM x BK tile of A once (a log
// or rsqrt costs ~36 DFMA) and contracts it with the BK x (256 CPT) slice of X
// staged in shared memory, so every generated entry feeds up to 1280 DFMAs.
#include <algorithm>

#include "common.cuh"
#include "mixed.cuh"

namespace tblr {
namespace {

constexpr int kTM = 32;  // points per test-matrix tile

// Omega(I_i, j r + q) = T[i, j] G_i(:, q); side 0 writes Omega from G, side 1
// writes Psi from H.  Output K-major: out[(side*C + j r + q) * n + p].
__global__ void __launch_bounds__(256) test_matrices_kernel(
    const double *__restrict__ T, const double *__restrict__ G, const double *__restrict__ H,
    const int32_t *__restrict__ perm, const int32_t *__restrict__ box_of, int64_t n, int r,
    int ell, double *__restrict__ out) {
  extern __shared__ double sm[];
  double *tile = sm;                     // [kTM][r + 1]
  double *tb = sm + kTM * (r + 1);       // [kTM][ell]
  const int side = blockIdx.y;
  const double *src = side ? H : G;
  const int64_t p0 = (int64_t)blockIdx.x * kTM;
  for (int idx = threadIdx.x; idx < kTM * r; idx += blockDim.x) {
    const int pl = idx / r, q = idx % r;
    const int64_t p = p0 + pl;
    tile[pl * (r + 1) + q] = (p < n) ? src[(int64_t)perm[p] * r + q] : 0.0;
  }
  for (int idx = threadIdx.x; idx < kTM * ell; idx += blockDim.x) {
    const int pl = idx / ell, j = idx % ell;
    const int64_t p = p0 + pl;
    tb[pl * ell + j] = (p < n) ? T[(int64_t)box_of[p] * ell + j] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t C = (int64_t)ell * r;
  const int64_t p = p0 + lane;
  for (int64_t c = warp; c < C; c += nw) {
    const int j = (int)(c / r), q = (int)(c % r);
    if (p < n) out[(side * C + c) * n + p] = tb[lane * ell + j] * tile[lane * (r + 1) + q];
  }
}

constexpr int kBM = 16, kBK = 8, kThreads = 256;

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Two-stage pipeline: while the FP64 pipe contracts stage `cur`, the X slice of
// the next K step streams into the other stage with cp.async and the next
// kernel tile is generated.
// Tag factoring (TAGGED): entry (p, q) is scaled by tau[box_of[p] * b + box_of[q]], and
// output columns c >= split go to y2[p * ldy2 + c - split].
struct TagArgs {
  const double *tau;
  const int32_t *box_of;
  int b;
  int64_t split, ldy2;
  double *y2;
};

template <class Op, int CPT, bool TAGGED>
__global__ void __launch_bounds__(kThreads, 1)
    apply_fp64_kernel(Op op, const double *__restrict__ xt, int64_t n, int64_t ncols,
                      double *__restrict__ y, int64_t ldy, TagArgs tg) {
  extern __shared__ double sm[];
  constexpr int NT = kThreads * CPT;
  double *As = sm;                   // [2][kBK][kBM]
  double *Xs = sm + 2 * kBK * kBM;   // [2][kBK][NT]
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t row0 = (int64_t)blockIdx.x * kBM;
  const int64_t col0 = (int64_t)blockIdx.y * NT;
  bool active[CPT];
#pragma unroll
  for (int s = 0; s < CPT; ++s) active[s] = col0 + kThreads * s + warp * 32 < ncols;

  auto stage_in = [&](int buf, int64_t k0) {
#pragma unroll
    for (int s = 0; s < CPT; ++s) {
      const int cl = tid + kThreads * s;
      const int64_t c = col0 + cl;
      double *dst = Xs + buf * kBK * NT + cl;
#pragma unroll
      for (int kk = 0; kk < kBK; ++kk) {
        if (c < ncols && k0 + kk < n)
          cp_async8(dst + kk * NT, xt + c * n + k0 + kk);
        else
          dst[kk * NT] = 0.0;
      }
    }
    cp_async_commit();
    if (tid < kBM * kBK) {
      const int r = tid % kBM, kk = tid / kBM;
      const int64_t gi = row0 + r, gj = k0 + kk;
      double v = 0.0;
      if (gi < n && gj < n) {
        v = op(gi, gj);
        if (TAGGED) v *= tg.tau[(int64_t)tg.box_of[gi] * tg.b + tg.box_of[gj]];
      }
      As[buf * kBK * kBM + kk * kBM + r] = v;
    }
  };

  double acc[kBM][CPT];
#pragma unroll
  for (int r = 0; r < kBM; ++r)
#pragma unroll
    for (int s = 0; s < CPT; ++s) acc[r][s] = 0.0;

  const int64_t nsteps = (n + kBK - 1) / kBK;
  stage_in(0, 0);
  cp_async_wait_all();
  __syncthreads();
  for (int64_t step = 0; step < nsteps; ++step) {
    const int cur = (int)(step & 1);
    if (step + 1 < nsteps) stage_in(cur ^ 1, (step + 1) * kBK);
    const double *Ac = As + cur * kBK * kBM;
    const double *Xc = Xs + cur * kBK * NT;
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      double a[kBM];
#pragma unroll
      for (int r = 0; r < kBM; r += 2) {
        const double2 t = *reinterpret_cast<const double2 *>(Ac + kk * kBM + r);
        a[r] = t.x;
        a[r + 1] = t.y;
      }
#pragma unroll
      for (int s = 0; s < CPT; ++s) {
        if (active[s]) {
          const double x = Xc[kk * NT + tid + kThreads * s];
#pragma unroll
          for (int r = 0; r < kBM; ++r) acc[r][s] = fma(a[r], x, acc[r][s]);
        }
      }
    }
    cp_async_wait_all();
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < CPT; ++s) {
    const int64_t c = col0 + tid + kThreads * s;
    if (c >= ncols) continue;
#pragma unroll
    for (int r = 0; r < kBM; ++r) {
      const int64_t gi = row0 + r;
      if (gi < n) {
        if (!TAGGED || c < tg.split)
          y[gi * ldy + c] = acc[r][s];
        else
          tg.y2[gi * tg.ldy2 + (c - tg.split)] = acc[r][s];
      }
    }
  }
}

template <class Op, int CPT, bool TAGGED>
int launch_apply_fp64_cpt(const Op &op, const double *xt, int64_t n, int64_t ncols, double *y,
                          int64_t ldy, const TagArgs &tg, cudaStream_t s) {
  const size_t smem = sizeof(double) * 2 * (kBK * kBM + kBK * kThreads * CPT);
  auto kern = apply_fp64_kernel<Op, CPT, TAGGED>;
  TBLR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((unsigned)cdiv(n, kBM), (unsigned)cdiv(ncols, kThreads * CPT));
  kern<<<grid, kThreads, smem, s>>>(op, xt, n, ncols, y, ldy, tg);
  return launch_status("apply_fp64_kernel");
}

template <class Op, bool TAGGED = false>
int launch_apply_fp64(const Op &op, const double *xt, int64_t n, int64_t ncols, double *y,
                      int64_t ldy, cudaStream_t s, const TagArgs &tg = TagArgs{}) {
  const int64_t cpt = cdiv(ncols, kThreads);
  if (cpt <= 1) return launch_apply_fp64_cpt<Op, 1, TAGGED>(op, xt, n, ncols, y, ldy, tg, s);
  if (cpt <= 2) return launch_apply_fp64_cpt<Op, 2, TAGGED>(op, xt, n, ncols, y, ldy, tg, s);
  if (cpt <= 3) return launch_apply_fp64_cpt<Op, 3, TAGGED>(op, xt, n, ncols, y, ldy, tg, s);
  if (cpt <= 4) return launch_apply_fp64_cpt<Op, 4, TAGGED>(op, xt, n, ncols, y, ldy, tg, s);
  return launch_apply_fp64_cpt<Op, 5, TAGGED>(op, xt, n, ncols, y, ldy, tg, s);
}

// [G | H] in box-major order, K-major: out[c * n + p] (c < r from G, else H).
__global__ void gather_gh_kernel(const double *__restrict__ G, const double *__restrict__ H,
                                 const int32_t *__restrict__ perm, int64_t n, int r, int sides,
                                 double *__restrict__ out) {
  const int64_t total = n * r * sides;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / n, p = i % n;
    const int64_t src = (int64_t)perm[p] * r + (c < r ? c : c - r);
    out[i] = (c < r) ? G[src] : H[src];
  }
}

}  // namespace

int apply_any(const Prob &P, const tblr_layout *lay, const double *dense, const double *xt,
              int64_t ncols, double *y, int64_t ldy, int adjoint, int precision, void *ws,
              size_t ws_bytes, cudaStream_t s) {
  if (ncols == 0) return TBLR_OK;
  if (precision == TBLR_MIXED) {
    TBLR_REQUIRE(symmetric_kernel(P.kernel), "mixed precision needs a built-in kernel operator");
    return apply_mixed(P, lay, xt, ncols, y, ldy, ws, ws_bytes, s);
  }
  return with_operator(P, lay, dense, adjoint, [&](auto op) {
    return launch_apply_fp64(op, xt, P.n, ncols, y, ldy, s);
  });
}

}  // namespace tblr

using namespace tblr;

extern "C" int tblr_test_matrices(const tblr_problem *prob, const tblr_layout *lay,
                                  const double *T, const double *G, const double *H,
                                  double *omega_psi, void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_TRY(check_layout(P, lay));
  TBLR_REQUIRE(T && G && H && omega_psi, "T, G, H and omega_psi must be non-NULL");
  TBLR_REQUIRE(P.r <= 512 && P.ell <= 128, "r <= 512 and ell <= 128 required");
  const size_t smem = sizeof(double) * (kTM * (P.r + 1) + kTM * P.ell);
  if (smem > 48 * 1024)
    TBLR_CUDA(cudaFuncSetAttribute(test_matrices_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  dim3 grid((unsigned)cdiv(P.n, kTM), 2);
  test_matrices_kernel<<<grid, 256, smem, as_stream(stream)>>>(T, G, H, lay->perm, lay->box_of, P.n,
                                                               P.r, P.ell, omega_psi);
  return launch_status("test_matrices_kernel");
}

extern "C" size_t tblr_apply_workspace(const tblr_problem *prob, int64_t ncols, int precision) {
  Prob P;
  if (check_problem(prob, &P) != TBLR_OK) return 0;
  return precision == TBLR_MIXED ? mixed_workspace(P, ncols) : 0;
}

extern "C" int tblr_apply(const tblr_problem *prob, const tblr_layout *lay, const double *dense,
                          const double *xt, int64_t ncols, double *y, int64_t ldy, int adjoint,
                          int precision, void *ws, size_t ws_bytes, void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_TRY(check_layout(P, lay));
  TBLR_REQUIRE(xt && y, "xt and y must be non-NULL");
  TBLR_REQUIRE(ncols >= 0 && ncols <= 8192 && ldy >= ncols, "need 0 <= ncols <= 8192, ldy >= ncols");
  TBLR_REQUIRE(precision == TBLR_FP64 || precision == TBLR_MIXED, "bad precision");
  return apply_any(P, lay, dense, xt, ncols, y, ldy, adjoint, precision, ws, ws_bytes,
                   as_stream(stream));
}

extern "C" size_t tblr_sketch_workspace(const tblr_problem *prob) {
  Prob P;
  if (check_problem(prob, &P) != TBLR_OK) return 0;
  return P.precision == TBLR_MIXED ? mixed_workspace(P, 2 * P.C) : 0;
}

extern "C" int tblr_sketch(const tblr_problem *prob, const tblr_layout *lay, const double *dense,
                           const double *omega_psi, double *yz, void *ws, size_t ws_bytes,
                           void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_TRY(check_layout(P, lay));
  TBLR_REQUIRE(omega_psi && yz, "omega_psi and yz must be non-NULL");
  TBLR_REQUIRE(2 * P.C <= 8192, "2 ell r must be <= 8192");
  cudaStream_t s = as_stream(stream);
  const int64_t C = P.C;
  if (symmetric_kernel(P.kernel)) {
    // A^T = A: Y and Z come from one pass over A with [Omega | Psi].
    return apply_any(P, lay, dense, omega_psi, 2 * C, yz, 2 * C, 0, P.precision, ws, ws_bytes, s);
  }
  TBLR_REQUIRE(P.precision == TBLR_FP64, "mixed precision needs a built-in kernel operator");
  TBLR_TRY(apply_any(P, lay, dense, omega_psi, C, yz, 2 * C, 0, TBLR_FP64, ws, ws_bytes, s));
  return apply_any(P, lay, dense, omega_psi + C * P.n, C, yz + C, 2 * C, 1, TBLR_FP64, ws, ws_bytes,
                   s);
}

extern "C" size_t tblr_tagged_sketch_workspace(const tblr_problem *prob) {
  Prob P;
  if (check_problem(prob, &P) != TBLR_OK) return 0;
  if (P.precision == TBLR_MIXED && symmetric_kernel(P.kernel)) return tagged_mixed_workspace(P);
  return align256(sizeof(double) * 2 * P.r * P.n);
}

extern "C" int tblr_tagged_sketch(const tblr_problem *prob, const tblr_layout *lay,
                                  const double *dense, const double *tau, const double *G,
                                  const double *H, double *s_out, double *r_out, void *ws,
                                  size_t ws_bytes, void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_TRY(check_layout(P, lay));
  TBLR_REQUIRE(tau && G && s_out && (P.selfadjoint || (H && r_out)),
               "tau, G, s (and, unless self-adjoint, H and rr) must be non-NULL");
  TBLR_REQUIRE(ws != nullptr && ws_bytes >= tblr_tagged_sketch_workspace(prob),
               "tagged sketch workspace too small");
  cudaStream_t s = as_stream(stream);
  if (P.precision == TBLR_MIXED) {
    TBLR_REQUIRE(symmetric_kernel(P.kernel), "mixed precision needs a built-in kernel operator");
    return tagged_sketch_mixed(P, lay, tau, G, H, s_out, r_out, ws, ws_bytes, s);
  }
  double *x = static_cast<double *>(ws);
  const bool sym = symmetric_kernel(P.kernel);
  if (P.selfadjoint) {
    // A = A^T and H = G: R = S, so only S = A' G is formed.
    gather_gh_kernel<<<(unsigned)std::min<int64_t>(cdiv(P.r * P.n, 256), 152 * 32), 256, 0, s>>>(
        G, G, lay->perm, P.n, P.r, 1, x);
    TBLR_TRY(launch_status("gather_gh_kernel"));
    TagArgs only{tau, lay->box_of, (int)P.b, P.r, P.r, nullptr};
    return with_operator(P, lay, dense, 0, [&](auto op) {
      return launch_apply_fp64<decltype(op), true>(op, x, P.n, P.r, s_out, P.r, s, only);
    });
  }
  gather_gh_kernel<<<(unsigned)std::min<int64_t>(cdiv(2 * P.r * P.n, 256), 152 * 32), 256, 0, s>>>(
      G, H, lay->perm, P.n, P.r, 2, x);
  TBLR_TRY(launch_status("gather_gh_kernel"));
  TagArgs tg{tau, lay->box_of, (int)P.b, P.r, P.r, r_out};
  if (sym) {
    // S | R = A' [G | H] with A'(p, q) = tau[box p][box q] A(p, q), one pass over A.
    return with_operator(P, lay, dense, 0, [&](auto op) {
      return launch_apply_fp64<decltype(op), true>(op, x, P.n, 2 * P.r, s_out, P.r, s, tg);
    });
  }
  TagArgs only{tau, lay->box_of, (int)P.b, P.r, P.r, nullptr};
  TBLR_TRY(with_operator(P, lay, dense, 0, [&](auto op) {
    return launch_apply_fp64<decltype(op), true>(op, x, P.n, P.r, s_out, P.r, s, only);
  }));
  // R_i = sum_c tau_ic (A^T)_ic H_c
  return with_operator(P, lay, dense, 1, [&](auto op) {
    return launch_apply_fp64<decltype(op), true>(op, x + P.r * P.n, P.n, P.r, r_out, P.r, s, only);
  });
}
