// a1: tessellation into a regular grid of boxes, stable box-major order,
// neighbour lists N_i and colours (§2.5 strong admissibility; §6.1 probes).
// Also tblr_tessellate_noalloc, the same tessellation with its scratch in a
// fixed static device array instead of a caller workspace.
//
// Stable counting sort in three launches: per-chunk box histograms, one
// exclusive scan over (box, chunk) in box-major order, and a per-chunk scatter
// that ranks equal boxes in input order (warp match + warps taking turns).
#include <mutex>

#include "common.cuh"

namespace tblr {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 2048;  // points per histogram chunk (8 rounds of 256)

__device__ __forceinline__ int box_of_point(const double *pts, int64_t p, int d, int g0, int g1,
                                            int g2, double lo0, double lo1, double lo2,
                                            double w0, double w1, double w2) {
  // q_a = clamp(floor((x_a - lo_a) / (hi_a - lo_a) * g_a), 0, g_a - 1), rounded
  // step by step exactly as written (no contraction) so the integer result is
  // reproducible on any IEEE machine.
  const double g[3] = {(double)g0, (double)g1, (double)g2};
  const double lo[3] = {lo0, lo1, lo2};
  const double w[3] = {w0, w1, w2};
  int q[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) {
    double t = __dmul_rn(__ddiv_rn(__dsub_rn(pts[p * d + a], lo[a]), w[a]), g[a]);
    t = fmin(fmax(floor(t), 0.0), g[a] - 1.0);
    q[a] = (int)t;
  }
  return q[0] + g0 * (q[1] + g1 * q[2]);
}

struct GridArgs {
  int d, g0, g1, g2;
  double lo0, lo1, lo2, w0, w1, w2;
};

__global__ void __launch_bounds__(kThreads) tess_hist(const double *__restrict__ pts, int64_t n,
                                                      GridArgs ga, int b, int nchunks,
                                                      int32_t *__restrict__ box_orig,
                                                      int32_t *__restrict__ hist) {
  extern __shared__ int32_t sh[];
  for (int i = threadIdx.x; i < b; i += kThreads) sh[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  for (int t = threadIdx.x; t < kChunk; t += kThreads) {
    int64_t p = base + t;
    if (p < n) {
      int bx = box_of_point(pts, p, ga.d, ga.g0, ga.g1, ga.g2, ga.lo0, ga.lo1, ga.lo2, ga.w0,
                            ga.w1, ga.w2);
      box_orig[p] = bx;
      atomicAdd(&sh[bx], 1);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < b; i += kThreads) hist[(int64_t)i * nchunks + blockIdx.x] = sh[i];
}

// Exclusive scan of len values in place by one block of 1024 threads.
template <class T>
__global__ void __launch_bounds__(1024) block_exclusive_scan(T *__restrict__ v, int64_t len,
                                                             T *__restrict__ total) {
  __shared__ T part[1024];
  const int t = threadIdx.x;
  const int64_t seg = (len + 1023) / 1024;
  const int64_t s0 = min((int64_t)t * seg, len), s1 = min(s0 + seg, len);
  T sum = 0;
  for (int64_t i = s0; i < s1; ++i) sum += v[i];
  part[t] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {  // Hillis-Steele on the 1024 partials
    T x = (t >= off) ? part[t - off] : T(0);
    __syncthreads();
    part[t] += x;
    __syncthreads();
  }
  T run = part[t] - sum;
  for (int64_t i = s0; i < s1; ++i) {
    T x = v[i];
    v[i] = run;
    run += x;
  }
  if (t == 1023 && total) *total = part[1023];
}

__global__ void __launch_bounds__(kThreads) tess_scatter(const double *__restrict__ pts, int64_t n,
                                                         int d, int b, int nchunks,
                                                         const int32_t *__restrict__ box_orig,
                                                         const int32_t *__restrict__ start,
                                                         int32_t *__restrict__ perm,
                                                         int32_t *__restrict__ box_of,
                                                         double *__restrict__ spts) {
  extern __shared__ int32_t run[];
  for (int i = threadIdx.x; i < b; i += kThreads) run[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  for (int round = 0; round < kChunk / kThreads; ++round) {
    const int64_t p = base + round * kThreads + threadIdx.x;
    const bool valid = p < n;
    const int key = valid ? box_orig[p] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int rank = __popc(peers & lt);
    const int leader = __ffs(peers) - 1;
    const int cnt = __popc(peers);
    for (int w = 0; w < kThreads / 32; ++w) {
      if (warp == w && valid) {
        const int before = run[key];
        __syncwarp(peers);
        if (lane == leader) run[key] = before + cnt;
        const int64_t pos = (int64_t)start[(int64_t)key * nchunks + blockIdx.x] + before + rank;
        perm[pos] = (int32_t)p;
        box_of[pos] = key;
        for (int a = 0; a < d; ++a) spts[(int64_t)a * n + pos] = pts[p * d + a];
      }
      __syncthreads();
    }
  }
}

__global__ void tess_boxes(const int32_t *__restrict__ start, int nchunks, int b, int64_t n,
                           GridArgs ga, int s3, int32_t *__restrict__ offsets,
                           int32_t *__restrict__ nbr, int32_t *__restrict__ nnbr,
                           int32_t *__restrict__ colour) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) offsets[b] = (int32_t)n;
  if (i >= b) return;
  offsets[i] = start[(int64_t)i * nchunks];
  const int g[3] = {ga.g0, ga.g1, ga.g2};
  const int q[3] = {i % ga.g0, (i / ga.g0) % ga.g1, i / (ga.g0 * ga.g1)};
  int col = 0, pw = 1;
  for (int a = 0; a < ga.d; ++a) {
    col += (q[a] % 3) * pw;
    pw *= 3;
  }
  colour[i] = col;
  // Grid coordinates within one of box i on every axis; the z-outer, x-inner
  // loop order visits box ids in ascending order.
  int cnt = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = q[2] + dz;
    if (z < 0 || z >= g[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int y = q[1] + dy;
      if (y < 0 || y >= g[1]) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int x = q[0] + dx;
        if (x < 0 || x >= g[0]) continue;
        nbr[(int64_t)i * s3 + cnt++] = x + g[0] * (y + g[1] * z);
      }
    }
  }
  nnbr[i] = cnt;
  for (int s = cnt; s < s3; ++s) nbr[(int64_t)i * s3 + s] = -1;
}

// Near-field block sizes m_i * m_j per neighbour slot, and max m_i.
__global__ void nf_sizes(const int32_t *__restrict__ offsets, const int32_t *__restrict__ nbr,
                         const int32_t *__restrict__ nnbr, int b, int s3,
                         int64_t *__restrict__ sz, int32_t *__restrict__ m_max) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)b * s3) return;
  const int i = (int)(t / s3), s = (int)(t % s3);
  const int mi = offsets[i + 1] - offsets[i];
  if (s == 0) atomicMax(m_max, mi);
  if (s < nnbr[i]) {
    const int j = nbr[t];
    sz[t] = (int64_t)mi * (offsets[j + 1] - offsets[j]);
  } else {
    sz[t] = 0;
  }
}

GridArgs grid_args(const Prob &P) {
  GridArgs g;
  g.d = P.d;
  g.g0 = P.grid[0];
  g.g1 = P.grid[1];
  g.g2 = P.grid[2];
  g.lo0 = P.lo[0];
  g.lo1 = P.lo[1];
  g.lo2 = P.lo[2];
  // (hi - lo) rounded once, as a plain subtraction would be
  g.w0 = P.hi[0] - P.lo[0];
  g.w1 = P.hi[1] - P.lo[1];
  g.w2 = P.hi[2] - P.lo[2];
  return g;
}

int64_t num_chunks(int64_t n) { return cdiv(n, kChunk); }

}  // namespace
}  // namespace tblr

using namespace tblr;

extern "C" size_t tblr_tessellate_workspace(const tblr_problem *prob) {
  Prob P;
  if (check_problem(prob, &P) != TBLR_OK) return 0;
  const int64_t nch = num_chunks(P.n);
  return align256(sizeof(int32_t) * P.n) + align256(sizeof(int32_t) * (P.b * nch + 1));
}

extern "C" int tblr_tessellate(const tblr_problem *prob, const double *points,
                               const tblr_layout *out, void *ws, size_t ws_bytes, void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_TRY(check_layout(P, out));
  TBLR_REQUIRE(points != nullptr, "points is NULL");
  TBLR_REQUIRE(ws != nullptr && ws_bytes >= tblr_tessellate_workspace(prob),
               "tessellate workspace too small (%zu < %zu)", ws_bytes,
               tblr_tessellate_workspace(prob));
  cudaStream_t s = as_stream(stream);
  const int64_t nch = num_chunks(P.n);
  const int b = (int)P.b;
  char *w = static_cast<char *>(ws);
  int32_t *box_orig = reinterpret_cast<int32_t *>(w);
  int32_t *hist = reinterpret_cast<int32_t *>(w + align256(sizeof(int32_t) * P.n));
  const GridArgs ga = grid_args(P);
  const size_t shb = sizeof(int32_t) * b;
  if (shb > 48 * 1024) {
    TBLR_CUDA(cudaFuncSetAttribute(tess_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb));
    TBLR_CUDA(cudaFuncSetAttribute(tess_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb));
  }
  tess_hist<<<(unsigned)nch, kThreads, shb, s>>>(points, P.n, ga, b, (int)nch, box_orig, hist);
  TBLR_TRY(launch_status("tess_hist"));
  block_exclusive_scan<int32_t><<<1, 1024, 0, s>>>(hist, (int64_t)b * nch, nullptr);
  TBLR_TRY(launch_status("block_exclusive_scan"));
  tess_scatter<<<(unsigned)nch, kThreads, shb, s>>>(points, P.n, P.d, b, (int)nch, box_orig, hist,
                                                    out->perm, out->box_of, out->pts);
  TBLR_TRY(launch_status("tess_scatter"));
  tess_boxes<<<(unsigned)cdiv(b, 128), 128, 0, s>>>(hist, (int)nch, b, P.n, ga, P.s3, out->offsets,
                                                   out->nbr, out->nnbr, out->colour);
  TBLR_TRY(launch_status("tess_boxes"));
  return TBLR_OK;
}

extern "C" int tblr_nearfield_offsets(const tblr_problem *prob, const tblr_layout *lay,
                                      int64_t *nf_off, int32_t *m_max, void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_TRY(check_layout(P, lay));
  TBLR_REQUIRE(nf_off != nullptr && m_max != nullptr, "nf_off and m_max must be non-NULL");
  cudaStream_t s = as_stream(stream);
  const int64_t len = P.b * P.s3;
  TBLR_CUDA(cudaMemsetAsync(m_max, 0, sizeof(int32_t), s));
  nf_sizes<<<(unsigned)cdiv(len, 256), 256, 0, s>>>(lay->offsets, lay->nbr, lay->nnbr, (int)P.b,
                                                   P.s3, nf_off, m_max);
  TBLR_TRY(launch_status("nf_sizes"));
  block_exclusive_scan<int64_t><<<1, 1024, 0, s>>>(nf_off, len, nf_off + len);
  TBLR_TRY(launch_status("block_exclusive_scan"));
  return TBLR_OK;
}

// ------------------------------------------------- allocation-free variant
// Scratch for tblr_tessellate_noalloc: one fixed array per device, created
// when the library is loaded on that device and held until process exit.
static __device__ __align__(256) unsigned char g_tess_scratch[TBLR_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_tess_scratch on the current device.  Host code cannot
// use the symbol itself (on the host it names a stand-in, not device memory),
// so the address is looked up once per device and cached.
int scratch_address(void **out) {
  int dev = 0;
  TBLR_CUDA(cudaGetDevice(&dev));
  TBLR_REQUIRE(dev >= 0 && dev < kMaxDevices, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void *p = nullptr;
    TBLR_CUDA(cudaGetSymbolAddress(&p, g_tess_scratch));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return TBLR_OK;
}
}  // namespace

extern "C" int tblr_tessellate_noalloc(const tblr_problem *prob, const double *points,
                                       const tblr_layout *out, void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  const size_t need = tblr_tessellate_workspace(prob);
  TBLR_REQUIRE(need <= (size_t)TBLR_NOALLOC_SCRATCH_BYTES,
               "tblr_tessellate_noalloc: this problem needs %zu bytes of scratch, more than the "
               "fixed %d-byte array (use tblr_tessellate with a workspace)",
               need, (int)TBLR_NOALLOC_SCRATCH_BYTES);
  void *scratch = nullptr;
  TBLR_TRY(scratch_address(&scratch));
  // Every scratch byte the tessellation reads is written earlier in the same
  // call (box ids, then the per-chunk histograms), so nothing needs clearing.
  return tblr_tessellate(prob, points, out, scratch, (size_t)TBLR_NOALLOC_SCRATCH_BYTES, stream);
}
