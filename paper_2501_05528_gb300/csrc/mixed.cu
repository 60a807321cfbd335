// Mixed-precision black-box apply Y = A X on tcgen05 tensor cores (sm_103a).
//
// Split precision: X = Xh + Xl and A = Ah + Al with FP16 parts (11-bit
// significands each), and A X ~ Ah Xh + Ah Xl + Al Xh, three FP16 MMAs with
// FP32 accumulation (the dropped Al Xl term is ~2^-22 relative).  Tensor-core
// FP32 accumulation is flushed every `flush` K chunks (64 points each) into a
// Kahan-compensated FP32 sum kept in TMEM, so the long K = n reduction keeps
// ~2^-40 accumulation error; the result is written in FP64.
//
// One CTA computes a 128-row x 128-column tile of Y over all n points:
//   warp 0      TMA producer: FP16 hi/lo tiles of X (128 columns x 64 points)
//   warp 1      TMEM allocator and single-thread MMA issuer
//   warps 2-5   epilogue: drain the FP32 accumulator into the Kahan sums
//   warps 6-13  generators: evaluate the 128 x 64 kernel tile A(rows, chunk)
//               from double-float coordinates, split it into FP16 hi/lo and
//               write it in the 128-byte-swizzled K-major operand layout
// Stages of shared memory (3 x 64 KiB) and two TMEM accumulators let the
// generators, the TMA, the tensor core and the epilogue overlap.  Every
// mbarrier wait is bounded by a clock budget; a timeout is counted in a device
// counter (read by tblr_device_timeouts) and the CTA drains and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdlib.h>

#include <algorithm>

#include "kernels_f32.cuh"
#include "mixed.cuh"
#include "tc_utils.cuh"

namespace tblr {

static __device__ unsigned int g_mixed_timeouts;

namespace {

constexpr int MB = 128;   // tile rows
constexpr int NB = 128;   // tile columns
constexpr int KC = 64;    // points per K chunk
constexpr int STAGES = 3;
constexpr int kGenWarps = 8;
constexpr int kEpiWarps = 4;
constexpr int kThreads = 32 * (2 + kEpiWarps + kGenWarps);
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitBudget = 1000000000LL;  // clock cycles (~0.5 s) per wait
constexpr int kTileBytes = MB * 128;             // one FP16 plane of a tile

template <int NBT>
struct __align__(1024) Smem {
  uint8_t a[STAGES][2][kTileBytes];  // A hi, A lo: 128 rows x 128 bytes
  uint8_t x[STAGES][2][NBT * 128];   // X hi, X lo: NBT rows x 128 bytes
  uint64_t full_a[STAGES], full_b[STAGES], empty[STAGES];
  uint64_t dfull[2], dempty[2], done;
  uint32_t tmem_base;
  volatile int abort;
};

struct MixedArgs {
  const float *ch, *cl;  // coordinates, hi and lo floats, [d][npad]
  int64_t n, npad;
  int d, kernel, nk, flush;
  int64_t ncols, ldy;
  double *y;
  // Output columns c >= split go to y2[p * ldy2 + c - split] instead of y.
  int64_t split, ldy2;
  double *y2;
  // Tag factoring: entry (p, q) is scaled by tau[box_of[p] * b + box_of[q]].
  const float *tau;
  const int32_t *box_of;
  int b;
  float scale_a;
  double unscale;
  volatile int *status;  // set to 1 by any timed-out wait of this launch
};

template <class SM>
__device__ __forceinline__ bool wait_or_abort(SM &S, volatile int *status, uint64_t *bar,
                                              uint32_t parity) {
  if (tc::mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if (S.abort || *status) {
      S.abort = 1;
      return false;
    }
    if (clock64() - t0 > kWaitBudget) {
      atomicAdd(&g_mixed_timeouts, 1u);
      *status = 1;
      S.abort = 1;
      return false;
    }
  }
}

template <int KERNEL, int NBT, bool TAGGED>
__global__ void __launch_bounds__(kThreads, 1)
    mixed_apply_kernel(const __grid_constant__ CUtensorMap map_hi,
                       const __grid_constant__ CUtensorMap map_lo, MixedArgs a) {
  extern __shared__ uint8_t smem_raw[];
  using SM = Smem<NBT>;
  SM &S = *reinterpret_cast<SM *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                  ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t row0 = (int64_t)blockIdx.x * MB;
  const int col0 = blockIdx.y * NBT;
  const int nk = a.nk, flush = a.flush;
  const int ngroups = (nk + flush - 1) / flush;

  if (warp == 1) {
    tc::tmem_alloc(&S.tmem_base, kTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    // A launch that already timed out elsewhere skips its work.
    S.abort = *a.status;
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&S.full_a[s], kGenWarps);
      tc::mbar_init(&S.full_b[s], 1);
      tc::mbar_init(&S.empty[s], 1);
    }
    for (int d = 0; d < 2; ++d) {
      tc::mbar_init(&S.dfull[d], 1);
      tc::mbar_init(&S.dempty[d], kEpiWarps);
    }
    tc::mbar_init(&S.done, 1);
    tc::fence_mbar_init();
    tc::tma_prefetch(&map_hi);
    tc::tma_prefetch(&map_lo);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int issued = 0;
      for (int c = 0; c < nk && !S.abort; ++c) {
        const int s = c % STAGES;
        const uint32_t ph = (c / STAGES) & 1;
        if (c >= STAGES && !wait_or_abort(S, a.status, &S.empty[s], ph ^ 1)) break;
        tc::mbar_arrive_expect_tx(&S.full_b[s], 2 * NBT * 128);
        tc::tma_load_2d(S.x[s][0], &map_hi, &S.full_b[s], c * KC, col0);
        tc::tma_load_2d(S.x[s][1], &map_lo, &S.full_b[s], c * KC, col0);
        issued = c + 1;
      }
      // Copies still in flight must land before the CTA exits.
      for (int c = (issued > STAGES ? issued - STAGES : 0); c < issued; ++c) {
        const uint32_t ph = (c / STAGES) & 1;
        const long long t0 = clock64();
        while (!tc::mbar_try_wait(&S.full_b[c % STAGES], ph) && clock64() - t0 < kWaitBudget) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_f16_f32(MB, NBT);
      for (int c = 0; c < nk && !S.abort; ++c) {
        const int s = c % STAGES;
        const uint32_t ph = (c / STAGES) & 1;
        const int g = c / flush, d = g & 1;
        const bool first = (c % flush) == 0;
        const bool last = (c % flush) == flush - 1 || c == nk - 1;
        if (first && g >= 2 && !wait_or_abort(S, a.status, &S.dempty[d], ((g >> 1) - 1) & 1)) break;
        if (!wait_or_abort(S, a.status, &S.full_a[s], ph)) break;
        if (!wait_or_abort(S, a.status, &S.full_b[s], ph)) break;
        tc::tc_fence_after();
        const uint32_t ah = tc::smem_u32(S.a[s][0]), al = tc::smem_u32(S.a[s][1]);
        const uint32_t bh = tc::smem_u32(S.x[s][0]), bl = tc::smem_u32(S.x[s][1]);
        const uint32_t dt = tmem + d * NBT;
#pragma unroll
        for (int kk = 0; kk < KC / 16; ++kk) {
          const uint32_t off = kk * 32;  // 16 FP16 along K inside the 128-byte row
          const uint64_t dah = tc::sw128_desc(ah + off), dal = tc::sw128_desc(al + off);
          const uint64_t dbh = tc::sw128_desc(bh + off), dbl = tc::sw128_desc(bl + off);
          tc::mma_f16(dt, dah, dbh, idesc, (first && kk == 0) ? 0u : 1u);
          tc::mma_f16(dt, dah, dbl, idesc, 1u);
          tc::mma_f16(dt, dal, dbh, idesc, 1u);
        }
        tc::mma_commit(&S.empty[s]);
        if (last) tc::mma_commit(&S.dfull[d]);
      }
      // Every MMA issued so far has finished once `done` completes.
      tc::mma_commit(&S.done);
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(&S.done, 0) && clock64() - t0 < kWaitBudget) {
      }
    }
    __syncwarp();
  } else if (warp < 2 + kEpiWarps) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    const uint32_t hi_t = tmem + 2 * NBT + lanes, cc_t = tmem + 3 * NBT + lanes;
    float hv[32], cv[32], dv[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) hv[t] = 0.f;
#pragma unroll
    for (int cg = 0; cg < NBT / 32; ++cg) {
      tc::tmem_st32(hi_t + cg * 32, hv);
      tc::tmem_st32(cc_t + cg * 32, hv);
    }
    tc::tmem_wait_st();
    bool ok = !S.abort;
    for (int g = 0; g < ngroups && ok; ++g) {
      const int d = g & 1;
      if (!wait_or_abort(S, a.status, &S.dfull[d], (g >> 1) & 1)) {
        ok = false;
        break;
      }
      tc::tc_fence_after();
      const uint32_t d_t = tmem + d * NBT + lanes;
#pragma unroll 1
      for (int cg = 0; cg < NBT / 32; ++cg) {
        tc::tmem_ld32(d_t + cg * 32, dv);
        tc::tmem_ld32(hi_t + cg * 32, hv);
        tc::tmem_ld32(cc_t + cg * 32, cv);
#pragma unroll
        for (int t = 0; t < 32; ++t) {  // Kahan: hi + (d - c), c keeps the lost low part
          const float yv = dv[t] - cv[t];
          const float tt = hv[t] + yv;
          cv[t] = (tt - hv[t]) - yv;
          hv[t] = tt;
        }
        tc::tmem_st32(hi_t + cg * 32, hv);
        tc::tmem_st32(cc_t + cg * 32, cv);
      }
      tc::tmem_wait_st();
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&S.dempty[d]);
    }
    if (ok) {
      const int64_t p = row0 + 32 * q + lane;
#pragma unroll 1
      for (int cg = 0; cg < NBT / 32; ++cg) {
        tc::tmem_ld32(hi_t + cg * 32, hv);
        tc::tmem_ld32(cc_t + cg * 32, cv);
        if (p < a.n) {
#pragma unroll
          for (int t = 0; t < 32; ++t) {
            const int64_t c = (int64_t)col0 + cg * 32 + t;
            const double val = ((double)hv[t] - (double)cv[t]) * a.unscale;
            if (c < a.split)
              a.y[p * a.ldy + c] = val;
            else if (c < a.ncols)
              a.y2[p * a.ldy2 + (c - a.split)] = val;
          }
        }
      }
    }
  } else {
    // ---------------------------------------------------------- generators
    const int gt = tid - 32 * (2 + kEpiWarps);  // 0 .. 255
    const int j = gt & 7;                        // 16-byte chunk (8 points) within the 64
    const int rbase = gt >> 3;                   // rows rbase + 32 i, i = 0..3
    float rh[4][3], rl[4][3];
    int64_t prow[4];
    int brow[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      prow[i] = row0 + rbase + 32 * i;
      brow[i] = (TAGGED && prow[i] < a.n) ? a.box_of[prow[i]] : 0;
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        const bool in = ax < a.d && prow[i] < a.n;
        rh[i][ax] = in ? a.ch[ax * a.npad + prow[i]] : 0.f;
        rl[i][ax] = in ? a.cl[ax * a.npad + prow[i]] : 0.f;
      }
    }
    for (int c = 0; c < nk && !S.abort; ++c) {
      const int s = c % STAGES;
      const uint32_t ph = (c / STAGES) & 1;
      if (c >= STAGES && !wait_or_abort(S, a.status, &S.empty[s], ph ^ 1)) break;
      const int64_t q0 = (int64_t)c * KC + 8 * j;
      float qh[8][3], ql[8][3];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        if (ax < a.d) {
          const float4 h0 = *reinterpret_cast<const float4 *>(a.ch + ax * a.npad + q0);
          const float4 h1 = *reinterpret_cast<const float4 *>(a.ch + ax * a.npad + q0 + 4);
          const float4 l0 = *reinterpret_cast<const float4 *>(a.cl + ax * a.npad + q0);
          const float4 l1 = *reinterpret_cast<const float4 *>(a.cl + ax * a.npad + q0 + 4);
          qh[0][ax] = h0.x; qh[1][ax] = h0.y; qh[2][ax] = h0.z; qh[3][ax] = h0.w;
          qh[4][ax] = h1.x; qh[5][ax] = h1.y; qh[6][ax] = h1.z; qh[7][ax] = h1.w;
          ql[0][ax] = l0.x; ql[1][ax] = l0.y; ql[2][ax] = l0.z; ql[3][ax] = l0.w;
          ql[4][ax] = l1.x; ql[5][ax] = l1.y; ql[6][ax] = l1.z; ql[7][ax] = l1.w;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) qh[e][ax] = ql[e][ax] = 0.f;
        }
      }
      // Column boxes of the 8 points (tag factoring only); usually one box.
      int bq[8];
      bool one_box = true;
      if (TAGGED) {
#pragma unroll
        for (int e = 0; e < 8; ++e) bq[e] = a.box_of[min(q0 + e, a.n - 1)];
        one_box = bq[0] == bq[7];
      }
      // A chunk that cannot meet the diagonal or the ragged edge needs no
      // per-entry checks (the test is uniform over the CTA).
      const int64_t kc0 = (int64_t)c * KC;
      const bool clean = (kc0 + KC <= row0 || kc0 >= row0 + MB) && kc0 + KC <= a.n &&
                         row0 + MB <= a.n;
      const float factor = entry_f32_factor<KERNEL>() * a.scale_a;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = rbase + 32 * i;
        uint32_t hw[4], lw[4];
        float w_row = factor;
        if (TAGGED && one_box) w_row *= a.tau[(int64_t)brow[i] * a.b + bq[0]];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          float v2[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            float w = w_row;
            if (TAGGED && !one_box) w = factor * a.tau[(int64_t)brow[i] * a.b + bq[e + u]];
            float v = entry_f32_raw<KERNEL>(rh[i], rl[i], qh[e + u], ql[e + u]) * w;
            if (!clean) {
              const int64_t qq = q0 + e + u;
              if (qq == prow[i] || qq >= a.n || prow[i] >= a.n) v = 0.f;
            }
            v2[u] = v;
          }
          const __half2 h = __floats2half2_rn(v2[0], v2[1]);
          const float2 hf = __half22float2(h);
          const __half2 l = __floats2half2_rn(v2[0] - hf.x, v2[1] - hf.y);
          hw[e / 2] = *reinterpret_cast<const uint32_t *>(&h);
          lw[e / 2] = *reinterpret_cast<const uint32_t *>(&l);
        }
        const int off = r * 128 + ((j ^ (r & 7)) << 4);  // 128-byte swizzle
        *reinterpret_cast<uint4 *>(S.a[s][0] + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(S.a[s][1] + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&S.full_a[s]);
    }
  }

  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// Coordinates as hi/lo floats (x = hi + lo to ~48 bits), zero padded to npad.
__global__ void split_coords_kernel(const double *__restrict__ pts, int64_t n, int64_t npad, int d,
                                    float *__restrict__ ch, float *__restrict__ cl) {
  const int64_t total = npad * d;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ax = i / npad, p = i % npad;
    float h = 0.f, l = 0.f;
    if (p < n) {
      const double x = pts[ax * n + p];
      h = (float)x;
      l = (float)(x - (double)h);
    }
    ch[i] = h;
    cl[i] = l;
  }
}

// X (FP64, K-major [ncols][n]) scaled by 2^4 and split into FP16 hi/lo planes
// [ncols_pad][npad], zero padded.
__global__ void split_x_kernel(const double *__restrict__ xt, int64_t n, int64_t ncols,
                               int64_t npad, int64_t ncols_pad, float scale,
                               __half *__restrict__ xh, __half *__restrict__ xl) {
  const int64_t total = npad * ncols_pad;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / npad, p = i % npad;
    float v = 0.f;
    if (c < ncols && p < n) v = (float)(xt[c * n + p] * (double)scale);
    const __half h = __float2half_rn(v);
    xh[i] = h;
    xl[i] = __float2half_rn(v - __half2float(h));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

int make_map(CUtensorMap *map, const __half *base, int64_t npad, int64_t rows, int box_rows) {
  auto fn = encode_fn();
  TBLR_REQUIRE(fn != nullptr, "cuTensorMapEncodeTiled is unavailable");
  cuuint64_t dims[2] = {(cuuint64_t)npad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)npad * sizeof(__half)};
  cuuint32_t box[2] = {KC, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half *>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return TBLR_ECUDA;
  }
  return TBLR_OK;
}

// Column tiling of `ncols` outputs: tiles of equal width, a multiple of 32, at most 128.
struct ColTiles {
  int width, ntiles;
  int64_t padded;
};

ColTiles col_tiles(int64_t ncols, bool tagged) {
  ColTiles t;
  if (!tagged) {
    t.width = NB;
    t.ntiles = (int)cdiv(ncols, NB);
  } else {
    t.ntiles = (int)cdiv(ncols, 128);
    t.width = (int)(cdiv(cdiv(ncols, t.ntiles), 32) * 32);
  }
  t.padded = (int64_t)t.width * t.ntiles;
  return t;
}

struct MixedLayout {
  int64_t npad, ncols_pad;
  size_t head, coords, planes, tau, total;
};

MixedLayout mixed_layout(const Prob &P, int64_t ncols, bool tagged) {
  MixedLayout L;
  L.npad = cdiv(P.n, KC) * KC;
  L.ncols_pad = col_tiles(ncols, tagged).padded;
  L.head = 256;
  L.coords = align256(sizeof(float) * 2 * 3 * L.npad);
  L.planes = align256(sizeof(__half) * L.npad * L.ncols_pad);
  L.tau = tagged ? align256(sizeof(float) * P.b * P.b) : 0;
  L.total = L.head + L.coords + 2 * L.planes + L.tau;
  return L;
}

int env_flush() {
  static int f = -1;
  if (f < 0) {
    const char *e = getenv("TBLR_MIXED_FLUSH");
    f = e ? atoi(e) : 1;
    if (f < 1) f = 1;
  }
  return f;
}

// [G | H] gathered to box-major order, scaled by 2^4 and split into FP16 hi/lo
// planes [ncols_pad][npad] (rows c < r from G, r <= c < 2r from H, zero padded).
__global__ void split_gh_kernel(const double *__restrict__ G, const double *__restrict__ H,
                                const int32_t *__restrict__ perm, int64_t n, int r, int64_t npad,
                                int64_t ncols_pad, float scale, __half *__restrict__ xh,
                                __half *__restrict__ xl) {
  const int64_t total = npad * ncols_pad;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / npad, p = i % npad;
    float v = 0.f;
    if (p < n && c < 2 * r) {
      const int64_t src = (int64_t)perm[p] * r + (c < r ? c : c - r);
      v = (float)((c < r ? G[src] : H[src]) * (double)scale);
    }
    const __half h = __float2half_rn(v);
    xh[i] = h;
    xl[i] = __float2half_rn(v - __half2float(h));
  }
}

__global__ void tau_to_f32(const double *__restrict__ tau, int64_t len, float *__restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)tau[i];
}

template <int KERNEL, int NBT, bool TAGGED>
int launch_mixed(const CUtensorMap &mh, const CUtensorMap &ml, const MixedArgs &a, int64_t n,
                 int ntiles, cudaStream_t s) {
  auto k = mixed_apply_kernel<KERNEL, NBT, TAGGED>;
  const size_t smem = sizeof(Smem<NBT>) + 1024;
  TBLR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k<<<dim3((unsigned)cdiv(n, MB), (unsigned)ntiles), kThreads, smem, s>>>(mh, ml, a);
  return launch_status("mixed_apply_kernel");
}

template <bool TAGGED>
int dispatch_mixed(int kernel, int width, const CUtensorMap &mh, const CUtensorMap &ml,
                   const MixedArgs &a, int64_t n, int ntiles, cudaStream_t s) {
#define TBLR_MIXED_CASE(W)                                                                      \
  if (width == W)                                                                               \
    return kernel == TBLR_KERNEL_LAPLACE2D                                                      \
               ? launch_mixed<TBLR_KERNEL_LAPLACE2D, W, TAGGED>(mh, ml, a, n, ntiles, s)        \
               : launch_mixed<TBLR_KERNEL_LAPLACE3D, W, TAGGED>(mh, ml, a, n, ntiles, s);
  if (TAGGED) {
    TBLR_MIXED_CASE(32)
    TBLR_MIXED_CASE(64)
    TBLR_MIXED_CASE(96)
  }
  TBLR_MIXED_CASE(128)
#undef TBLR_MIXED_CASE
  set_error("no tensor-core kernel for tile width %d", width);
  return TBLR_EUNSUPPORTED;
}

MixedArgs base_args(const Prob &P, const MixedLayout &L, float *ch, float *cl, volatile int *status) {
  MixedArgs a{};
  a.ch = ch;
  a.cl = cl;
  a.n = P.n;
  a.npad = L.npad;
  a.d = P.d;
  a.kernel = P.kernel;
  a.nk = (int)(L.npad / KC);
  a.flush = env_flush();
  a.scale_a = P.kernel == TBLR_KERNEL_LAPLACE2D ? 16.f : 1.f;
  a.unscale = 1.0 / ((double)a.scale_a * 16.0);
  a.status = status;
  return a;
}

}  // namespace

size_t mixed_workspace(const Prob &P, int64_t ncols) { return mixed_layout(P, ncols, false).total; }
size_t tagged_mixed_workspace(const Prob &P) { return mixed_layout(P, 2 * P.r, true).total; }

int apply_mixed(const Prob &P, const tblr_layout *lay, const double *xt, int64_t ncols, double *y,
                int64_t ldy, void *ws, size_t ws_bytes, cudaStream_t s) {
  TBLR_REQUIRE(P.kernel == TBLR_KERNEL_LAPLACE2D || P.kernel == TBLR_KERNEL_LAPLACE3D,
               "mixed precision supports the built-in Laplace kernels");
  const MixedLayout L = mixed_layout(P, ncols, false);
  TBLR_REQUIRE(ws != nullptr && ws_bytes >= L.total, "mixed workspace too small (%zu < %zu)",
               ws_bytes, L.total);
  TBLR_REQUIRE((reinterpret_cast<uintptr_t>(ws) & 255) == 0, "workspace must be 256-byte aligned");
  char *w = static_cast<char *>(ws);
  int *status = reinterpret_cast<int *>(w);
  float *ch = reinterpret_cast<float *>(w + L.head);
  float *cl = ch + 3 * L.npad;
  __half *xh = reinterpret_cast<__half *>(w + L.head + L.coords);
  __half *xl = reinterpret_cast<__half *>(w + L.head + L.coords + L.planes);
  TBLR_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
  split_coords_kernel<<<(unsigned)std::min<int64_t>(cdiv(3 * L.npad, 256), 4096), 256, 0, s>>>(
      lay->pts, P.n, L.npad, P.d, ch, cl);
  TBLR_TRY(launch_status("split_coords_kernel"));
  split_x_kernel<<<(unsigned)std::min<int64_t>(cdiv(L.npad * L.ncols_pad, 256), 152 * 32), 256, 0,
                   s>>>(xt, P.n, ncols, L.npad, L.ncols_pad, 16.f, xh, xl);
  TBLR_TRY(launch_status("split_x_kernel"));
  const ColTiles ct = col_tiles(ncols, false);
  CUtensorMap mh, ml;
  TBLR_TRY(make_map(&mh, xh, L.npad, L.ncols_pad, ct.width));
  TBLR_TRY(make_map(&ml, xl, L.npad, L.ncols_pad, ct.width));
  MixedArgs a = base_args(P, L, ch, cl, status);
  a.ncols = ncols;
  a.ldy = ldy;
  a.y = y;
  a.split = ncols;
  a.ldy2 = 0;
  a.y2 = nullptr;
  return dispatch_mixed<false>(P.kernel, ct.width, mh, ml, a, P.n, ct.ntiles, s);
}

int tagged_sketch_mixed(const Prob &P, const tblr_layout *lay, const double *tau, const double *G,
                        const double *H, double *S, double *R, void *ws, size_t ws_bytes,
                        cudaStream_t s) {
  TBLR_REQUIRE(P.kernel == TBLR_KERNEL_LAPLACE2D || P.kernel == TBLR_KERNEL_LAPLACE3D,
               "mixed precision supports the built-in Laplace kernels");
  const int64_t ncols = 2 * P.r;
  const MixedLayout L = mixed_layout(P, ncols, true);
  TBLR_REQUIRE(ws != nullptr && ws_bytes >= L.total, "tagged sketch workspace too small");
  TBLR_REQUIRE((reinterpret_cast<uintptr_t>(ws) & 255) == 0, "workspace must be 256-byte aligned");
  char *w = static_cast<char *>(ws);
  int *status = reinterpret_cast<int *>(w);
  float *ch = reinterpret_cast<float *>(w + L.head);
  float *cl = ch + 3 * L.npad;
  __half *xh = reinterpret_cast<__half *>(w + L.head + L.coords);
  __half *xl = reinterpret_cast<__half *>(w + L.head + L.coords + L.planes);
  float *tf = reinterpret_cast<float *>(w + L.head + L.coords + 2 * L.planes);
  TBLR_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
  split_coords_kernel<<<(unsigned)std::min<int64_t>(cdiv(3 * L.npad, 256), 4096), 256, 0, s>>>(
      lay->pts, P.n, L.npad, P.d, ch, cl);
  TBLR_TRY(launch_status("split_coords_kernel"));
  split_gh_kernel<<<(unsigned)std::min<int64_t>(cdiv(L.npad * L.ncols_pad, 256), 152 * 32), 256, 0,
                    s>>>(G, H, lay->perm, P.n, P.r, L.npad, L.ncols_pad, 16.f, xh, xl);
  TBLR_TRY(launch_status("split_gh_kernel"));
  tau_to_f32<<<(unsigned)std::min<int64_t>(cdiv(P.b * P.b, 256), 1024), 256, 0, s>>>(tau, P.b * P.b,
                                                                                     tf);
  TBLR_TRY(launch_status("tau_to_f32"));
  const ColTiles ct = col_tiles(ncols, true);
  CUtensorMap mh, ml;
  TBLR_TRY(make_map(&mh, xh, L.npad, L.ncols_pad, ct.width));
  TBLR_TRY(make_map(&ml, xl, L.npad, L.ncols_pad, ct.width));
  MixedArgs a = base_args(P, L, ch, cl, status);
  a.ncols = ncols;
  a.ldy = P.r;
  a.y = S;
  a.split = P.r;
  a.ldy2 = P.r;
  a.y2 = R;
  a.tau = tf;
  a.box_of = lay->box_of;
  a.b = (int)P.b;
  return dispatch_mixed<true>(P.kernel, ct.width, mh, ml, a, P.n, ct.ntiles, s);
}

}  // namespace tblr

extern "C" int tblr_device_timeouts(unsigned int *count) {
  TBLR_REQUIRE(count != nullptr, "count is NULL");
  unsigned int zero = 0;
  TBLR_CUDA(cudaDeviceSynchronize());
  TBLR_CUDA(cudaMemcpyFromSymbol(count, tblr::g_mixed_timeouts, sizeof(unsigned int)));
  TBLR_CUDA(cudaMemcpyToSymbol(tblr::g_mixed_timeouts, &zero, sizeof(unsigned int)));
  return TBLR_OK;
}
