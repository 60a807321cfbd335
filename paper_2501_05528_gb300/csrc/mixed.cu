// Mixed-precision black-box apply Y = A X on tcgen05 tensor cores (sm_103a).
//
// Split precision: every operand value v is carried as three BF16 parts,
// v = h + m + l with |v - h - m - l| <= 2^-24 |v| (each part rounds the
// remainder of the previous one to 8 significant bits; BF16 keeps the FP32
// exponent range, so no scaling is needed and nothing underflows or
// overflows).  A X is then the sum of six BF16 products with FP32
// accumulation:
//   l*h + m*m + h*l   (~2^-16 relative)   issued first,
//   m*h + h*m         (~2^-8)             next,
//   h*h                                   last,
// dropping m*l, l*m and l*l (<= 2^-24).  Issuing the small terms first keeps
// the roundings of the tensor-core adder (which truncates) on small partial
// sums: only the four h*h steps of a K chunk round at the size of the chunk's
// sum.  The FP32 accumulator is flushed every `flush` K chunks (64 points) into
// a Kahan-compensated FP32 sum kept in TMEM, so the long K = n reduction keeps
// ~2^-40 accumulation error; the result is written in FP64.
//
// One CTA computes a 128-row x NBT-column tile of Y over all n points:
//   warp 0      TMA producer: BF16 h/m/l tiles of X (NBT columns x 64 points)
//   warp 1      TMEM allocator and single-thread MMA issuer
//   warps 2-5   epilogue: drain the FP32 accumulator into the Kahan sums
//   warps 6-13  generators: evaluate the 128 x 64 kernel tile A(rows, chunk)
//               from double-float coordinates, split it into BF16 h/m/l and
//               write it in the 128-byte-swizzled K-major operand layout
// Two or three stages of shared memory and (for NBT <= 128) two TMEM
// accumulators let the generators, the TMA, the tensor core and the epilogue
// overlap; NBT = 160 (up to 160 sketch columns in one tile, so each kernel
// tile is generated once) has one accumulator.  Every mbarrier wait is bounded
// by a clock budget; a timeout is counted in a device counter (read by
// tblr_device_timeouts) and the CTA drains and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "coupling_tc.cuh"
#include "kernels_f32.cuh"
#include "mixed.cuh"
#include "tc_pipeline.cuh"
#include "tc_utils.cuh"

namespace tblr {

static __device__ unsigned int g_mixed_timeouts;

namespace {

constexpr int MB = 128;   // tile rows
constexpr int KC = 64;    // points per K chunk (one 128-byte BF16 row)
constexpr int kMaxNB = 160;
constexpr int kParts = 3;  // BF16 parts per operand value
constexpr int kGenWarps = 8;
constexpr int kEpiWarps = 4;
constexpr int kThreads = 32 * (2 + kEpiWarps + kGenWarps);
constexpr uint32_t kTmemCols = 512;
constexpr int kTileBytes = MB * 128;             // one BF16 part of an A tile
constexpr int kSmemLimit = 232448;               // 227 KiB of opt-in shared memory per CTA
constexpr int kCS = 3;      // slots of staged point data (copied kCS - 1 chunks ahead)
constexpr int kQcBytes = KC / 2 * 12 * 4;  // one chunk's staged coordinates
constexpr int kCoordBytes = kCS * (kQcBytes + KC * 4);

// Shared-memory stages and TMEM accumulators for an NBT-column tile.  The
// tile's columns are accumulated in H units of UC = NBT / H columns; units
// (chunk group g, part h) take turns in two TMEM slots, so the tensor core
// fills one slot while the epilogue drains the other.  NBT <= 128: one unit
// per tile (a double-buffered accumulator); NBT = 160: two units of 80.
template <int NBT>
struct Cfg {
  static constexpr int kStageBytes = kParts * (kTileBytes + NBT * 128);
  static constexpr int STAGES = (kSmemLimit - 2048 - kCoordBytes) / kStageBytes >= 3 ? 3 : 2;
  static constexpr int H = 4 * NBT <= (int)kTmemCols ? 1 : 2;
  static constexpr int UC = NBT / H;
  static_assert(NBT % 32 == 0 && NBT <= kMaxNB, "tile width");
  static_assert(UC % 16 == 0 && (UC * 128) % 1024 == 0, "unit width");
  static_assert(STAGES * kStageBytes + kCoordBytes + 2048 <= kSmemLimit, "shared memory");
  // Room left for the tag rows tau(row box, :) of the tile's row boxes.
  static constexpr int kTauFloats =
      ((kSmemLimit - 2048 - STAGES * kStageBytes - kCoordBytes) / 4) & ~3;
  static_assert(2 * UC + 2 * NBT <= (int)kTmemCols, "tensor memory");
};

template <int NBT>
struct __align__(1024) Smem {
  static constexpr int STAGES = Cfg<NBT>::STAGES;
  uint8_t a[STAGES][kParts][kTileBytes];  // A h, m, l: 128 rows x 128 bytes
  uint8_t x[STAGES][kParts][NBT * 128];   // X h, m, l: NBT rows x 128 bytes
  // Point data of a chunk, bulk-copied by the producer from the staged
  // layout (one 1.5 KiB block per chunk): point pair P = 4 j + pr (points
  // 2P, 2P + 1) sits at [f][pr][j], so the 8 pairs a warp reads at once are 8
  // consecutive 16-byte words (no bank conflicts); the three float4 fields f
  // hold the negated coordinates {xh, yh}, {zh, xl}, {yl, zl} of the pair.
  // bq: the column box of each point (tag factoring).
  float4 qc[kCS][3][4][8];
  int bq[kCS][KC];
  float taus[Cfg<NBT>::kTauFloats];  // tau rows of the tile's row boxes
  uint64_t cfull[kCS], cfree[kCS];
  uint64_t full_a[STAGES], full_b[STAGES], empty[STAGES];
  uint64_t dfull[2], dempty[2], done;
  uint32_t tmem_base;
  volatile int abort;
};

struct Maps {
  CUtensorMap part[kParts];  // X h, m, l planes
};

struct MixedArgs {
  const float4 *qst;     // staged coordinates, [npad / 64][3][4][8] (see Smem::qc)
  const int32_t *boxpad; // box of each point, padded to npad with the last box
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
  volatile int *status;  // set to 1 by any timed-out wait of this launch
};

template <class SM>
__device__ __forceinline__ bool wait_or_abort(SM &S, volatile int *status, uint64_t *bar,
                                              uint32_t parity) {
  return pipe::wait_or_abort(S, status, bar, parity, &g_mixed_timeouts);
}
template <class SM>
__device__ __forceinline__ bool warp_wait(SM &S, volatile int *status, uint64_t *bar,
                                          uint32_t parity) {
  return pipe::warp_wait(S, status, bar, parity, &g_mixed_timeouts);
}
using pipe::split3;
using pipe::split3_fp64;
using pipe::warp_aborted;

template <int KERNEL, int NBT, bool TAGGED>
__global__ void __launch_bounds__(kThreads, 1)
    mixed_apply_kernel(const __grid_constant__ Maps maps, MixedArgs a) {
  extern __shared__ uint8_t smem_raw[];
  using SM = Smem<NBT>;
  constexpr int STAGES = Cfg<NBT>::STAGES, H = Cfg<NBT>::H, UC = Cfg<NBT>::UC;
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
    for (int t = 0; t < kCS; ++t) {
      tc::mbar_init(&S.cfull[t], 1);
      tc::mbar_init(&S.cfree[t], kGenWarps);
    }
    tc::mbar_init(&S.done, 1);
    tc::fence_mbar_init();
    for (int t = 0; t < kParts; ++t) tc::tma_prefetch(&maps.part[t]);
  }
  // Boxes of this tile's rows (rows are box-major, so they form a range) and
  // their tag rows tau(row box, :) in shared memory when they fit.
  const int n32 = (int)a.n;
  const int rb0 = TAGGED ? a.box_of[(int)row0] : 0;
  const int nrb = TAGGED ? a.box_of[min((int)row0 + MB, n32) - 1] - rb0 + 1 : 1;
  const bool tau_smem = TAGGED && (int64_t)nrb * a.b <= Cfg<NBT>::kTauFloats;
  if (tau_smem)
    for (int idx = tid; idx < nrb * a.b; idx += kThreads)
      S.taus[idx] = a.tau[(int64_t)rb0 * a.b + idx];
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = S.tmem_base;
  const float factor = entry_f32_factor<KERNEL>();

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    // X tiles by TMA into the stages; each chunk's staged coordinates (and
    // column boxes) by bulk copy into the point slots, kCS - 1 chunks ahead.
    if (lane == 0) {
      const uint32_t pbytes = kQcBytes + (TAGGED ? KC * 4 : 0);
      auto copy_points = [&](int cc) {
        const int cs = cc % kCS;
        tc::mbar_arrive_expect_tx(&S.cfull[cs], pbytes);
        tc::bulk_load(S.qc[cs], a.qst + (int64_t)cc * (KC / 2 * 3), kQcBytes, &S.cfull[cs]);
        if (TAGGED) tc::bulk_load(S.bq[cs], a.boxpad + (int64_t)cc * KC, KC * 4, &S.cfull[cs]);
      };
      int issued = 0, pissued = 0;
      for (; pissued < kCS - 1 && pissued < nk; ++pissued) copy_points(pissued);
      for (int c = 0; c < nk && !S.abort; ++c) {
        const int s = c % STAGES;
        const uint32_t ph = (c / STAGES) & 1;
        if (c >= STAGES && !wait_or_abort(S, a.status, &S.empty[s], ph ^ 1)) break;
        tc::mbar_arrive_expect_tx(&S.full_b[s], kParts * NBT * 128);
#pragma unroll
        for (int t = 0; t < kParts; ++t)
          tc::tma_load_2d(S.x[s][t], &maps.part[t], &S.full_b[s], c * KC, col0);
        issued = c + 1;
        if (pissued < nk) {
          // Slot of chunk pissued is free once the generators released chunk pissued - kCS.
          const int cs = pissued % kCS;
          if (pissued >= kCS && !wait_or_abort(S, a.status, &S.cfree[cs], ((pissued / kCS) & 1) ^ 1))
            break;
          copy_points(pissued++);
        }
      }
      // Copies still in flight must land before the CTA exits.
      for (int c = (issued > STAGES ? issued - STAGES : 0); c < issued; ++c)
        pipe::drain(&S.full_b[c % STAGES], (c / STAGES) & 1);
      for (int c = (pissued > kCS ? pissued - kCS : 0); c < pissued; ++c)
        pipe::drain(&S.cfull[c % kCS], (c / kCS) & 1);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(MB, UC);
      bool ok = true;
      for (int c = 0; c < nk && ok && !S.abort; ++c) {
        const int s = c % STAGES;
        const uint32_t ph = (c / STAGES) & 1;
        const int g = c / flush;
        const bool first = (c % flush) == 0;
        const bool last = (c % flush) == flush - 1 || c == nk - 1;
        if (!wait_or_abort(S, a.status, &S.full_a[s], ph)) break;
        if (!wait_or_abort(S, a.status, &S.full_b[s], ph)) break;
        tc::tc_fence_after();
        // Operand descriptors of the stage's parts; a K step of 16 BF16 (32
        // bytes) or a unit's row offset only moves the start-address field.
        uint64_t ad[kParts], bd[kParts];
#pragma unroll
        for (int t = 0; t < kParts; ++t) {
          ad[t] = tc::sw128_desc(tc::smem_u32(S.a[s][t]));
          bd[t] = tc::sw128_desc(tc::smem_u32(S.x[s][t]));
        }
#pragma unroll
        for (int h = 0; h < H; ++h) {
          const int u = g * H + h, slot = u & 1, use = u >> 1;
          // The slot is free once the epilogue drained its previous unit.
          if (first && use >= 1 && !wait_or_abort(S, a.status, &S.dempty[slot], (use - 1) & 1)) {
            ok = false;
            break;
          }
          if (first && use >= 1) tc::tc_fence_after();
          const uint32_t dt = tmem + slot * UC;
          const uint64_t boff = (uint64_t)(h * UC * 128) >> 4;
          uint32_t acc = first ? 0u : 1u;
          // (A part, X part) products, smallest first.
          constexpr int kOrder[6][2] = {{2, 0}, {1, 1}, {0, 2}, {1, 0}, {0, 1}, {0, 0}};
#pragma unroll
          for (int o = 0; o < 6; ++o) {
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk) {
              tc::mma_f16(dt, ad[kOrder[o][0]] + 2 * kk, bd[kOrder[o][1]] + boff + 2 * kk, idesc,
                          acc);
              acc = 1u;
            }
          }
          if (last) tc::mma_commit(&S.dfull[slot]);
        }
        if (!ok) break;
        tc::mma_commit(&S.empty[s]);
      }
      // Every MMA issued so far has finished once `done` completes.
      tc::mma_commit(&S.done);
      pipe::drain(&S.done, 0);
    }
    __syncwarp();
  } else if (warp < 2 + kEpiWarps) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    const uint32_t hi_t = tmem + 2 * UC + lanes, cc_t = hi_t + NBT;
    float hv[16], cv[16], dv[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) hv[t] = 0.f;
#pragma unroll
    for (int cg = 0; cg < NBT / 16; ++cg) {
      tc::tmem_st16(hi_t + cg * 16, hv);
      tc::tmem_st16(cc_t + cg * 16, hv);
    }
    tc::tmem_wait_st();
    bool ok = !warp_aborted(S);
    for (int g = 0; g < ngroups && ok; ++g) {
      for (int h = 0; h < H; ++h) {
        const int u = g * H + h, slot = u & 1;
        if (!warp_wait(S, a.status, &S.dfull[slot], (u >> 1) & 1)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const uint32_t d_t = tmem + slot * UC + lanes;
#pragma unroll 1
        for (int cg = 0; cg < UC / 16; ++cg) {
          const uint32_t col = h * UC + cg * 16;
          tc::tmem_ld16x3(d_t + cg * 16, hi_t + col, cc_t + col, dv, hv, cv);
          kahan_add16(hv, cv, dv);  // hi + (d - c); c keeps the lost low part
          tc::tmem_st16(hi_t + col, hv);
          tc::tmem_st16(cc_t + col, cv);
        }
        tc::tmem_wait_st();
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&S.dempty[slot]);
      }
    }
    if (ok) {
      const int64_t p = row0 + 32 * q + lane;
#pragma unroll 1
      for (int cg = 0; cg < NBT / 16; ++cg) {
        tc::tmem_ld16x2(hi_t + cg * 16, cc_t + cg * 16, hv, cv);
        if (p < a.n) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int64_t c = (int64_t)col0 + cg * 16 + t;
            const double val = (double)hv[t] - (double)cv[t];
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
    // Thread (j, rbase): rows rbase + 32 i (i < 4) x points 8 j .. 8 j + 7 of
    // each chunk, two points at a time in packed FP32x2 arithmetic.
    const int gt = tid - 32 * (2 + kEpiWarps);  // 0 .. 255
    const int j = gt & 7;                        // 16-byte chunk (8 points) within the 64
    const int rbase = gt >> 3;
    const int prow0 = (int)row0 + rbase;         // n < 2^30 is checked on the host
    float2 rx[4][3], lx[4][3];                   // row coordinates, hi and lo, as (v, v) pairs
    const float *trow[4];                        // tau(box of the row, :)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int p = prow0 + 32 * i;
      const int bx = (TAGGED && p < n32) ? a.box_of[p] : rb0;
      trow[i] = tau_smem ? S.taus + (bx - rb0) * a.b : a.tau + (int64_t)bx * a.b;
      // Point p in the staged layout: chunk p / 64, pair P = (p % 64) / 2 = 4 j + pr.
      const int w = p & (KC - 1), P = w >> 1, u = w & 1;
      const float4 *blk = a.qst + (int64_t)(p / KC) * (KC / 2 * 3) + (P & 3) * 8 + (P >> 2);
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 f0 = p < n32 ? blk[0] : z4, f1 = p < n32 ? blk[32] : z4;
      const float4 f2 = p < n32 ? blk[64] : z4;
      const float v[6] = {u ? f0.y : f0.x, u ? f0.w : f0.z, u ? f1.y : f1.x,
                          u ? f1.w : f1.z, u ? f2.y : f2.x, u ? f2.w : f2.z};
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        rx[i][ax] = make_float2(-v[ax], -v[ax]);
        lx[i][ax] = make_float2(-v[3 + ax], -v[3 + ax]);
      }
    }
    const float2 f2 = make_float2(factor, factor);
    for (int c = 0; c < nk && !warp_aborted(S); ++c) {
      const int s = c % STAGES, cs = c % kCS;
      const uint32_t ph = (c / STAGES) & 1;
      if (c >= STAGES && !warp_wait(S, a.status, &S.empty[s], ph ^ 1)) break;
      if (!warp_wait(S, a.status, &S.cfull[cs], (c / kCS) & 1)) break;
      // A chunk that cannot meet the diagonal or the ragged edge needs no
      // per-entry checks (the test is uniform over the CTA).
      const int kc0 = c * KC;
      const bool clean = (kc0 + KC <= (int)row0 || kc0 >= (int)row0 + MB) && kc0 + KC <= n32 &&
                         (int)row0 + MB <= n32;
      // Tag weights: a chunk inside one column box has one weight per row.
      int bq0 = 0;
      bool one_box = true;
      if (TAGGED) {
        bq0 = S.bq[cs][0];
        one_box = bq0 == S.bq[cs][KC - 1];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = rbase + 32 * i, p = prow0 + 32 * i;
        uint32_t pw[kParts][4];
        float wrow = factor;
        if (TAGGED && one_box) wrow = factor * trow[i][bq0];
#pragma unroll
        for (int pr = 0; pr < 4; ++pr) {
          const int P = 4 * j + pr;  // point pair within the chunk
          const float4 q0 = S.qc[cs][0][pr][j], q1 = S.qc[cs][1][pr][j], q2 = S.qc[cs][2][pr][j];
          const float2 dx = __fadd2_rn(__fadd2_rn(rx[i][0], make_float2(q0.x, q0.y)),
                                       __fadd2_rn(lx[i][0], make_float2(q1.z, q1.w)));
          const float2 dy = __fadd2_rn(__fadd2_rn(rx[i][1], make_float2(q0.z, q0.w)),
                                       __fadd2_rn(lx[i][1], make_float2(q2.x, q2.y)));
          float2 r2;
          if (KERNEL == TBLR_KERNEL_LAPLACE3D) {
            const float2 dz = __fadd2_rn(__fadd2_rn(rx[i][2], make_float2(q1.x, q1.y)),
                                         __fadd2_rn(lx[i][2], make_float2(q2.z, q2.w)));
            r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
          } else {
            r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
          }
          const float2 e = make_float2(entry_f32_of_r2<KERNEL>(r2.x), entry_f32_of_r2<KERNEL>(r2.y));
          float2 w = f2;
          if (TAGGED) {
            if (one_box)
              w = make_float2(wrow, wrow);
            else
              w = make_float2(factor * trow[i][S.bq[cs][2 * P]], factor * trow[i][S.bq[cs][2 * P + 1]]);
          }
          float2 v = __fmul2_rn(e, w);
          if (!clean) {
            const int qq = kc0 + 2 * P;
            if (qq == p || qq >= n32 || p >= n32) v.x = 0.f;
            if (qq + 1 == p || qq + 1 >= n32 || p >= n32) v.y = 0.f;
          }
          split3(v.x, v.y, pw[0][pr], pw[1][pr], pw[2][pr]);
        }
        const int off = r * 128 + ((j ^ (r & 7)) << 4);  // 128-byte swizzle
#pragma unroll
        for (int t = 0; t < kParts; ++t)
          *reinterpret_cast<uint4 *>(S.a[s][t] + off) =
              make_uint4(pw[t][0], pw[t][1], pw[t][2], pw[t][3]);
      }
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(&S.cfree[cs]);
        tc::mbar_arrive(&S.full_a[s]);
      }
    }
  }

  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// Coordinates as negated double-float pairs (x = hi + lo to ~48 bits) in the
// staged layout the tensor-core kernel copies per chunk: chunk c, point pair
// P = 4 j + pr at qst[c][f][pr][j] with f = {xh, yh}, {zh, xl}, {yl, zl} for
// the pair (points past n are zero), and the box of each point padded to npad
// with the last box.
__global__ void stage_coords_kernel(const double *__restrict__ pts, const int32_t *__restrict__ box_of,
                                    int64_t n, int64_t npad, int d, float4 *__restrict__ qst,
                                    int32_t *__restrict__ boxpad) {
  const int64_t npairs = npad / 2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < npairs;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / (KC / 2);
    const int P = (int)(t % (KC / 2)), j = P >> 2, pr = P & 3;
    float h[2][3], l[2][3];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t p = 2 * t + u;
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        h[u][ax] = l[u][ax] = 0.f;
        if (ax < d && p < n) {
          const double x = pts[ax * n + p];
          h[u][ax] = (float)x;
          l[u][ax] = (float)(x - (double)h[u][ax]);
        }
      }
      if (boxpad) boxpad[p] = box_of[p < n ? p : n - 1];
    }
    float4 *blk = qst + c * (KC / 2 * 3) + pr * 8 + j;
    blk[0] = make_float4(-h[0][0], -h[1][0], -h[0][1], -h[1][1]);
    blk[32] = make_float4(-h[0][2], -h[1][2], -l[0][0], -l[1][0]);
    blk[64] = make_float4(-l[0][1], -l[1][1], -l[0][2], -l[1][2]);
  }
}

// X (FP64, K-major [ncols][n]) split into BF16 h/m/l planes [ncols_pad][npad],
// zero padded.
__global__ void split_x_kernel(const double *__restrict__ xt, int64_t n, int64_t ncols,
                               int64_t npad, int64_t ncols_pad, __nv_bfloat16 *__restrict__ xh,
                               __nv_bfloat16 *__restrict__ xm, __nv_bfloat16 *__restrict__ xl) {
  const int64_t total = npad * ncols_pad;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / npad, p = i % npad;
    const double v = (c < ncols && p < n) ? xt[c * n + p] : 0.0;
    split3_fp64(v, xh[i], xm[i], xl[i]);
  }
}

int make_map(CUtensorMap *map, const __nv_bfloat16 *base, int64_t npad, int64_t rows,
             int box_rows) {
  return pipe::make_plane_map(map, base, npad, rows, box_rows);
}

// Column tiling of `ncols` outputs: the fewest tiles of at most 160 columns,
// of equal width rounded up to a multiple of 32 (the black-box apply uses
// widths 128 and 160 only).
struct ColTiles {
  int width, ntiles;
  int64_t padded;
};

ColTiles col_tiles(int64_t ncols, bool tagged) {
  ColTiles t;
  t.ntiles = (int)cdiv(std::max<int64_t>(ncols, 1), kMaxNB);
  t.width = (int)(cdiv(cdiv(std::max<int64_t>(ncols, 1), t.ntiles), 32) * 32);
  if (!tagged) t.width = t.width <= 128 ? 128 : kMaxNB;
  t.padded = (int64_t)t.width * t.ntiles;
  return t;
}

// Tile widths of the tag-factored sketch and the ones a tuner may try for
// `ncols` columns: at most 64 padded columns beyond the 32-column round-up.
constexpr int kTagWidths[5] = {32, 64, 96, 128, 160};
bool tagged_width_ok(int64_t ncols, int w) {
  return cdiv(std::max<int64_t>(ncols, 1), w) * w <= cdiv(std::max<int64_t>(ncols, 1), 32) * 32 + 64;
}
int64_t tagged_padded_max(int64_t ncols) {
  int64_t mx = col_tiles(ncols, true).padded;
  for (int w : kTagWidths)
    if (tagged_width_ok(ncols, w)) mx = std::max<int64_t>(mx, cdiv(std::max<int64_t>(ncols, 1), w) * w);
  return mx;
}
ColTiles col_tiles_w(int64_t ncols, int w) {
  ColTiles t;
  t.width = w;
  t.ntiles = (int)cdiv(std::max<int64_t>(ncols, 1), w);
  t.padded = (int64_t)w * t.ntiles;
  return t;
}

// Tile widths picked by tblr_tune_tagged_sketch, per (kernel, columns, size
// class floor(log2 n)), for this process; a width forced by the tuner while it
// times the candidates (this thread only).
std::mutex g_tune_mu;
std::map<std::tuple<int, int64_t, int>, int> g_tune;
thread_local int t_force_width = 0;
int size_class(int64_t n) {
  int c = 0;
  while (c < 62 && ((int64_t)1 << (c + 1)) <= n) ++c;
  return c;
}
int chosen_width(const Prob &P, int64_t ncols) {
  if (t_force_width) return t_force_width;
  std::lock_guard<std::mutex> g(g_tune_mu);
  const auto it = g_tune.find(std::make_tuple(P.kernel, ncols, size_class(P.n)));
  return it == g_tune.end() ? 0 : it->second;
}

struct MixedLayout {
  int64_t npad, ncols_pad;
  size_t head, coords, planes, tau, boxes, total;
};

MixedLayout mixed_layout(const Prob &P, int64_t ncols, bool tagged) {
  MixedLayout L;
  L.npad = cdiv(P.n, KC) * KC;
  L.ncols_pad = tagged ? tagged_padded_max(ncols) : col_tiles(ncols, false).padded;
  L.head = 256;
  L.coords = align256(sizeof(float) * 2 * 3 * L.npad);
  L.planes = align256(sizeof(__nv_bfloat16) * L.npad * L.ncols_pad);
  L.tau = tagged ? align256(sizeof(float) * P.b * P.b) : 0;
  L.boxes = tagged ? align256(sizeof(int32_t) * L.npad) : 0;
  L.total = L.head + L.coords + kParts * L.planes + L.tau + L.boxes;
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

// [G | H] (or G alone: ncols = r) gathered to box-major order and split into
// BF16 h/m/l planes [ncols_pad][npad] (rows c < r from G, r <= c < ncols from
// H, zero padded).
__global__ void split_gh_kernel(const double *__restrict__ G, const double *__restrict__ H,
                                const int32_t *__restrict__ perm, int64_t n, int r, int64_t ncols,
                                int64_t npad, int64_t ncols_pad, __nv_bfloat16 *__restrict__ xh,
                                __nv_bfloat16 *__restrict__ xm, __nv_bfloat16 *__restrict__ xl) {
  const int64_t total = npad * ncols_pad;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / npad, p = i % npad;
    double v = 0.0;
    if (p < n && c < ncols) {
      const int64_t src = (int64_t)perm[p] * r + (c < r ? c : c - r);
      v = c < r ? G[src] : H[src];
    }
    split3_fp64(v, xh[i], xm[i], xl[i]);
  }
}

__global__ void tau_to_f32(const double *__restrict__ tau, int64_t len, float *__restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)tau[i];
}

template <int KERNEL, int NBT, bool TAGGED>
int launch_mixed(const Maps &maps, const MixedArgs &a, int64_t n, int ntiles, cudaStream_t s) {
  auto k = mixed_apply_kernel<KERNEL, NBT, TAGGED>;
  const size_t smem = sizeof(Smem<NBT>) + 1024;
  TBLR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k<<<dim3((unsigned)cdiv(n, MB), (unsigned)ntiles), kThreads, smem, s>>>(maps, a);
  return launch_status("mixed_apply_kernel");
}

template <bool TAGGED>
int dispatch_mixed(int kernel, int width, const Maps &maps, const MixedArgs &a, int64_t n,
                   int ntiles, cudaStream_t s) {
#define TBLR_MIXED_CASE(W)                                                                     \
  if (width == W)                                                                              \
    return kernel == TBLR_KERNEL_LAPLACE2D                                                     \
               ? launch_mixed<TBLR_KERNEL_LAPLACE2D, W, TAGGED>(maps, a, n, ntiles, s)         \
               : launch_mixed<TBLR_KERNEL_LAPLACE3D, W, TAGGED>(maps, a, n, ntiles, s);
  if constexpr (TAGGED) {
    TBLR_MIXED_CASE(32)
    TBLR_MIXED_CASE(64)
    TBLR_MIXED_CASE(96)
  }
  TBLR_MIXED_CASE(128)
  TBLR_MIXED_CASE(160)
#undef TBLR_MIXED_CASE
  set_error("no tensor-core kernel for tile width %d", width);
  return TBLR_EUNSUPPORTED;
}

MixedArgs base_args(const Prob &P, const MixedLayout &L, const float4 *qst, const int32_t *boxpad,
                    volatile int *status) {
  MixedArgs a{};
  a.qst = qst;
  a.boxpad = boxpad;
  a.n = P.n;
  a.npad = L.npad;
  a.d = P.d;
  a.kernel = P.kernel;
  a.nk = (int)(L.npad / KC);
  a.flush = env_flush();
  a.status = status;
  return a;
}

// The three X planes of the workspace and their tensor maps.
struct Planes {
  __nv_bfloat16 *part[kParts];
};

Planes planes_of(char *w, const MixedLayout &L) {
  Planes pl;
  for (int t = 0; t < kParts; ++t)
    pl.part[t] = reinterpret_cast<__nv_bfloat16 *>(w + L.head + L.coords + t * L.planes);
  return pl;
}

int make_maps(Maps *maps, const Planes &pl, const MixedLayout &L, int width) {
  for (int t = 0; t < kParts; ++t)
    TBLR_TRY(make_map(&maps->part[t], pl.part[t], L.npad, L.ncols_pad, width));
  return TBLR_OK;
}

}  // namespace

size_t mixed_workspace(const Prob &P, int64_t ncols) { return mixed_layout(P, ncols, false).total; }
size_t tagged_mixed_workspace(const Prob &P) {
  return mixed_layout(P, (P.selfadjoint ? 1 : 2) * P.r, true).total;
}

int apply_mixed(const Prob &P, const tblr_layout *lay, const double *xt, int64_t ncols, double *y,
                int64_t ldy, void *ws, size_t ws_bytes, cudaStream_t s) {
  TBLR_REQUIRE(P.kernel == TBLR_KERNEL_LAPLACE2D || P.kernel == TBLR_KERNEL_LAPLACE3D,
               "mixed precision supports the built-in Laplace kernels");
  TBLR_REQUIRE(P.n < (int64_t)1 << 30, "mixed precision supports n < 2^30 points");
  const MixedLayout L = mixed_layout(P, ncols, false);
  TBLR_REQUIRE(ws != nullptr && ws_bytes >= L.total, "mixed workspace too small (%zu < %zu)",
               ws_bytes, L.total);
  TBLR_REQUIRE((reinterpret_cast<uintptr_t>(ws) & 255) == 0, "workspace must be 256-byte aligned");
  char *w = static_cast<char *>(ws);
  int *status = reinterpret_cast<int *>(w);
  float4 *qst = reinterpret_cast<float4 *>(w + L.head);
  const Planes pl = planes_of(w, L);
  TBLR_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
  stage_coords_kernel<<<(unsigned)std::min<int64_t>(cdiv(L.npad / 2, 256), 4096), 256, 0, s>>>(
      lay->pts, lay->box_of, P.n, L.npad, P.d, qst, nullptr);
  TBLR_TRY(launch_status("stage_coords_kernel"));
  split_x_kernel<<<(unsigned)std::min<int64_t>(cdiv(L.npad * L.ncols_pad, 256), 152 * 32), 256, 0,
                   s>>>(xt, P.n, ncols, L.npad, L.ncols_pad, pl.part[0], pl.part[1], pl.part[2]);
  TBLR_TRY(launch_status("split_x_kernel"));
  const ColTiles ct = col_tiles(ncols, false);
  Maps maps;
  TBLR_TRY(make_maps(&maps, pl, L, ct.width));
  MixedArgs a = base_args(P, L, qst, nullptr, status);
  a.ncols = ncols;
  a.ldy = ldy;
  a.y = y;
  a.split = ncols;
  a.ldy2 = 0;
  a.y2 = nullptr;
  return dispatch_mixed<false>(P.kernel, ct.width, maps, a, P.n, ct.ntiles, s);
}

int tagged_sketch_mixed(const Prob &P, const tblr_layout *lay, const double *tau, const double *G,
                        const double *H, double *S, double *R, void *ws, size_t ws_bytes,
                        cudaStream_t s) {
  TBLR_REQUIRE(P.kernel == TBLR_KERNEL_LAPLACE2D || P.kernel == TBLR_KERNEL_LAPLACE3D,
               "mixed precision supports the built-in Laplace kernels");
  TBLR_REQUIRE(P.n < (int64_t)1 << 30, "mixed precision supports n < 2^30 points");
  TBLR_REQUIRE(P.b * P.b < (int64_t)1 << 31, "too many boxes for the tag table");
  // Self-adjoint (H = G): only S = A' G, r columns.
  const int64_t ncols = (P.selfadjoint ? 1 : 2) * P.r;
  const MixedLayout L = mixed_layout(P, ncols, true);
  TBLR_REQUIRE(ws != nullptr && ws_bytes >= L.total, "tagged sketch workspace too small");
  TBLR_REQUIRE((reinterpret_cast<uintptr_t>(ws) & 255) == 0, "workspace must be 256-byte aligned");
  char *w = static_cast<char *>(ws);
  int *status = reinterpret_cast<int *>(w);
  float4 *qst = reinterpret_cast<float4 *>(w + L.head);
  const Planes pl = planes_of(w, L);
  float *tf = reinterpret_cast<float *>(w + L.head + L.coords + kParts * L.planes);
  int32_t *boxpad = reinterpret_cast<int32_t *>(w + L.head + L.coords + kParts * L.planes + L.tau);
  TBLR_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
  stage_coords_kernel<<<(unsigned)std::min<int64_t>(cdiv(L.npad / 2, 256), 4096), 256, 0, s>>>(
      lay->pts, lay->box_of, P.n, L.npad, P.d, qst, boxpad);
  TBLR_TRY(launch_status("stage_coords_kernel"));
  split_gh_kernel<<<(unsigned)std::min<int64_t>(cdiv(L.npad * L.ncols_pad, 256), 152 * 32), 256, 0,
                    s>>>(G, H, lay->perm, P.n, P.r, ncols, L.npad, L.ncols_pad, pl.part[0],
                         pl.part[1], pl.part[2]);
  TBLR_TRY(launch_status("split_gh_kernel"));
  tau_to_f32<<<(unsigned)std::min<int64_t>(cdiv(P.b * P.b, 256), 1024), 256, 0, s>>>(tau, P.b * P.b,
                                                                                     tf);
  TBLR_TRY(launch_status("tau_to_f32"));
  const int tw = chosen_width(P, ncols);
  const ColTiles ct = tw ? col_tiles_w(ncols, tw) : col_tiles(ncols, true);
  Maps maps;
  TBLR_TRY(make_maps(&maps, pl, L, ct.width));
  MixedArgs a = base_args(P, L, qst, boxpad, status);
  a.ncols = ncols;
  a.ldy = P.r;
  a.y = S;
  a.split = P.r;  // self-adjoint: ncols = r, every column goes to S
  a.ldy2 = P.r;
  a.y2 = P.selfadjoint ? nullptr : R;
  a.tau = tf;
  a.box_of = lay->box_of;
  a.b = (int)P.b;
  return dispatch_mixed<true>(P.kernel, ct.width, maps, a, P.n, ct.ntiles, s);
}

}  // namespace tblr

namespace {
// Resets the forced width however the tuner leaves its loop.
struct ForceWidth {
  explicit ForceWidth(int w) { tblr::t_force_width = w; }
  ~ForceWidth() { tblr::t_force_width = 0; }
};
}  // namespace

extern "C" int tblr_tune_tagged_sketch(const tblr_problem *prob, const tblr_layout *lay,
                                       const double *tau, const double *G, const double *H,
                                       double *s_out, double *r_out, void *ws, size_t ws_bytes,
                                       int32_t *width, void *stream) {
  using namespace tblr;
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_TRY(check_layout(P, lay));
  TBLR_REQUIRE(P.precision == TBLR_MIXED &&
                   (P.kernel == TBLR_KERNEL_LAPLACE2D || P.kernel == TBLR_KERNEL_LAPLACE3D),
               "tuning applies to the mixed-precision sketch of the built-in kernels");
  TBLR_REQUIRE(tau && G && s_out && width && (P.selfadjoint || (H && r_out)),
               "tau, G, s, width (and, unless self-adjoint, H and rr) must be non-NULL");
  TBLR_REQUIRE(ws != nullptr && ws_bytes >= tagged_mixed_workspace(P),
               "tagged sketch workspace too small");
  cudaStream_t s = as_stream(stream);
  const int64_t ncols = (P.selfadjoint ? 1 : 2) * P.r;
  cudaEvent_t e0, e1;
  TBLR_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    set_error("cudaEventCreate failed");
    return TBLR_ECUDA;
  }
  int best = 0, st = TBLR_OK;
  float best_ms = 0.f;
  for (int w : kTagWidths) {
    if (!tagged_width_ok(ncols, w)) continue;
    ForceWidth force(w);
    st = tagged_sketch_mixed(P, lay, tau, G, H, s_out, r_out, ws, ws_bytes, s);  // warm-up
    if (st == TBLR_OK && cudaEventRecord(e0, s) != cudaSuccess) st = TBLR_ECUDA;
    for (int rep = 0; rep < 2 && st == TBLR_OK; ++rep)
      st = tagged_sketch_mixed(P, lay, tau, G, H, s_out, r_out, ws, ws_bytes, s);
    float ms = 0.f;
    if (st == TBLR_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                          cudaEventSynchronize(e1) != cudaSuccess ||
                          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = TBLR_ECUDA;
    if (st != TBLR_OK) break;
    if (best == 0 || ms < best_ms) {
      best = w;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != TBLR_OK) return st;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[std::make_tuple(P.kernel, ncols, size_class(P.n))] = best;
  }
  *width = best;
  // Leave the chosen width's result in s (and rr).
  return tagged_sketch_mixed(P, lay, tau, G, H, s_out, r_out, ws, ws_bytes, s);
}

extern "C" int tblr_tuned_width(const tblr_problem *prob, int32_t *width) {
  using namespace tblr;
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_REQUIRE(width != nullptr, "width is NULL");
  *width = chosen_width(P, (P.selfadjoint ? 1 : 2) * P.r);
  return TBLR_OK;
}

extern "C" void tblr_tune_clear(void) {
  std::lock_guard<std::mutex> g(tblr::g_tune_mu);
  tblr::g_tune.clear();
}

extern "C" int tblr_device_timeouts(unsigned int *count) {
  TBLR_REQUIRE(count != nullptr, "count is NULL");
  unsigned int zero = 0;
  TBLR_CUDA(cudaDeviceSynchronize());
  TBLR_CUDA(cudaMemcpyFromSymbol(count, tblr::g_mixed_timeouts, sizeof(unsigned int)));
  TBLR_CUDA(cudaMemcpyToSymbol(tblr::g_mixed_timeouts, &zero, sizeof(unsigned int)));
  *count += tblr::coupling_tc_take_timeouts();
  return TBLR_OK;
}
