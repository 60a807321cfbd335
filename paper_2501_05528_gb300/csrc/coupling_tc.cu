// Coupling blocks Atilde_ij = U_i^T (A_ij V_j) (§2.5, Table 1 step 2) of the
// mixed-precision path on tcgen05 tensor cores (sm_103a).
//
// W = A_ij V_j is the dense contraction.  For every 128-row tile of box i the
// CTA generates the kernel tile A(rows, chunk of box j) chunk by chunk (64
// points), splits it and the chunk's rows of V_j into three BF16 parts each and
// accumulates the six significant part products in TMEM, small ones first, as
// the mixed apply does (same error budget: ~2^-24 per operand, truncation only
// at the size of one chunk's sum).  The generated tile goes straight into
// tensor memory and is the MMA's A operand there, so the tensor core reads only
// the V tile from shared memory.  Each chunk's FP32 accumulator is added into
// a Kahan-compensated copy of W in TMEM.  After a row tile the epilogue warps
// stage W and the tile's rows of U_i (FP32) in shared memory and add
// U_i(tile)^T W into Kahan-compensated sums of Atilde_ij, spread over the
// drain steps of the next tile.
//
// The points of every box are padded to a multiple of 64 in a box-padded order
// (box j starts at poff[j]), so each chunk's V rows are one 64-point TMA tile
// at an aligned coordinate and its coordinates one 1.5 KiB bulk copy.
//
// CTA per box pair (i, j), 448 threads:
//   warp 0      producer: V_j tiles (TMA) and chunk coordinates (bulk copies)
//   warp 1      TMEM allocator and single-thread MMA issuer
//   warps 2-5   epilogue: W sums in TMEM, then U_i^T W
//   warps 6-13  generators: the 128 x 64 kernel tile, written into TMEM
// Every wait is bounded; a timeout is counted (tblr_device_timeouts), sets
// the launch's status word and the CTA drains and exits.
#include <algorithm>

#include "coupling_tc.cuh"
#include "kernels_f32.cuh"
#include "tc_pipeline.cuh"
#include "tc_utils.cuh"

namespace tblr {

static __device__ unsigned int g_coupling_timeouts;

namespace {

constexpr int MB = 128;    // tile rows (points of box i)
constexpr int KC = 64;     // points of box j per chunk
constexpr int kParts = 3;  // BF16 parts per operand value
constexpr int kGenWarps = 8;
constexpr int kEpiWarps = 4;
constexpr int kThreads = 32 * (2 + kEpiWarps + kGenWarps);
constexpr int kSmemLimit = 232448;    // 227 KiB of opt-in shared memory per CTA
constexpr int kCS = 3;                // chunk coordinate slots (copied kCS - 1 ahead)
constexpr int kQcBytes = KC / 2 * 12 * 4;

template <int KP>
struct CplCfg {
  static constexpr int RS = KP + 4;  // row stride of W and U in shared memory (floats)
  static constexpr int AC = KP >= 32 ? 4 : 2;     // Atilde columns per epilogue thread
  static constexpr int AA = KP * KP / (MB * AC);  // Atilde rows per epilogue thread
  static constexpr int NTC = KP / AC;             // epilogue threads across Atilde's columns
  static constexpr int NACC = AA * AC;
  // Each epilogue thread's Atilde sums and compensations live in its own TMEM
  // lane when there are 16 or more of them (registers would spill).
  static constexpr bool kAccTmem = NACC >= 16;
  // TMEM columns: two accumulator slots [0, 2 KP), W's sum and compensation
  // [2 KP, 4 KP), the Atilde sums, then the kernel-tile stages from kABase:
  // three BF16 parts of 32 columns each (64 points, two per 32-bit column).
  static constexpr uint32_t kTmemCols = 512;
  static constexpr uint32_t kAStage = kParts * (KC / 2);
  static constexpr uint32_t kABase = (4 * KP + (kAccTmem ? 2 * NACC : 0) + 31) / 32 * 32;
  static constexpr int STAGES = (kTmemCols - kABase) / kAStage >= 3 ? 3 : 2;
  static constexpr int kStageBytes = kParts * KP * 128;  // the V_j tile
  static constexpr int kFixed = 2048 + kCS * kQcBytes + MB * (RS + KP) * 4;
  static_assert(KP == 16 || KP == 32 || KP == 64, "rank tile");
  static_assert(kABase + STAGES * kAStage <= kTmemCols, "tensor memory");
  static_assert(STAGES * kStageBytes + kFixed <= kSmemLimit, "shared memory");
  static_assert(AA * AC * MB == KP * KP, "Atilde tiling");
  static_assert(!kAccTmem || NACC % 16 == 0, "Atilde sums in TMEM groups of 16");
};

template <int KP>
struct __align__(1024) CplSmem {
  static constexpr int STAGES = CplCfg<KP>::STAGES, RS = CplCfg<KP>::RS;
  uint8_t x[STAGES][kParts][KP * 128];    // V_j h, m, l: KP rows x 128 bytes
  float4 qc[kCS][3][4][8];                // chunk coordinates (the mixed apply's layout)
  float w[MB][RS];                        // W of the finished row tile
  float u[MB][KP];                        // U_i rows of the tile (one bulk copy)
  uint64_t cfull[kCS], cfree[kCS];
  uint64_t full_a[STAGES], full_b[STAGES], empty[STAGES];
  uint64_t dfull[2], dempty[2], done, ufull;
  uint32_t tmem_base;
  volatile int abort;
};

struct CplMaps {
  CUtensorMap part[kParts];  // V h, m, l planes [KP][npb]
};

struct CplArgs {
  const float4 *qst;       // box-padded staged coordinates, [npb / 64][3][4][8]
  const int32_t *offsets;  // b + 1 point offsets of the boxes
  const int32_t *poff;     // b + 1 box-padded offsets (multiples of 64)
  const int32_t *ranks;
  // U in FP32 in the box-padded order, rows of KP (zero past the rank and in
  // padding slots), with MB spare rows at the end.
  const float *u;
  int k, b, sym;
  double *at;
  volatile int *status;
};

__device__ __forceinline__ void epi_sync() {
  asm volatile("bar.sync 1, %0;\n" ::"n"(32 * kEpiWarps) : "memory");
}

template <int KERNEL, int KP>
__global__ void __launch_bounds__(kThreads, 1)
    coupling_tc_kernel(const __grid_constant__ CplMaps maps, CplArgs a) {
  extern __shared__ uint8_t smem_raw[];
  using SM = CplSmem<KP>;
  using C = CplCfg<KP>;
  constexpr int STAGES = C::STAGES, AA = C::AA, AC = C::AC, NTC = C::NTC, NACC = C::NACC;
  SM &S = *reinterpret_cast<SM *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                  ~uintptr_t(1023));
  const int i = blockIdx.x, j = blockIdx.y;
  // Self-adjoint (V = U, A = A^T): CTA (i, j), i < j, also writes Atilde_ji = Atilde_ij^T.
  if (a.sym && i > j) return;
  const bool mirror = a.sym && i != j;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int oi = a.offsets[i], mi = a.offsets[i + 1] - oi;
  const int oj = a.offsets[j], mj = a.offsets[j + 1] - oj;
  const int ki = a.ranks[i], kj = a.ranks[j], k = a.k;
  double *out = a.at + ((int64_t)i * a.b + j) * k * k;
  double *out_t = a.at + ((int64_t)j * a.b + i) * k * k;
  if (ki == 0 || kj == 0 || mi == 0 || mj == 0) {
    for (int idx = tid; idx < k * k; idx += kThreads) {
      out[idx] = 0.0;
      if (mirror) out_t[idx] = 0.0;
    }
    return;
  }
  const int pi = a.poff[i], pj = a.poff[j];
  const int nch = (mj + KC - 1) / KC, ntiles = (mi + MB - 1) / MB;
  const int nsteps = nch * ntiles;  // step st: row tile st / nch, chunk st % nch
  unsigned int *timeouts = &g_coupling_timeouts;

  if (warp == 1) {
    tc::tmem_alloc(&S.tmem_base, C::kTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    S.abort = *a.status;  // a launch that already timed out elsewhere skips its work
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
    tc::mbar_init(&S.ufull, 1);
    tc::fence_mbar_init();
    for (int t = 0; t < kParts; ++t) tc::tma_prefetch(&maps.part[t]);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      auto copy_points = [&](int st) {
        const int cs = st % kCS;
        tc::mbar_arrive_expect_tx(&S.cfull[cs], kQcBytes);
        tc::bulk_load(S.qc[cs], a.qst + (int64_t)(pj / KC + st % nch) * (KC / 2 * 3), kQcBytes,
                      &S.cfull[cs]);
      };
      int issued = 0, pissued = 0;
      for (; pissued < kCS - 1 && pissued < nsteps; ++pissued) copy_points(pissued);
      for (int st = 0; st < nsteps && !S.abort; ++st) {
        const int s = st % STAGES;
        const uint32_t ph = (st / STAGES) & 1;
        if (st >= STAGES && !pipe::wait_or_abort(S, a.status, &S.empty[s], ph ^ 1, timeouts)) break;
        tc::mbar_arrive_expect_tx(&S.full_b[s], kParts * KP * 128);
#pragma unroll
        for (int t = 0; t < kParts; ++t)
          tc::tma_load_2d(S.x[s][t], &maps.part[t], &S.full_b[s], pj + (st % nch) * KC, 0);
        issued = st + 1;
        if (pissued < nsteps) {
          const int cs = pissued % kCS;
          if (pissued >= kCS &&
              !pipe::wait_or_abort(S, a.status, &S.cfree[cs], ((pissued / kCS) & 1) ^ 1, timeouts))
            break;
          copy_points(pissued++);
        }
      }
      // Copies still in flight must land before the CTA exits.
      for (int st = issued > STAGES ? issued - STAGES : 0; st < issued; ++st)
        pipe::drain(&S.full_b[st % STAGES], (st / STAGES) & 1);
      for (int st = pissued > kCS ? pissued - kCS : 0; st < pissued; ++st)
        pipe::drain(&S.cfull[st % kCS], (st / kCS) & 1);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(MB, KP);
      for (int st = 0; st < nsteps && !S.abort; ++st) {
        const int s = st % STAGES;
        const uint32_t ph = (st / STAGES) & 1;
        const int slot = st & 1, use = st >> 1;
        if (!pipe::wait_or_abort(S, a.status, &S.full_a[s], ph, timeouts)) break;
        if (!pipe::wait_or_abort(S, a.status, &S.full_b[s], ph, timeouts)) break;
        // The slot is free once the epilogue drained its previous chunk.
        if (use >= 1 && !pipe::wait_or_abort(S, a.status, &S.dempty[slot], (use - 1) & 1, timeouts))
          break;
        tc::tc_fence_after();
        // A parts in TMEM (a K step of 16 BF16 is 8 columns), V parts in shared
        // memory (a K step is 32 bytes: 2 in the descriptor's address field).
        uint32_t at[kParts];
        uint64_t bd[kParts];
#pragma unroll
        for (int t = 0; t < kParts; ++t) {
          at[t] = tmem + C::kABase + s * C::kAStage + t * (KC / 2);
          bd[t] = tc::sw128_desc(tc::smem_u32(S.x[s][t]));
        }
        const uint32_t dt = tmem + slot * KP;
        uint32_t acc = 0u;
        // (A part, V part) products, smallest first.
        constexpr int kOrder[6][2] = {{2, 0}, {1, 1}, {0, 2}, {1, 0}, {0, 1}, {0, 0}};
#pragma unroll
        for (int o = 0; o < 6; ++o) {
#pragma unroll
          for (int kk = 0; kk < KC / 16; ++kk) {
            tc::mma_f16_ts(dt, at[kOrder[o][0]] + 8 * kk, bd[kOrder[o][1]] + 2 * kk, idesc, acc);
            acc = 1u;
          }
        }
        tc::mma_commit(&S.dfull[slot]);
        tc::mma_commit(&S.empty[s]);
      }
      tc::mma_commit(&S.done);
      pipe::drain(&S.done, 0);
    }
    __syncwarp();
  } else if (warp < 2 + kEpiWarps) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    const uint32_t hi_t = tmem + 2 * KP + lanes, cc_t = hi_t + KP;
    const int r = 32 * q + lane;  // tile row drained by this thread
    const int et = tid - 64;      // 0 .. 127
    const int ta = et / NTC, tcol = et % NTC;  // Atilde rows AA ta .., columns AC tcol ..
    // Atilde(AA ta + x, AC tcol + y) = sum - compensation, entry e = AC x + y:
    // in registers, or in TMEM columns acc_t + e (sum) and acc_t + NACC + e.
    constexpr int NR = C::kAccTmem ? 1 : NACC;
    float rhi[NR], rcc[NR], tacc[NACC];
#pragma unroll
    for (int e = 0; e < NR; ++e) rhi[e] = rcc[e] = 0.f;
    const uint32_t acc_t = tmem + 4 * KP + lanes;
    if constexpr (C::kAccTmem) {
      float z[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) z[e] = 0.f;
#pragma unroll
      for (int g = 0; g < 2 * NACC / 16; ++g) tc::tmem_st16(acc_t + 16 * g, z);
      tc::tmem_wait_st();
    }
    // Adds tacc into the compensated sums and clears it.
    auto fold = [&]() {
      if constexpr (C::kAccTmem) {
#pragma unroll
        for (int g = 0; g < NACC / 16; ++g) {
          float hv[16], cv[16];
          tc::tmem_ld16x2(acc_t + 16 * g, acc_t + NACC + 16 * g, hv, cv);
          float tv[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) tv[e] = tacc[16 * g + e];
          kahan_add16(hv, cv, tv);
          tc::tmem_st16(acc_t + 16 * g, hv);
          tc::tmem_st16(acc_t + NACC + 16 * g, cv);
        }
        tc::tmem_wait_st();
      } else {
#pragma unroll
        for (int e = 0; e < NACC; ++e) kahan_add(rhi[e], rcc[e], tacc[e]);
      }
#pragma unroll
      for (int e = 0; e < NACC; ++e) tacc[e] = 0.f;
    };
    bool ok = !pipe::warp_aborted(S);
    // U_i rows of row tile tt: one bulk copy of MB rows of KP floats.
    constexpr uint32_t kUBytes = MB * KP * 4;
    auto copy_u = [&](int tt) {
      tc::mbar_arrive_expect_tx(&S.ufull, kUBytes);
      tc::bulk_load(&S.u[0][0], a.u + (int64_t)(pi + MB * tt) * KP, kUBytes, &S.ufull);
    };
    int u_issued = 0;
    // U_i(tile)^T W of a finished tile is spread over the drain steps of the
    // next tile ("pieces" of prows rows after a slot has been released), so
    // the epilogue keeps draining accumulator slots on time.  pend = the tile
    // whose W sits in S.w (-1: none), prow = its next row; u_tile = the last
    // tile whose U_i rows were requested into S.u (issued as soon as the
    // pending reduction no longer reads S.u, one step or more ahead of use).
    int pend = -1, prow = 0, pend_rows = 0, prows = MB, u_tile = 0;
    bool u_ready = false;
    if (et == 0 && ok) copy_u(u_issued++);
    auto reduce_rows = [&](int r_end) {
      if (!u_ready) {
        if (ok && !pipe::warp_wait(S, a.status, &S.ufull, pend & 1, timeouts)) ok = false;
        u_ready = true;
      }
      if (ok) {
        // Atilde += U_i(rows)^T W(rows) in packed FP32x2: pairs of U columns
        // (Atilde rows) times one W column.
        float2 tp[NACC / 2];
#pragma unroll
        for (int e = 0; e < NACC / 2; ++e) tp[e] = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int rr = prow; rr < r_end; ++rr) {
          float wv[AC];
#pragma unroll
          for (int y = 0; y < AC; ++y) wv[y] = S.w[rr][AC * tcol + y];
          if constexpr (AA % 2 == 0) {
            float2 up[AA / 2];
#pragma unroll
            for (int x = 0; x < AA / 2; ++x)
              up[x] = *reinterpret_cast<const float2 *>(&S.u[rr][AA * ta + 2 * x]);
            // tp[(x / 2) * AC + y] holds entries (x, y) and (x + 1, y), x even.
#pragma unroll
            for (int x = 0; x < AA / 2; ++x)
#pragma unroll
              for (int y = 0; y < AC; ++y)
                tp[x * AC + y] = __ffma2_rn(up[x], make_float2(wv[y], wv[y]), tp[x * AC + y]);
          } else {
            const float uv = S.u[rr][AA * ta];
#pragma unroll
            for (int y = 0; y < AC / 2; ++y)
              tp[y] = __ffma2_rn(make_float2(uv, uv), make_float2(wv[2 * y], wv[2 * y + 1]), tp[y]);
          }
        }
#pragma unroll
        for (int e = 0; e < NACC / 2; ++e) {
          if constexpr (AA % 2 == 0) {
            const int x = 2 * (e / AC), y = e % AC;
            tacc[AC * x + y] = tp[e].x;
            tacc[AC * (x + 1) + y] = tp[e].y;
          } else {
            tacc[2 * e] = tp[e].x;
            tacc[2 * e + 1] = tp[e].y;
          }
        }
        fold();
      }
      prow = r_end;
    };
    // Every epilogue warp runs all nsteps iterations (skipping waits once a
    // wait failed), so the named barriers below are always reached by all four.
    for (int st = 0; st < nsteps; ++st) {
      const int slot = st & 1, c = st % nch, t = st / nch;
      const bool last = c == nch - 1;
      if (ok && !pipe::warp_wait(S, a.status, &S.dfull[slot], (st >> 1) & 1, timeouts)) ok = false;
      if (last && u_tile < t) {
        // The pending tile's remaining rows; then S.w and S.u are free.
        if (pend >= 0 && prow < pend_rows) reduce_rows(pend_rows);
        epi_sync();
        if (et == 0 && ok) copy_u(u_issued++);  // U_i rows of tile t
        u_tile = t;
      }
      if (ok) {
        tc::tc_fence_after();
        const uint32_t d_t = tmem + slot * KP + lanes;
#pragma unroll 1
        for (int cg = 0; cg < KP / 16; ++cg) {
          float dv[16], hv[16], cv[16];
          tc::tmem_ld16x3(d_t + cg * 16, hi_t + cg * 16, cc_t + cg * 16, dv, hv, cv);
          if (c == 0) {
#pragma unroll
            for (int e = 0; e < 16; ++e) hv[e] = cv[e] = 0.f;
          }
          kahan_add16(hv, cv, dv);  // hi + (d - c); c keeps the lost low part
          if (last) {
            float4 *wr = reinterpret_cast<float4 *>(&S.w[r][cg * 16]);
#pragma unroll
            for (int e = 0; e < 4; ++e)
              wr[e] = make_float4(hv[4 * e] - cv[4 * e], hv[4 * e + 1] - cv[4 * e + 1],
                                  hv[4 * e + 2] - cv[4 * e + 2], hv[4 * e + 3] - cv[4 * e + 3]);
          } else {
            tc::tmem_st16(hi_t + cg * 16, hv);
            tc::tmem_st16(cc_t + cg * 16, cv);
          }
        }
        if (!last) tc::tmem_wait_st();
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&S.dempty[slot]);
      }
      if (last) {
        epi_sync();  // W of tile t complete
        pend = t;
        prow = 0;
        pend_rows = min(MB, mi - MB * t);
        u_ready = false;
        // Spread over the next tile's first nch - 1 steps (all at once after
        // the last tile).
        prows = (t + 1 < ntiles && nch > 1) ? (pend_rows + nch - 2) / (nch - 1) : pend_rows;
        if (t + 1 == ntiles) reduce_rows(pend_rows);
      } else if (pend >= 0 && prow < pend_rows) {
        reduce_rows(min(pend_rows, prow + prows));
        if (prow == pend_rows && u_tile < t) {
          epi_sync();  // every warp is done with S.u
          if (et == 0 && ok) copy_u(u_issued++);  // U_i rows of tile t
          u_tile = t;
        }
      }
    }
    // A U copy still in flight must land before the CTA exits.
    if (et == 0 && u_issued > 0) pipe::drain(&S.ufull, (u_issued - 1) & 1);
    if (ok) {
      auto emit = [&](int e, float hv, float cv) {
        const int ar = AA * ta + e / AC, ac = AC * tcol + e % AC;
        if (ar < k && ac < k) {
          const double val = (ar < ki && ac < kj) ? (double)hv - (double)cv : 0.0;
          out[(int64_t)ar * k + ac] = val;
          if (mirror) out_t[(int64_t)ac * k + ar] = val;
        }
      };
      if constexpr (C::kAccTmem) {
#pragma unroll 1
        for (int g = 0; g < NACC / 16; ++g) {
          float hv[16], cv[16];
          tc::tmem_ld16x2(acc_t + 16 * g, acc_t + NACC + 16 * g, hv, cv);
#pragma unroll
          for (int e = 0; e < 16; ++e) emit(16 * g + e, hv[e], cv[e]);
        }
      } else {
#pragma unroll
        for (int e = 0; e < NACC; ++e) emit(e, rhi[e], rcc[e]);
      }
    }
  } else {
    // ---------------------------------------------------------- generators
    // Generator warp gw writes TMEM lane quadrant q = warp % 4: its thread is
    // tile row 32 q + lane and takes points 32 h .. 32 h + 31 of each chunk
    // (h = gw / 4), two at a time in packed FP32x2 arithmetic; each group of
    // four point pairs goes out as three 4-column TMEM stores (one per part).
    const int gw = warp - (2 + kEpiWarps);  // 0 .. 7
    const int q = warp & 3, h = gw >> 2;
    const int r = 32 * q + lane;
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    const float factor = entry_f32_factor<KERNEL>();
    const float2 f2 = make_float2(factor, factor);
    float2 rx[3], lx[3];  // this row's coordinates, hi and lo, as (v, v) pairs
    for (int st = 0; st < nsteps && !pipe::warp_aborted(S); ++st) {
      const int s = st % STAGES, cs = st % kCS, c = st % nch, t = st / nch;
      const uint32_t ph = (st / STAGES) & 1;
      const int lr = MB * t + r;
      if (c == 0) {
        // Coordinates of this thread's row of tile t (zero past the box).
        const int sp = pi + (lr < mi ? lr : 0);  // slot in the box-padded order
        const int w = sp & (KC - 1), P = w >> 1, u = w & 1;
        const float4 *blk = a.qst + (int64_t)(sp / KC) * (KC / 2 * 3) + (P & 3) * 8 + (P >> 2);
        const float4 f0 = blk[0], f1 = blk[32], fz = blk[64];
        const float v[6] = {u ? f0.y : f0.x, u ? f0.w : f0.z, u ? f1.y : f1.x,
                            u ? f1.w : f1.z, u ? fz.y : fz.x, u ? fz.w : fz.z};
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          rx[ax] = make_float2(-v[ax], -v[ax]);
          lx[ax] = make_float2(-v[3 + ax], -v[3 + ax]);
        }
      }
      if (st >= STAGES && !pipe::warp_wait(S, a.status, &S.empty[s], ph ^ 1, timeouts)) break;
      if (!pipe::warp_wait(S, a.status, &S.cfull[cs], (st / kCS) & 1, timeouts)) break;
      tc::tc_fence_after();  // the MMAs that read this TMEM stage have completed
      const int r0 = MB * t, q0 = KC * c;
      // A chunk away from the diagonal and the ragged edges needs no per-entry
      // checks (the test is uniform over the CTA).
      const bool clean =
          r0 + MB <= mi && q0 + KC <= mj && (i != j || q0 + KC <= r0 || q0 >= r0 + MB);
      const uint32_t a_t = tmem + lanes + C::kABase + s * C::kAStage + 16 * h;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        uint32_t pw[kParts][4];
#pragma unroll
        for (int pr = 0; pr < 4; ++pr) {
          const int jj = 4 * h + g;   // point pair P = 4 jj + pr = 16 h + 4 g + pr
          const float4 q0v = S.qc[cs][0][pr][jj], q1v = S.qc[cs][1][pr][jj],
                       q2v = S.qc[cs][2][pr][jj];
          const float2 dx = __fadd2_rn(__fadd2_rn(rx[0], make_float2(q0v.x, q0v.y)),
                                       __fadd2_rn(lx[0], make_float2(q1v.z, q1v.w)));
          const float2 dy = __fadd2_rn(__fadd2_rn(rx[1], make_float2(q0v.z, q0v.w)),
                                       __fadd2_rn(lx[1], make_float2(q2v.x, q2v.y)));
          float2 r2;
          if (KERNEL == TBLR_KERNEL_LAPLACE3D) {
            const float2 dz = __fadd2_rn(__fadd2_rn(rx[2], make_float2(q1v.x, q1v.y)),
                                         __fadd2_rn(lx[2], make_float2(q2v.z, q2v.w)));
            r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
          } else {
            r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
          }
          float2 v = __fmul2_rn(
              make_float2(entry_f32_of_r2<KERNEL>(r2.x), entry_f32_of_r2<KERNEL>(r2.y)), f2);
          if (!clean) {
            const int lq = q0 + 2 * (4 * jj + pr);
            if (lr >= mi || lq >= mj || (i == j && lq == lr)) v.x = 0.f;
            if (lr >= mi || lq + 1 >= mj || (i == j && lq + 1 == lr)) v.y = 0.f;
          }
          pipe::split3(v.x, v.y, pw[0][pr], pw[1][pr], pw[2][pr]);
        }
#pragma unroll
        for (int p = 0; p < kParts; ++p)
          tc::tmem_st4(a_t + p * (KC / 2) + 4 * g, pw[p][0], pw[p][1], pw[p][2], pw[p][3]);
      }
      tc::tmem_wait_st();
      tc::tc_fence_before();
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
    tc::tmem_dealloc(tmem, C::kTmemCols);
  }
}

// Box-padded offsets: box j's points take ceil(m_j / 64) * 64 slots starting
// at poff[j] (one block; per-thread runs of boxes, then a block scan).
__global__ void pad_offsets_kernel(const int32_t *__restrict__ offsets, int b,
                                   int32_t *__restrict__ poff) {
  __shared__ int32_t part[1024];
  const int t = threadIdx.x, per = (b + 1023) / 1024;
  const int j0 = min(b, t * per), j1 = min(b, j0 + per);
  auto padded = [&](int jb) { return (offsets[jb + 1] - offsets[jb] + KC - 1) / KC * KC; };
  int32_t sum = 0;
  for (int jb = j0; jb < j1; ++jb) sum += padded(jb);
  part[t] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int32_t v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int32_t run = part[t] - sum;
  for (int jb = j0; jb < j1; ++jb) {
    poff[jb] = run;
    run += padded(jb);
  }
  if (t == 1023) poff[b] = part[1023];
}

// Coordinates in the box-padded order, in the mixed apply's staged layout
// (negated double-float pairs; chunk c, pair P = 4 jj + pr at
// qst[c][f][pr][jj], f = {xh, yh}, {zh, xl}, {yl, zl}); padding slots are zero.
__global__ void stage_boxpad_kernel(const double *__restrict__ pts,
                                    const int32_t *__restrict__ offsets,
                                    const int32_t *__restrict__ poff, int64_t n, int d, int b,
                                    float4 *__restrict__ qst) {
  for (int jb = blockIdx.x; jb < b; jb += gridDim.x) {
    const int o = offsets[jb], m = offsets[jb + 1] - o, p0 = poff[jb];
    const int npairs = (poff[jb + 1] - p0) / 2;
    for (int t = threadIdx.x; t < npairs; t += blockDim.x) {
      const int tt = p0 / 2 + t;  // pair index in the box-padded order
      const int64_t c = tt / (KC / 2);
      const int P = tt % (KC / 2), jj = P >> 2, pr = P & 3;
      float h[2][3], l[2][3];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int loc = 2 * t + u;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          h[u][ax] = l[u][ax] = 0.f;
          if (ax < d && loc < m) split_coord(pts[ax * n + o + loc], h[u][ax], l[u][ax]);
        }
      }
      float4 *blk = qst + c * (KC / 2 * 3) + pr * 8 + jj;
      blk[0] = make_float4(-h[0][0], -h[1][0], -h[0][1], -h[1][1]);
      blk[32] = make_float4(-h[0][2], -h[1][2], -l[0][0], -l[1][0]);
      blk[64] = make_float4(-l[0][1], -l[1][1], -l[0][2], -l[1][2]);
    }
  }
}

// V's rows in the box-padded order split into BF16 h/m/l planes [kp][npb]:
// column c < rank_j of the box's point in slot t, zero for padding slots and
// for the other columns.
__global__ void split_v_boxpad_kernel(const double *__restrict__ v,
                                      const int32_t *__restrict__ offsets,
                                      const int32_t *__restrict__ poff,
                                      const int32_t *__restrict__ ranks, int k, int kp, int b,
                                      int64_t npb, __nv_bfloat16 *__restrict__ xh,
                                      __nv_bfloat16 *__restrict__ xm,
                                      __nv_bfloat16 *__restrict__ xl) {
  for (int jb = blockIdx.x; jb < b; jb += gridDim.x) {
    const int o = offsets[jb], m = offsets[jb + 1] - o, p0 = poff[jb];
    const int len = poff[jb + 1] - p0, kj = ranks[jb];
    for (int idx = threadIdx.x; idx < len * kp; idx += blockDim.x) {
      const int c = idx / len, l = idx % len;
      const double x = (l < m && c < kj) ? v[(int64_t)(o + l) * k + c] : 0.0;
      const int64_t dst = (int64_t)c * npb + p0 + l;
      pipe::split3_fp64(x, xh[dst], xm[dst], xl[dst]);
    }
  }
}

// U in FP32 in the box-padded order, rows of kp floats: column a < rank_i of
// the box's point in slot t, zero for padding slots and the other columns
// (the MB spare rows at the end stay unset and are never used).
__global__ void u_boxpad_kernel(const double *__restrict__ u, const int32_t *__restrict__ offsets,
                                const int32_t *__restrict__ poff,
                                const int32_t *__restrict__ ranks, int k, int kp, int b,
                                float *__restrict__ uf) {
  for (int jb = blockIdx.x; jb < b; jb += gridDim.x) {
    const int o = offsets[jb], m = offsets[jb + 1] - o, p0 = poff[jb];
    const int len = poff[jb + 1] - p0, kj = ranks[jb];
    for (int idx = threadIdx.x; idx < len * kp; idx += blockDim.x) {
      const int l = idx / kp, c = idx % kp;
      uf[(int64_t)(p0 + l) * kp + c] = (l < m && c < kj) ? (float)u[(int64_t)(o + l) * k + c] : 0.f;
    }
  }
}

struct CplLayout {
  int kp;
  int64_t npb;
  size_t head, coords, planes, uf, poff, total;
};

CplLayout cpl_layout(const Prob &P) {
  CplLayout L;
  L.kp = P.k <= 16 ? 16 : P.k <= 32 ? 32 : 64;
  L.npb = cdiv(P.n, KC) * KC + (int64_t)KC * P.b;  // >= sum of ceil(m_j / 64) * 64
  L.head = 256;
  L.coords = align256(sizeof(float4) * 3 * (L.npb / 2));
  L.planes = align256(sizeof(__nv_bfloat16) * L.kp * L.npb);
  L.uf = align256(sizeof(float) * (L.npb + MB) * L.kp);
  L.poff = align256(sizeof(int32_t) * (P.b + 1));
  L.total = L.head + L.coords + kParts * L.planes + L.uf + L.poff;
  return L;
}

template <int KERNEL, int KP>
int launch_coupling_tc(const CplMaps &maps, const CplArgs &a, cudaStream_t s) {
  static_assert(sizeof(CplSmem<KP>) + 1024 <= (size_t)kSmemLimit, "shared memory");
  auto kern = coupling_tc_kernel<KERNEL, KP>;
  const size_t smem = sizeof(CplSmem<KP>) + 1024;
  TBLR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<dim3((unsigned)a.b, (unsigned)a.b), kThreads, smem, s>>>(maps, a);
  return launch_status("coupling_tc_kernel");
}

template <int KERNEL>
int dispatch_coupling_tc(int kp, const CplMaps &maps, const CplArgs &a, cudaStream_t s) {
  if (kp == 16) return launch_coupling_tc<KERNEL, 16>(maps, a, s);
  if (kp == 32) return launch_coupling_tc<KERNEL, 32>(maps, a, s);
  return launch_coupling_tc<KERNEL, 64>(maps, a, s);
}

}  // namespace

size_t coupling_tc_workspace(const Prob &P) { return cpl_layout(P).total; }

int coupling_tc(const Prob &P, const tblr_layout *lay, const double *u, const double *v,
                const int32_t *ranks, double *at, void *ws, size_t ws_bytes, cudaStream_t s) {
  TBLR_REQUIRE(P.kernel == TBLR_KERNEL_LAPLACE2D || P.kernel == TBLR_KERNEL_LAPLACE3D,
               "tensor-core coupling supports the built-in Laplace kernels");
  TBLR_REQUIRE(P.k >= 1 && P.k <= 64, "tensor-core coupling supports 1 <= k <= 64");
  TBLR_REQUIRE(P.n < (int64_t)1 << 30 && P.b <= 65535, "tensor-core coupling: problem too large");
  const CplLayout L = cpl_layout(P);
  TBLR_REQUIRE(ws != nullptr && ws_bytes >= L.total, "coupling workspace too small (%zu < %zu)",
               ws_bytes, L.total);
  TBLR_REQUIRE((reinterpret_cast<uintptr_t>(ws) & 255) == 0, "workspace must be 256-byte aligned");
  char *w = static_cast<char *>(ws);
  int *status = reinterpret_cast<int *>(w);
  float4 *qst = reinterpret_cast<float4 *>(w + L.head);
  __nv_bfloat16 *part[kParts];
  for (int t = 0; t < kParts; ++t)
    part[t] = reinterpret_cast<__nv_bfloat16 *>(w + L.head + L.coords + t * L.planes);
  float *uf = reinterpret_cast<float *>(w + L.head + L.coords + kParts * L.planes);
  int32_t *poff = reinterpret_cast<int32_t *>(w + L.head + L.coords + kParts * L.planes + L.uf);
  const int b = (int)P.b;
  const unsigned gb = (unsigned)std::min(b, 4096);
  TBLR_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
  pad_offsets_kernel<<<1, 1024, 0, s>>>(lay->offsets, b, poff);
  TBLR_TRY(launch_status("pad_offsets_kernel"));
  stage_boxpad_kernel<<<gb, 256, 0, s>>>(lay->pts, lay->offsets, poff, P.n, P.d, b, qst);
  TBLR_TRY(launch_status("stage_boxpad_kernel"));
  split_v_boxpad_kernel<<<gb, 256, 0, s>>>(v, lay->offsets, poff, ranks, (int)P.k, L.kp, b, L.npb,
                                           part[0], part[1], part[2]);
  TBLR_TRY(launch_status("split_v_boxpad_kernel"));
  u_boxpad_kernel<<<gb, 256, 0, s>>>(u, lay->offsets, poff, ranks, (int)P.k, L.kp, b, uf);
  TBLR_TRY(launch_status("u_boxpad_kernel"));
  CplMaps maps;
  for (int t = 0; t < kParts; ++t)
    TBLR_TRY(pipe::make_plane_map(&maps.part[t], part[t], L.npb, L.kp, L.kp));
  CplArgs a{};
  a.qst = qst;
  a.offsets = lay->offsets;
  a.poff = poff;
  a.ranks = ranks;
  a.u = uf;
  a.k = (int)P.k;
  a.b = b;
  a.sym = P.selfadjoint ? 1 : 0;
  a.at = at;
  a.status = status;
  return P.kernel == TBLR_KERNEL_LAPLACE2D
             ? dispatch_coupling_tc<TBLR_KERNEL_LAPLACE2D>(L.kp, maps, a, s)
             : dispatch_coupling_tc<TBLR_KERNEL_LAPLACE3D>(L.kp, maps, a, s);
}

unsigned int coupling_tc_take_timeouts() {
  unsigned int count = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&count, g_coupling_timeouts, sizeof(unsigned int)) != cudaSuccess)
    return 0;
  cudaMemcpyToSymbol(g_coupling_timeouts, &zero, sizeof(unsigned int));
  return count;
}

}  // namespace tblr
