// Steps II and III (Table 1) for the mixed-precision path, on the FP32 pipes
// (GB300 runs FP32 FMA ~60x faster than FP64).  Kernel entries come from
// double-float coordinates (~2^-23 relative), products are FP32, and every
// long sum is accumulated in FP32 chunks of at most 32 terms that are added
// into Kahan-compensated FP32 sums, so each output keeps ~1e-7 relative error.
//   coupling   Atilde_ij = U_i^T (A_ij V_j)                  (§2.5, Table 1 step 2)
//   nf lowrank M_is = sum_{c in set} Atilde_ic V_c(0:m_j,:)^T  (§6.1 eq. sparse_struct_ids)
//   nf block   B_ij = sum_{c in set} A(I_i, I_c(0:m_j)) - U_i M_is
#include <stdlib.h>

#include "coupling_tc.cuh"
#include "kernels_f32.cuh"
#include "recon_mixed.cuh"

namespace tblr {
namespace {

constexpr int kThreads = 256;

template <int KERNEL>
__device__ __forceinline__ void load_point(const double *__restrict__ pts, int64_t n, int d,
                                           int64_t p, float (&h)[3], float (&l)[3]) {
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (ax < d)
      split_coord(pts[ax * n + p], h[ax], l[ax]);
    else
      h[ax] = l[ax] = 0.f;
  }
}

// CTA per (i, j): a register-tiled FP32 GEMM on the packed FP32x2 pipes.
// Rows of box i go in chunks of RC; for each chunk W = A(chunk, I_j) V_j is
// accumulated over KT-point steps: the CTA generates the KT x RC kernel tile
// into shared memory (two rows at a time in FP32x2 arithmetic from double-float
// coordinates) next to the step's rows of V_j stored as duplicated pairs
// (v, v), and each thread updates an 8 x 4 block of W as 4 x 4 row pairs with
// one FFMA2 per pair (a 16-FFMA2 inner step from four 16-byte loads).  Each
// step's FP32 sum (64 terms) is added to a running FP32 sum, so a W entry
// carries ~sqrt(64) + sqrt(m_j / 64) roundings instead of sqrt(m_j).  Then
// Atilde_ij += U_i(chunk)^T W with U's rows and W in shared memory (aliasing
// the step buffers).
template <int KP>
struct CouplingShape {
  static constexpr int TX = KP / 4;       // threads across W's columns (4 each)
  static constexpr int TY = 256 / TX;     // threads across W's rows (8 each)
  static constexpr int RC = 8 * TY;       // rows per chunk
  static constexpr int AT = KP / 16;      // Atilde tile edge per thread (16 x 16 threads)
  static constexpr int KT = 64;           // points per K step
  static constexpr int AS = RC + 4;       // row stride of the generated tile
  static constexpr size_t kStep = sizeof(float) * KT * AS + sizeof(float2) * KT * KP;
  static constexpr size_t kChunk = sizeof(float) * 2 * (size_t)RC * (KP + 4);
  static constexpr size_t kBuf = kStep > kChunk ? kStep : kChunk;
  static constexpr size_t kBytes = kBuf + sizeof(float4) * 3 * (RC / 2) + sizeof(float) * 6 * KT;
};

template <int KP>
size_t coupling_f32_smem_bytes() {
  return CouplingShape<KP>::kBytes;
}

template <int KERNEL, int KP>
__global__ void __launch_bounds__(kThreads, 2) coupling_f32_kernel(
    const float *__restrict__ ch, const float *__restrict__ cl, int64_t npad,
    const int32_t *__restrict__ offsets, const int32_t *__restrict__ ranks,
    const float *__restrict__ U, const float *__restrict__ V, int k, int b, int sym,
    double *__restrict__ At) {
  using C = CouplingShape<KP>;
  constexpr int TX = C::TX, RC = C::RC, AT = C::AT, KT = C::KT, AS = C::AS;
  extern __shared__ __align__(16) float sf[];
  float *Ak = sf;                                            // [KT][AS]  A(step point, chunk row)
  float2 *Vd = reinterpret_cast<float2 *>(sf + KT * AS);     // [KT][KP]  (v, v) pairs of V_j
  float *Ws = sf;                                            // [RC][KP + 4]  (aliases Ak, Vd)
  float *Us = sf + RC * (KP + 4);                            // [RC][KP + 4]
  float4 *rc = reinterpret_cast<float4 *>(reinterpret_cast<char *>(sf) + C::kBuf);
  // rc[3 * pr + f]: row pair pr's coordinates {xh, yh}, {zh, xl}, {yl, zl}
  float *qs = reinterpret_cast<float *>(rc + 3 * (RC / 2));  // [6][KT] step point coordinates
  const int i = blockIdx.x, j = blockIdx.y, tid = threadIdx.x;
  // Self-adjoint (V = U, A = A^T): CTA (i, j), i < j, also writes Atilde_ji = Atilde_ij^T.
  if (sym && i > j) return;
  const bool mirror = sym && i != j;
  const int oi = offsets[i], mi = offsets[i + 1] - oi;
  const int oj = offsets[j], mj = offsets[j + 1] - oj;
  const int ki = ranks[i], kj = ranks[j];
  double *out = At + ((int64_t)i * b + j) * k * k;
  double *out_t = At + ((int64_t)j * b + i) * k * k;
  if (ki == 0 || kj == 0) {
    for (int idx = tid; idx < k * k; idx += kThreads) {
      out[idx] = 0.0;
      if (mirror) out_t[idx] = 0.0;
    }
    return;
  }
  const int tx = tid % TX, ty = tid / TX;       // W block: rows 8 ty .., columns 4 tx ..
  const int ta = tid / 16, tc = tid % 16;       // Atilde tile: rows AT*ta.., columns AT*tc..
  const int lane = tid & 31, warp = tid >> 5;  // generation: points warp + 8 v, row pairs lane + 32 u
  const float factor = entry_f32_factor<KERNEL>();
  float thi[AT][AT], tcc[AT][AT];
#pragma unroll
  for (int x = 0; x < AT; ++x)
#pragma unroll
    for (int y = 0; y < AT; ++y) thi[x][y] = tcc[x][y] = 0.f;

  for (int r0 = 0; r0 < mi; r0 += RC) {
    __syncthreads();
    for (int pr = tid; pr < RC / 2; pr += kThreads) {
      float h[2][3], l[2][3];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int r = r0 + 2 * pr + u;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          h[u][ax] = r < mi ? ch[ax * npad + oi + r] : 0.f;
          l[u][ax] = r < mi ? cl[ax * npad + oi + r] : 0.f;
        }
      }
      rc[3 * pr + 0] = make_float4(h[0][0], h[1][0], h[0][1], h[1][1]);
      rc[3 * pr + 1] = make_float4(h[0][2], h[1][2], l[0][0], l[1][0]);
      rc[3 * pr + 2] = make_float4(l[0][1], l[1][1], l[0][2], l[1][2]);
    }
    float2 acc[4][4], hi[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = hi[x][y] = make_float2(0.f, 0.f);
    for (int q0 = 0; q0 < mj; q0 += KT) {
      __syncthreads();
      // Step rows of V_j as (v, v) pairs, interleaved so that the column pairs
      // (4 tx, 4 tx + 1) of all tx come first, then (4 tx + 2, 4 tx + 3): each of
      // a thread's two 16-byte loads then reads a contiguous run across tx.
      for (int idx = tid; idx < KT * KP; idx += kThreads) {
        const int q = idx / KP, c = idx % KP;
        const float v = (q0 + q < mj && c < kj) ? V[((int64_t)oj + q0 + q) * k + c] : 0.f;
        const int ctx = c >> 2, half = (c >> 1) & 1, e = c & 1;
        Vd[((q * 2 + half) * TX + ctx) * 2 + e] = make_float2(v, v);
      }
      // The step's point coordinates (negated double-float pairs).
      for (int q = tid; q < KT; q += kThreads) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          const bool in = q0 + q < mj;
          qs[ax * KT + q] = in ? -ch[ax * npad + oj + q0 + q] : 0.f;
          qs[(3 + ax) * KT + q] = in ? -cl[ax * npad + oj + q0 + q] : 0.f;
        }
      }
      __syncthreads();
      // Kernel tile: each warp takes points warp + 8 v (coordinates warp-uniform,
      // negated and broadcast as pairs), its lanes consecutive row pairs, so the
      // 8-byte stores of a warp are contiguous.
      const float2 f2 = make_float2(factor, factor);
      for (int gq = warp; gq < KT; gq += kThreads / 32) {
        const bool qin = q0 + gq < mj;
        const float2 nxh = make_float2(qs[gq], qs[gq]), nyh = make_float2(qs[KT + gq], qs[KT + gq]);
        const float2 nzh = make_float2(qs[2 * KT + gq], qs[2 * KT + gq]);
        const float2 nxl = make_float2(qs[3 * KT + gq], qs[3 * KT + gq]);
        const float2 nyl = make_float2(qs[4 * KT + gq], qs[4 * KT + gq]);
        const float2 nzl = make_float2(qs[5 * KT + gq], qs[5 * KT + gq]);
        for (int pr = lane; pr < RC / 2; pr += 32) {
          const float4 c0 = rc[3 * pr], c1 = rc[3 * pr + 1], c2 = rc[3 * pr + 2];
          const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(c0.x, c0.y), nxh),
                                       __fadd2_rn(make_float2(c1.z, c1.w), nxl));
          const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(c0.z, c0.w), nyh),
                                       __fadd2_rn(make_float2(c2.x, c2.y), nyl));
          float2 r2;
          if (KERNEL == TBLR_KERNEL_LAPLACE3D) {
            const float2 dz = __fadd2_rn(__fadd2_rn(make_float2(c1.x, c1.y), nzh),
                                         __fadd2_rn(make_float2(c2.z, c2.w), nzl));
            r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
          } else {
            r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
          }
          float2 v = __fmul2_rn(make_float2(entry_f32_of_r2<KERNEL>(r2.x),
                                            entry_f32_of_r2<KERNEL>(r2.y)), f2);
          const int rr = r0 + 2 * pr;
          if (!qin || rr >= mi || (i == j && rr == q0 + gq)) v.x = 0.f;
          if (!qin || rr + 1 >= mi || (i == j && rr + 1 == q0 + gq)) v.y = 0.f;
          *reinterpret_cast<float2 *>(Ak + gq * AS + 2 * pr) = v;
        }
      }
      __syncthreads();
#pragma unroll 4
      for (int q = 0; q < KT; ++q) {
        const float4 a0 = *reinterpret_cast<const float4 *>(Ak + q * AS + 8 * ty);
        const float4 a1 = *reinterpret_cast<const float4 *>(Ak + q * AS + 8 * ty + 4);
        const float4 v0 = *reinterpret_cast<const float4 *>(Vd + ((q * 2 + 0) * TX + tx) * 2);
        const float4 v1 = *reinterpret_cast<const float4 *>(Vd + ((q * 2 + 1) * TX + tx) * 2);
        const float2 ap[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w),
                              make_float2(a1.x, a1.y), make_float2(a1.z, a1.w)};
        const float2 vp[4] = {make_float2(v0.x, v0.y), make_float2(v0.z, v0.w),
                              make_float2(v1.x, v1.y), make_float2(v1.z, v1.w)};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = __ffma2_rn(ap[x], vp[y], acc[x][y]);
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          hi[x][y] = __fadd2_rn(hi[x][y], acc[x][y]);
          acc[x][y] = make_float2(0.f, 0.f);
        }
    }
    // W chunk and U rows to shared memory (over the step buffers), then
    // Atilde += U^T W.
    __syncthreads();
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        Ws[(8 * ty + 2 * x) * (KP + 4) + 4 * tx + y] = hi[x][y].x;
        Ws[(8 * ty + 2 * x + 1) * (KP + 4) + 4 * tx + y] = hi[x][y].y;
      }
    for (int idx = tid; idx < RC * KP; idx += kThreads) {
      const int r = idx / KP, a = idx % KP;
      Us[r * (KP + 4) + a] = (r0 + r < mi && a < ki) ? U[((int64_t)oi + r0 + r) * k + a] : 0.f;
    }
    __syncthreads();
    float tacc[AT][AT];
#pragma unroll
    for (int x = 0; x < AT; ++x)
#pragma unroll
      for (int y = 0; y < AT; ++y) tacc[x][y] = 0.f;
    const int rend = min(RC, mi - r0);
    for (int r = 0; r < rend; ++r) {
      float u[AT], w[AT];
#pragma unroll
      for (int x = 0; x < AT; ++x) u[x] = Us[r * (KP + 4) + AT * ta + x];
#pragma unroll
      for (int y = 0; y < AT; ++y) w[y] = Ws[r * (KP + 4) + AT * tc + y];
#pragma unroll
      for (int x = 0; x < AT; ++x)
#pragma unroll
        for (int y = 0; y < AT; ++y) tacc[x][y] = fmaf(u[x], w[y], tacc[x][y]);
      if ((r & 31) == 31 || r == rend - 1) {
#pragma unroll
        for (int x = 0; x < AT; ++x)
#pragma unroll
          for (int y = 0; y < AT; ++y) {
            kahan_add(thi[x][y], tcc[x][y], tacc[x][y]);
            tacc[x][y] = 0.f;
          }
      }
    }
  }
#pragma unroll
  for (int x = 0; x < AT; ++x)
#pragma unroll
    for (int y = 0; y < AT; ++y) {
      const int a = AT * ta + x, c = AT * tc + y;
      if (a < k && c < k) {
        const double val = (a < ki && c < kj) ? (double)thi[x][y] - (double)tcc[x][y] : 0.0;
        out[(int64_t)a * k + c] = val;
        if (mirror) out_t[(int64_t)c * k + a] = val;
      }
    }
}

// CTA per (i, s, 128-column tile of M): M_is(a, q) for a < k, q in the tile.
// Each set member c contributes Atilde_ic V_c(q, :)^T: Atilde_ic^T and the
// tile's columns of V_c^T are staged in shared memory (t-major, so a thread
// reads its 4 rows and 8 columns with three 16-byte loads per rank index t),
// each thread accumulates a 4 x 8 block over 16 rank indices at a time and
// adds it to Kahan sums.
constexpr int kQT = 128;     // columns of M per CTA
constexpr int kAS = 64 + 4;  // row stride of Atilde^T in shared memory (k <= 64)
constexpr int kVS = kQT + 4;  // row stride of V^T in shared memory
__global__ void __launch_bounds__(kThreads) nf_lowrank_f32_kernel(
    const int32_t *__restrict__ offsets, const int32_t *__restrict__ nbr,
    const int32_t *__restrict__ nnbr, const int32_t *__restrict__ colour, int b, int s3, int k,
    int mmax, int mode, const double *__restrict__ At, const float *__restrict__ vt, int64_t n,
    float *__restrict__ M) {
  extern __shared__ __align__(16) float sf[];
  const int i = blockIdx.x, s = blockIdx.y, q0 = blockIdx.z * kQT, tid = threadIdx.x;
  if (s >= nnbr[i]) return;
  const int j = nbr[(int64_t)i * s3 + s];
  const int mj = offsets[j + 1] - offsets[j];
  if (q0 >= mj) return;
  float *As = sf;               // [64][kAS]: As[t * kAS + a] = Atilde_ic(a, t)
  float *Vs = As + 64 * kAS;    // [64][kVS]: Vs[t * kVS + q] = V_c(q0 + q, t)
  int *set = reinterpret_cast<int *>(Vs + 64 * kVS);
  const int ns = block_probe_set(j, mode, colour, b, set);
  for (int idx = tid; idx < 64 * kAS; idx += kThreads) As[idx] = 0.f;  // rows a >= k stay 0
  const int ta = tid % 16, tq = tid / 16;  // rows 4 ta + x, columns 8 tq + y
  // Column pairs (8 tq + 2 yp, 8 tq + 2 yp + 1) in packed FP32x2; the
  // compensated adds use a - b = fma(b, -1, a) (exactly rounded).
  const float2 m1 = make_float2(-1.f, -1.f);
  float2 hi[4][4], cc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int yp = 0; yp < 4; ++yp) hi[x][yp] = cc[x][yp] = make_float2(0.f, 0.f);
  for (int u = 0; u < ns; ++u) {
    const int c = set[u];
    const int oc = offsets[c], mc = offsets[c + 1] - oc;
    if (q0 >= mc) continue;  // uniform over the CTA
    const int qn = min(min(mc, mj) - q0, kQT);
    __syncthreads();
    const double *Ac = At + ((int64_t)i * b + c) * k * k;
    for (int idx = tid; idx < k * k; idx += kThreads) {
      const int a = idx / k, t = idx % k;
      As[t * kAS + a] = (float)Ac[idx];
    }
    for (int idx = tid; idx < k * kQT; idx += kThreads) {
      const int t = idx / kQT, q = idx % kQT;
      Vs[t * kVS + q] = q < qn ? vt[(int64_t)t * n + oc + q0 + q] : 0.f;
    }
    __syncthreads();
    for (int t0 = 0; t0 < k; t0 += 16) {
      float2 acc[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int yp = 0; yp < 4; ++yp) acc[x][yp] = make_float2(0.f, 0.f);
      const int t1 = min(t0 + 16, k);
      for (int t = t0; t < t1; ++t) {
        const float4 av = *reinterpret_cast<const float4 *>(As + t * kAS + 4 * ta);
        const float4 v0 = *reinterpret_cast<const float4 *>(Vs + t * kVS + 8 * tq);
        const float4 v1 = *reinterpret_cast<const float4 *>(Vs + t * kVS + 8 * tq + 4);
        const float ar[4] = {av.x, av.y, av.z, av.w};
        const float2 vp[4] = {make_float2(v0.x, v0.y), make_float2(v0.z, v0.w),
                              make_float2(v1.x, v1.y), make_float2(v1.z, v1.w)};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int yp = 0; yp < 4; ++yp)
            acc[x][yp] = __ffma2_rn(make_float2(ar[x], ar[x]), vp[yp], acc[x][yp]);
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int yp = 0; yp < 4; ++yp) {
          const float2 y = __ffma2_rn(cc[x][yp], m1, acc[x][yp]);
          const float2 tt = __fadd2_rn(hi[x][yp], y);
          cc[x][yp] = __ffma2_rn(y, m1, __ffma2_rn(hi[x][yp], m1, tt));
          hi[x][yp] = tt;
        }
    }
  }
  float *out = M + ((int64_t)i * s3 + s) * k * mmax;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int a = 4 * ta + x;
    if (a >= k) continue;
#pragma unroll
    for (int y = 0; y < 8; ++y) {
      const int q = q0 + 8 * tq + y;
      const float h = y & 1 ? hi[x][y >> 1].y : hi[x][y >> 1].x;
      const float c = y & 1 ? cc[x][y >> 1].y : cc[x][y >> 1].x;
      if (q < mj) out[(int64_t)a * mmax + q] = h - c;
    }
  }
}

// V (FP64, n x k row-major) as FP32 V^T (k x n), the layout nf_lowrank reads.
__global__ void transpose_v_f32(const double *__restrict__ v, int64_t n, int k,
                                float *__restrict__ vt) {
  const int64_t total = n * k;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = idx / n, p = idx % n;
    vt[idx] = (float)v[p * k + t];
  }
}

// B_ij(p, q) = sum_{c in set, q < m_c} A(I_i[p], I_c[q]) - U_i(p, :) M_is(:, q), by
// 64 x 64 output tiles (grid.z = tile index): 4 x 4 outputs per thread; the
// column coordinates of each probe box are staged once per tile, the tile's
// rows of U_i and columns of M_is sit in shared memory for the low-rank part.
constexpr int kBT = 64;
constexpr int kNSC = 32;  // probe-set boxes whose coordinates are staged per barrier
template <int KERNEL>
__global__ void __launch_bounds__(kThreads) nf_block_f32_kernel(
    const float *__restrict__ chp, const float *__restrict__ clp, int64_t npad,
    const int32_t *__restrict__ offsets, const int32_t *__restrict__ nbr,
    const int32_t *__restrict__ nnbr, const int32_t *__restrict__ colour, int b, int s3, int k,
    int mmax, int mode, const double *__restrict__ U, const float *__restrict__ M,
    const int64_t *__restrict__ nf_off, double *__restrict__ Bn) {
  extern __shared__ float sf[];
  const int i = blockIdx.x, s = blockIdx.y, tid = threadIdx.x;
  if (s >= nnbr[i]) return;
  const int j = nbr[(int64_t)i * s3 + s];
  const int oi = offsets[i], mi = offsets[i + 1] - oi;
  const int mj = offsets[j + 1] - offsets[j];
  const int ntq = (mj + kBT - 1) / kBT;
  const int p0 = (blockIdx.z / ntq) * kBT, q0 = (blockIdx.z % ntq) * kBT;
  if (p0 >= mi) return;
  float *Us = sf;                          // [kBT][k + 1]
  float *Ms = Us + kBT * (k + 1);          // [k][kBT + 4]
  float *qh = Ms + k * (kBT + 4);          // [kNSC][3][kBT]
  float *ql = qh + kNSC * 3 * kBT;         // [kNSC][3][kBT]
  int *set = reinterpret_cast<int *>(ql + kNSC * 3 * kBT);
  const int ns = block_probe_set(j, mode, colour, b, set);
  for (int idx = tid; idx < kBT * k; idx += kThreads) {
    const int r = idx / k, a = idx % k;
    Us[r * (k + 1) + a] = (p0 + r < mi) ? (float)U[((int64_t)oi + p0 + r) * k + a] : 0.f;
  }
  const float *Mi = M + ((int64_t)i * s3 + s) * k * mmax;
  for (int idx = tid; idx < k * kBT; idx += kThreads) {
    const int a = idx / kBT, q = idx % kBT;
    Ms[a * (kBT + 4) + q] = (q0 + q < mj) ? Mi[(int64_t)a * mmax + q0 + q] : 0.f;
  }
  const int tx = tid % 16, ty = tid / 16;   // rows p0 + 4 ty + x, columns q0 + 4 tx + y
  // Row coordinates as (v, v) pairs; the step's point coordinates are staged
  // negated, so a column pair (q, q + 1) is one 8-byte load and every
  // difference, square and compensated add below is packed FP32x2.
  float2 rh[4][3], rl[4][3];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int64_t gp = (int64_t)oi + p0 + 4 * ty + x;
    const bool in = p0 + 4 * ty + x < mi;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const float h = in ? chp[ax * npad + gp] : 0.f, l = in ? clp[ax * npad + gp] : 0.f;
      rh[x][ax] = make_float2(h, h);
      rl[x][ax] = make_float2(l, l);
    }
  }
  const float2 f2 = make_float2(entry_f32_factor<KERNEL>(), entry_f32_factor<KERNEL>());
  const float2 m1 = make_float2(-1.f, -1.f);
  float2 hi[4][2], cc[4][2];  // columns (4 tx + 2 yp, 4 tx + 2 yp + 1)
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int yp = 0; yp < 2; ++yp) hi[x][yp] = cc[x][yp] = make_float2(0.f, 0.f);
  // hi + v with compensation c (packed Kahan; a - b as the exactly rounded fma(b, -1, a)).
  auto kahan2 = [&](float2 &h, float2 &c, float2 v) {
    const float2 y = __ffma2_rn(c, m1, v);
    const float2 t = __fadd2_rn(h, y);
    c = __ffma2_rn(y, m1, __ffma2_rn(h, m1, t));
    h = t;
  };
  for (int u0 = 0; u0 < ns; u0 += kNSC) {
    // The step's columns of up to kNSC probe-set boxes, staged at once.
    const int nb = min(kNSC, ns - u0);
    __syncthreads();
    for (int idx = tid; idx < nb * 3 * kBT; idx += kThreads) {
      const int uu = idx / (3 * kBT), ax = (idx / kBT) % 3, q = idx % kBT;
      const int cb = set[u0 + uu];
      const int ocb = offsets[cb], mcb = offsets[cb + 1] - ocb;
      const bool in = q0 + q < mcb;
      qh[idx] = in ? -chp[ax * npad + ocb + q0 + q] : 0.f;
      ql[idx] = in ? -clp[ax * npad + ocb + q0 + q] : 0.f;
    }
    __syncthreads();
    for (int uu = 0; uu < nb; ++uu) {
      const int c = set[u0 + uu];
      const int mc = offsets[c + 1] - offsets[c];
      if (q0 >= mc) continue;  // uniform over the CTA
      const float *qhb = qh + uu * 3 * kBT, *qlb = ql + uu * 3 * kBT;
      // A tile inside both boxes and off the diagonal needs no per-entry checks.
      const bool clean = q0 + kBT <= mc && q0 + kBT <= mj && p0 + kBT <= mi && c != i;
#pragma unroll
      for (int yp = 0; yp < 2; ++yp) {
        const int q = 4 * tx + 2 * yp;
        float2 nh[3], nl[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          nh[ax] = *reinterpret_cast<const float2 *>(&qhb[ax * kBT + q]);
          nl[ax] = *reinterpret_cast<const float2 *>(&qlb[ax * kBT + q]);
        }
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const float2 dx = __fadd2_rn(__fadd2_rn(rh[x][0], nh[0]), __fadd2_rn(rl[x][0], nl[0]));
          const float2 dy = __fadd2_rn(__fadd2_rn(rh[x][1], nh[1]), __fadd2_rn(rl[x][1], nl[1]));
          float2 r2;
          if (KERNEL == TBLR_KERNEL_LAPLACE3D) {
            const float2 dz = __fadd2_rn(__fadd2_rn(rh[x][2], nh[2]), __fadd2_rn(rl[x][2], nl[2]));
            r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
          } else {
            r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
          }
          float2 v = __fmul2_rn(
              make_float2(entry_f32_of_r2<KERNEL>(r2.x), entry_f32_of_r2<KERNEL>(r2.y)), f2);
          if (!clean) {
            const int p = p0 + 4 * ty + x, qq = q0 + q;
            if (qq >= mc || qq >= mj || p >= mi || (c == i && p == qq)) v.x = 0.f;
            if (qq + 1 >= mc || qq + 1 >= mj || p >= mi || (c == i && p == qq + 1)) v.y = 0.f;
          }
          kahan2(hi[x][yp], cc[x][yp], v);
        }
      }
    }
  }
  __syncthreads();
  // Low-rank part U_i M_is, subtracted from the compensated sums 8 rank terms
  // at a time (so each FP32 partial sum has at most 8 roundings).
  for (int a0 = 0; a0 < k; a0 += 8) {
    float2 lr[4][2];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int yp = 0; yp < 2; ++yp) lr[x][yp] = make_float2(0.f, 0.f);
    const int a1 = min(a0 + 8, k);
    for (int a = a0; a < a1; ++a) {
      float uu[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) uu[x] = Us[(4 * ty + x) * (k + 1) + a];
      const float4 m4 = *reinterpret_cast<const float4 *>(&Ms[a * (kBT + 4) + 4 * tx]);
      const float2 mm[2] = {make_float2(m4.x, m4.y), make_float2(m4.z, m4.w)};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int yp = 0; yp < 2; ++yp)
          lr[x][yp] = __ffma2_rn(make_float2(uu[x], uu[x]), mm[yp], lr[x][yp]);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int yp = 0; yp < 2; ++yp)
        kahan2(hi[x][yp], cc[x][yp], make_float2(-lr[x][yp].x, -lr[x][yp].y));
  }
  double *out = Bn + nf_off[(int64_t)i * s3 + s];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int p = p0 + 4 * ty + x;
    if (p >= mi) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int q = q0 + 4 * tx + y;
      const float h = y & 1 ? hi[x][y >> 1].y : hi[x][y >> 1].x;
      const float c = y & 1 ? cc[x][y >> 1].y : cc[x][y >> 1].x;
      if (q < mj) out[(int64_t)p * mj + q] = (double)h - (double)c;
    }
  }
}

__global__ void split_all_coords(const double *__restrict__ pts, int64_t n, int64_t npad, int d,
                                 float *__restrict__ ch, float *__restrict__ cl) {
  const int64_t total = 3 * npad;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ax = t / npad, p = t % npad;
    float h = 0.f, l = 0.f;
    if (ax < d && p < n) split_coord(pts[ax * n + p], h, l);
    ch[t] = h;
    cl[t] = l;
  }
}

}  // namespace

struct CouplingWs {
  float *ch, *cl, *u, *v;
  int64_t npad;
};

CouplingWs coupling_ws(const Prob &P, void *ws) {
  CouplingWs w;
  w.npad = cdiv(P.n, 64) * 64;
  char *p = static_cast<char *>(ws);
  w.ch = reinterpret_cast<float *>(p);
  p += align256(sizeof(float) * 3 * w.npad);
  w.cl = reinterpret_cast<float *>(p);
  p += align256(sizeof(float) * 3 * w.npad);
  w.u = reinterpret_cast<float *>(p);
  p += align256(sizeof(float) * P.n * P.k);
  w.v = reinterpret_cast<float *>(p);
  return w;
}

__global__ void to_f32(const double *__restrict__ x, int64_t len, float *__restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

template <int KERNEL, int KP>
int launch_coupling_f32(const Prob &P, const CouplingWs &w, const tblr_layout *lay,
                        const int32_t *ranks, double *at, cudaStream_t s) {
  auto kern = coupling_f32_kernel<KERNEL, KP>;
  const size_t smem = coupling_f32_smem_bytes<KP>();
  TBLR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<dim3((unsigned)P.b, (unsigned)P.b), kThreads, smem, s>>>(
      w.ch, w.cl, w.npad, lay->offsets, ranks, w.u, w.v, P.k, (int)P.b, P.selfadjoint ? 1 : 0, at);
  return launch_status("coupling_f32_kernel");
}

template <int KERNEL>
int coupling_f32_dispatch(const Prob &P, const CouplingWs &w, const tblr_layout *lay,
                          const int32_t *ranks, double *at, cudaStream_t s) {
  if (P.k <= 16) return launch_coupling_f32<KERNEL, 16>(P, w, lay, ranks, at, s);
  if (P.k <= 32) return launch_coupling_f32<KERNEL, 32>(P, w, lay, ranks, at, s);
  return launch_coupling_f32<KERNEL, 64>(P, w, lay, ranks, at, s);
}

size_t coupling_mixed_workspace(const Prob &P) {
  const int64_t npad = cdiv(P.n, 64) * 64;
  const size_t simt = 2 * align256(sizeof(float) * 3 * npad) + 2 * align256(sizeof(float) * P.n * P.k);
  return std::max(simt, coupling_tc_workspace(P));
}

// The FP32 SIMT coupling instead of the tensor-core one (TBLR_COUPLING_SIMT=1).
static bool coupling_simt() {
  static int v = -1;
  if (v < 0) {
    const char *e = getenv("TBLR_COUPLING_SIMT");
    v = (e && atoi(e) != 0) ? 1 : 0;
  }
  return v == 1;
}

int coupling_mixed(const Prob &P, const tblr_layout *lay, const double *u, const double *v,
                   const int32_t *ranks, double *at, int mmax, void *ws, cudaStream_t s) {
  (void)mmax;
  TBLR_REQUIRE(P.k <= 64, "mixed coupling supports k <= 64");
  TBLR_REQUIRE((reinterpret_cast<uintptr_t>(ws) & 255) == 0, "workspace must be 256-byte aligned");
  const bool same = v == u || P.selfadjoint;  // self-adjoint: the caller passes v = u
  if (!coupling_simt())
    return coupling_tc(P, lay, u, same ? u : v, ranks, at, ws, coupling_mixed_workspace(P), s);
  // FP32 operands once, instead of an FP64 -> FP32 conversion (on GB300's slow
  // FP64 pipe) every time a CTA stages a step.
  const CouplingWs w = coupling_ws(P, ws);
  split_all_coords<<<(unsigned)std::min<int64_t>(cdiv(3 * w.npad, 256), 4096), 256, 0, s>>>(
      lay->pts, P.n, w.npad, P.d, w.ch, w.cl);
  TBLR_TRY(launch_status("split_all_coords"));
  const unsigned g = (unsigned)std::min<int64_t>(cdiv(P.n * P.k, 256), 152 * 16);
  to_f32<<<g, 256, 0, s>>>(u, P.n * P.k, w.u);
  TBLR_TRY(launch_status("to_f32"));
  if (!same) {
    to_f32<<<g, 256, 0, s>>>(v, P.n * P.k, w.v);
    TBLR_TRY(launch_status("to_f32"));
  }
  CouplingWs wv = w;
  if (same) wv.v = w.u;
  return P.kernel == TBLR_KERNEL_LAPLACE2D
             ? coupling_f32_dispatch<TBLR_KERNEL_LAPLACE2D>(P, wv, lay, ranks, at, s)
             : coupling_f32_dispatch<TBLR_KERNEL_LAPLACE3D>(P, wv, lay, ranks, at, s);
}

size_t nearfield_mixed_workspace(const Prob &P, int mmax) {
  const int64_t npad = cdiv(P.n, 64) * 64;
  return align256(sizeof(float) * P.b * P.s3 * P.k * (size_t)mmax) +
         2 * align256(sizeof(float) * 3 * npad) + align256(sizeof(float) * P.n * P.k);
}

int nearfield_mixed(const Prob &P, const tblr_layout *lay, const double *u, const double *at,
                    const double *v, const int64_t *nf_off, int mmax, double *bnear, void *ws,
                    cudaStream_t s) {
  TBLR_REQUIRE(P.k <= 64, "mixed near field supports k <= 64");
  const int64_t npad = cdiv(P.n, 64) * 64;
  char *w = static_cast<char *>(ws);
  float *M = reinterpret_cast<float *>(w);
  float *ch = reinterpret_cast<float *>(w + align256(sizeof(float) * P.b * P.s3 * P.k * (size_t)mmax));
  float *cl = reinterpret_cast<float *>(reinterpret_cast<char *>(ch) +
                                        align256(sizeof(float) * 3 * npad));
  float *vt = reinterpret_cast<float *>(reinterpret_cast<char *>(cl) +
                                       align256(sizeof(float) * 3 * npad));
  split_all_coords<<<(unsigned)std::min<int64_t>(cdiv(3 * npad, 256), 4096), 256, 0, s>>>(
      lay->pts, P.n, npad, P.d, ch, cl);
  TBLR_TRY(launch_status("split_all_coords"));
  transpose_v_f32<<<(unsigned)std::min<int64_t>(cdiv(P.n * P.k, 256), 152 * 16), 256, 0, s>>>(
      v, P.n, P.k, vt);
  TBLR_TRY(launch_status("transpose_v_f32"));
  const size_t smem_lr = sizeof(float) * 64 * (kAS + kVS) + sizeof(int) * P.b;
  TBLR_REQUIRE(smem_lr <= 220 * 1024, "mixed near field: too many boxes for the probe set");
  TBLR_CUDA(cudaFuncSetAttribute(nf_lowrank_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_lr));
  nf_lowrank_f32_kernel<<<dim3((unsigned)P.b, (unsigned)P.s3, (unsigned)cdiv(mmax, kQT)), kThreads,
                          smem_lr, s>>>(lay->offsets, lay->nbr, lay->nnbr, lay->colour, (int)P.b,
                                        P.s3, P.k, mmax, P.nearfield, at, vt, P.n, M);
  TBLR_TRY(launch_status("nf_lowrank_f32_kernel"));
  const size_t smem_b = sizeof(float) * (kBT * (P.k + 1) + P.k * (kBT + 4) + kNSC * 6 * kBT) +
                        sizeof(int) * P.b;
  TBLR_REQUIRE(smem_b <= 220 * 1024, "mixed near field: too many boxes for the probe set");
  const int tiles = (int)cdiv(mmax, kBT);
  const dim3 grid((unsigned)P.b, (unsigned)P.s3, (unsigned)(tiles * tiles));
  if (P.kernel == TBLR_KERNEL_LAPLACE2D) {
    auto kern = nf_block_f32_kernel<TBLR_KERNEL_LAPLACE2D>;
    TBLR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
    kern<<<grid, kThreads, smem_b, s>>>(ch, cl, npad, lay->offsets, lay->nbr, lay->nnbr,
                                         lay->colour, (int)P.b, P.s3, P.k, mmax, P.nearfield, u,
                                         M, nf_off, bnear);
  } else {
    auto kern = nf_block_f32_kernel<TBLR_KERNEL_LAPLACE3D>;
    TBLR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
    kern<<<grid, kThreads, smem_b, s>>>(ch, cl, npad, lay->offsets, lay->nbr, lay->nnbr,
                                         lay->colour, (int)P.b, P.s3, P.k, mmax, P.nearfield, u,
                                         M, nf_off, bnear);
  }
  return launch_status("nf_block_f32_kernel");
}

}  // namespace tblr
