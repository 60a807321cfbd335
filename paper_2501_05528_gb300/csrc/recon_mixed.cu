// Steps II and III (Table 1) for the mixed-precision path, on the FP32 pipes
// (GB300 runs FP32 FMA ~60x faster than FP64).  Kernel entries come from
// double-float coordinates (~2^-23 relative), products are FP32, and every
// long sum is accumulated in FP32 chunks of at most 32 terms that are added
// into Kahan-compensated FP32 sums, so each output keeps ~1e-7 relative error.
//   coupling   Atilde_ij = U_i^T (A_ij V_j)                  (§2.5, Table 1 step 2)
//   nf lowrank M_is = sum_{c in set} Atilde_ic V_c(0:m_j,:)^T  (§6.1 eq. sparse_struct_ids)
//   nf block   B_ij = sum_{c in set} A(I_i, I_c(0:m_j)) - U_i M_is
#include "kernels_f32.cuh"
#include "recon_mixed.cuh"

namespace tblr {
namespace {

constexpr int kThreads = 256;
constexpr int kSlab = 32;  // V columns per coupling CTA

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

// CTA per (i, j, slab of 32 columns of V_j).  Phase 1: W = A_ij V_j(:, slab)
// row by row (one thread per row of box i), kept in shared memory.  Phase 2:
// Atilde_ij(:, slab) = U_i^T W.
template <int KERNEL>
__global__ void __launch_bounds__(kThreads) coupling_f32_kernel(
    const double *__restrict__ pts, int64_t n, int d, const int32_t *__restrict__ offsets,
    const int32_t *__restrict__ ranks, const double *__restrict__ U, const double *__restrict__ V,
    int k, int b, int mmax, double *__restrict__ At) {
  extern __shared__ float sf[];
  const int i = blockIdx.x, j = blockIdx.y, c0 = blockIdx.z * kSlab, tid = threadIdx.x;
  const int oi = offsets[i], mi = offsets[i + 1] - oi;
  const int oj = offsets[j], mj = offsets[j + 1] - oj;
  const int ki = ranks[i], kj = ranks[j];
  double *out = At + ((int64_t)i * b + j) * k * k;
  if (ki == 0 || kj == 0 || c0 >= kj) {
    for (int idx = tid; idx < k * kSlab; idx += kThreads) {
      const int a = idx / kSlab, c = c0 + idx % kSlab;
      if (c < k) out[(int64_t)a * k + c] = 0.0;
    }
    return;
  }
  float *Vs = sf;                       // [mmax][kSlab]
  float *qh = Vs + mmax * kSlab;        // [3][mmax]
  float *ql = qh + 3 * mmax;            // [3][mmax]
  float *Ws = ql + 3 * mmax;            // [mmax][kSlab + 1]
  for (int idx = tid; idx < mj * kSlab; idx += kThreads) {
    const int q = idx / kSlab, c = c0 + idx % kSlab;
    Vs[idx] = (c < kj) ? (float)V[((int64_t)oj + q) * k + c] : 0.f;
  }
  for (int idx = tid; idx < 3 * mj; idx += kThreads) {
    const int ax = idx / mj, q = idx % mj;
    float h = 0.f, l = 0.f;
    if (ax < d) split_coord(pts[ax * n + oj + q], h, l);
    qh[ax * mmax + q] = h;
    ql[ax * mmax + q] = l;
  }
  __syncthreads();
  for (int p = tid; p < mi; p += kThreads) {
    float rh[3], rl[3];
    load_point<KERNEL>(pts, n, d, (int64_t)oi + p, rh, rl);
    float acc[kSlab], hi[kSlab], cc[kSlab];
#pragma unroll
    for (int c = 0; c < kSlab; ++c) acc[c] = hi[c] = cc[c] = 0.f;
    for (int q = 0; q < mj; ++q) {
      const float ch[3] = {qh[q], qh[mmax + q], qh[2 * mmax + q]};
      const float cl[3] = {ql[q], ql[mmax + q], ql[2 * mmax + q]};
      float v = entry_f32<KERNEL>(rh, rl, ch, cl);
      if (i == j && p == q) v = 0.f;
      const float4 *vr = reinterpret_cast<const float4 *>(Vs + q * kSlab);
#pragma unroll
      for (int c4 = 0; c4 < kSlab / 4; ++c4) {
        const float4 w = vr[c4];
        acc[4 * c4] = fmaf(v, w.x, acc[4 * c4]);
        acc[4 * c4 + 1] = fmaf(v, w.y, acc[4 * c4 + 1]);
        acc[4 * c4 + 2] = fmaf(v, w.z, acc[4 * c4 + 2]);
        acc[4 * c4 + 3] = fmaf(v, w.w, acc[4 * c4 + 3]);
      }
      if ((q & 31) == 31 || q == mj - 1) {
#pragma unroll
        for (int c = 0; c < kSlab; ++c) {
          kahan_add(hi[c], cc[c], acc[c]);
          acc[c] = 0.f;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < kSlab; ++c) Ws[p * (kSlab + 1) + c] = hi[c] - cc[c];
  }
  __syncthreads();
  for (int idx = tid; idx < k * kSlab; idx += kThreads) {
    const int a = idx / kSlab, c = idx % kSlab;
    if (c0 + c >= k) continue;
    double res = 0.0;
    if (a < ki && c0 + c < kj) {
      float acc = 0.f, hi = 0.f, cc = 0.f;
      for (int p = 0; p < mi; ++p) {
        acc = fmaf((float)U[((int64_t)oi + p) * k + a], Ws[p * (kSlab + 1) + c], acc);
        if ((p & 31) == 31 || p == mi - 1) {
          kahan_add(hi, cc, acc);
          acc = 0.f;
        }
      }
      res = (double)hi - (double)cc;
    }
    out[(int64_t)a * k + c0 + c] = res;
  }
}

// The boxes whose columns enter B_ij (every box of colour(j) for the probe
// reading, j alone for the exact one), in shared memory.
__device__ int probe_set_f(int j, int mode, const int32_t *__restrict__ colour, int b, int *set) {
  __shared__ int cnt;
  if (threadIdx.x == 0) {
    int c = 0;
    if (mode == TBLR_NEARFIELD_EXACT) {
      set[c++] = j;
    } else {
      const int g = colour[j];
      for (int x = 0; x < b; ++x)
        if (colour[x] == g) set[c++] = x;
    }
    cnt = c;
  }
  __syncthreads();
  return cnt;
}

// CTA per (i, s, 64-column tile of M): M_is(a, q) for a < k, q in the tile.
// Each set member c contributes Atilde_ic V_c(q, :)^T; that contribution is
// summed in FP32 and added to Kahan sums.
constexpr int kQT = 64;
__global__ void __launch_bounds__(kThreads) nf_lowrank_f32_kernel(
    const int32_t *__restrict__ offsets, const int32_t *__restrict__ nbr,
    const int32_t *__restrict__ nnbr, const int32_t *__restrict__ colour, int b, int s3, int k,
    int mmax, int mode, const double *__restrict__ At, const double *__restrict__ V,
    float *__restrict__ M) {
  extern __shared__ float sf[];
  const int i = blockIdx.x, s = blockIdx.y, q0 = blockIdx.z * kQT, tid = threadIdx.x;
  if (s >= nnbr[i]) return;
  const int j = nbr[(int64_t)i * s3 + s];
  const int mj = offsets[j + 1] - offsets[j];
  if (q0 >= mj) return;
  float *As = sf;                 // [k][k]
  float *Vs = As + k * k;         // [kQT][k + 1]
  int *set = reinterpret_cast<int *>(Vs + kQT * (k + 1));
  const int ns = probe_set_f(j, mode, colour, b, set);
  const int q = tid % kQT, ag = tid / kQT;  // 4 groups of rows a = ag + 4 u
  constexpr int kU = 16;                    // k <= 64
  float hi[kU], cc[kU];
#pragma unroll
  for (int u = 0; u < kU; ++u) hi[u] = cc[u] = 0.f;
  for (int x = 0; x < ns; ++x) {
    const int c = set[x];
    const int oc = offsets[c], mc = offsets[c + 1] - oc;
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += kThreads)
      As[idx] = (float)At[((int64_t)i * b + c) * k * k + idx];
    for (int idx = tid; idx < kQT * k; idx += kThreads) {
      const int qq = idx / k, t = idx % k;
      Vs[qq * (k + 1) + t] = (q0 + qq < mc && q0 + qq < mj) ? (float)V[((int64_t)oc + q0 + qq) * k + t]
                                                             : 0.f;
    }
    __syncthreads();
    float acc[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) acc[u] = 0.f;
    for (int t = 0; t < k; ++t) {
      const float vq = Vs[q * (k + 1) + t];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int a = ag + 4 * u;
        if (a < k) acc[u] = fmaf(As[a * k + t], vq, acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) kahan_add(hi[u], cc[u], acc[u]);
  }
  if (q0 + q < mj) {
    float *out = M + ((int64_t)i * s3 + s) * k * mmax;
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int a = ag + 4 * u;
      if (a < k) out[(int64_t)a * mmax + q0 + q] = hi[u] - cc[u];
    }
  }
}

// B_ij(p, q) = sum_{c in set, q < m_c} A(I_i[p], I_c[q]) - U_i(p, :) M_is(:, q).
template <int KERNEL>
__global__ void __launch_bounds__(kThreads) nf_block_f32_kernel(
    const float *__restrict__ chp, const float *__restrict__ clp, int64_t npad,
    const int32_t *__restrict__ offsets, const int32_t *__restrict__ nbr,
    const int32_t *__restrict__ nnbr, const int32_t *__restrict__ colour, int b, int s3, int k,
    int mmax, int mode, const double *__restrict__ U, const float *__restrict__ M,
    const int64_t *__restrict__ nf_off, double *__restrict__ Bn) {
  extern __shared__ int set[];
  const int i = blockIdx.x, s = blockIdx.y;
  if (s >= nnbr[i]) return;
  const int j = nbr[(int64_t)i * s3 + s];
  const int oi = offsets[i], mi = offsets[i + 1] - oi;
  const int mj = offsets[j + 1] - offsets[j];
  const int ns = probe_set_f(j, mode, colour, b, set);
  const float *Mi = M + ((int64_t)i * s3 + s) * k * mmax;
  double *out = Bn + nf_off[(int64_t)i * s3 + s];
  for (int idx = threadIdx.x; idx < mi * mj; idx += kThreads) {
    const int p = idx / mj, q = idx % mj;
    const int64_t gp = (int64_t)oi + p;
    float rh[3], rl[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      rh[ax] = chp[ax * npad + gp];
      rl[ax] = clp[ax * npad + gp];
    }
    float hi = 0.f, cc = 0.f;
    for (int x = 0; x < ns; ++x) {
      const int c = set[x];
      const int oc = offsets[c];
      if (q >= offsets[c + 1] - oc) continue;
      const int64_t gq = (int64_t)oc + q;
      if (gq == gp) continue;  // zero diagonal
      float qh[3], ql[3];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        qh[ax] = chp[ax * npad + gq];
        ql[ax] = clp[ax * npad + gq];
      }
      kahan_add(hi, cc, entry_f32<KERNEL>(rh, rl, qh, ql));
    }
    float lr = 0.f;
    const double *ur = U + gp * k;
    for (int a = 0; a < k; ++a) lr = fmaf((float)ur[a], Mi[(int64_t)a * mmax + q], lr);
    out[idx] = ((double)hi - (double)cc) - (double)lr;
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

size_t coupling_f32_smem(int mmax) {
  return sizeof(float) * ((size_t)mmax * kSlab + 6 * (size_t)mmax + (size_t)mmax * (kSlab + 1));
}

int coupling_mixed(const Prob &P, const tblr_layout *lay, const double *u, const double *v,
                   const int32_t *ranks, double *at, int mmax, cudaStream_t s) {
  TBLR_REQUIRE(P.k <= 64, "mixed coupling supports k <= 64");
  const size_t smem = coupling_f32_smem(mmax);
  TBLR_REQUIRE(smem <= 220 * 1024, "mixed coupling supports boxes of at most ~780 points");
  const dim3 grid((unsigned)P.b, (unsigned)P.b, (unsigned)cdiv(P.k, kSlab));
  if (P.kernel == TBLR_KERNEL_LAPLACE2D) {
    auto kern = coupling_f32_kernel<TBLR_KERNEL_LAPLACE2D>;
    TBLR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, kThreads, smem, s>>>(lay->pts, P.n, P.d, lay->offsets, ranks, u, v, P.k, (int)P.b,
                                      mmax, at);
  } else {
    auto kern = coupling_f32_kernel<TBLR_KERNEL_LAPLACE3D>;
    TBLR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, kThreads, smem, s>>>(lay->pts, P.n, P.d, lay->offsets, ranks, u, v, P.k, (int)P.b,
                                      mmax, at);
  }
  return launch_status("coupling_f32_kernel");
}

size_t nearfield_mixed_workspace(const Prob &P, int mmax) {
  const int64_t npad = cdiv(P.n, 64) * 64;
  return align256(sizeof(float) * P.b * P.s3 * P.k * (size_t)mmax) +
         2 * align256(sizeof(float) * 3 * npad);
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
  split_all_coords<<<(unsigned)std::min<int64_t>(cdiv(3 * npad, 256), 4096), 256, 0, s>>>(
      lay->pts, P.n, npad, P.d, ch, cl);
  TBLR_TRY(launch_status("split_all_coords"));
  const size_t smem_lr = sizeof(float) * (P.k * P.k + kQT * (P.k + 1)) + sizeof(int) * P.b;
  TBLR_REQUIRE(smem_lr <= 220 * 1024, "mixed near field: too many boxes for the probe set");
  TBLR_CUDA(cudaFuncSetAttribute(nf_lowrank_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_lr));
  nf_lowrank_f32_kernel<<<dim3((unsigned)P.b, (unsigned)P.s3, (unsigned)cdiv(mmax, kQT)), kThreads,
                          smem_lr, s>>>(lay->offsets, lay->nbr, lay->nnbr, lay->colour, (int)P.b,
                                        P.s3, P.k, mmax, P.nearfield, at, v, M);
  TBLR_TRY(launch_status("nf_lowrank_f32_kernel"));
  const size_t smem_b = sizeof(int) * P.b;
  const dim3 grid((unsigned)P.b, (unsigned)P.s3);
  if (P.kernel == TBLR_KERNEL_LAPLACE2D)
    nf_block_f32_kernel<TBLR_KERNEL_LAPLACE2D><<<grid, kThreads, smem_b, s>>>(
        ch, cl, npad, lay->offsets, lay->nbr, lay->nnbr, lay->colour, (int)P.b, P.s3, P.k, mmax,
        P.nearfield, u, M, nf_off, bnear);
  else
    nf_block_f32_kernel<TBLR_KERNEL_LAPLACE3D><<<grid, kThreads, smem_b, s>>>(
        ch, cl, npad, lay->offsets, lay->nbr, lay->nnbr, lay->colour, (int)P.b, P.s3, P.k, mmax,
        P.nearfield, u, M, nf_off, bnear);
  return launch_status("nf_block_f32_kernel");
}

}  // namespace tblr
