// Steps II and III of reconstruct_tag (Table 1), FP64:
//   a7 coupling   Atilde_ij = U_i^T A_ij V_j for all box pairs   (§2.5, Table 1 step 2)
//   a8 near field B_ij for j in N_i from the identity probes     (§6.1 eq. sparse_struct_ids)
// A's blocks are regenerated tile by tile; A V and the probe products are
// never stored (V is block diagonal, so (A V)(I_i, block j) = A_ij V_j).
#include "common.cuh"
#include "recon_mixed.cuh"

namespace tblr {
namespace {

constexpr int kThreads = 256;
constexpr int kKMax = 64;
constexpr int kT = 32;  // rows and columns of one generated tile

// CTA per (i, j): for each 32-row slice of box i, W = A(slice, I_j) V_j
// (32 x k) then Atilde_ij += U_i(slice)^T W.
template <class Op>
__global__ void __launch_bounds__(kThreads) coupling_kernel(Op op, const int32_t *__restrict__ offsets,
                                                            const int32_t *__restrict__ ranks,
                                                            const double *__restrict__ U,
                                                            const double *__restrict__ V, int k,
                                                            int b, int sym,
                                                            double *__restrict__ At) {
  extern __shared__ double sm[];
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
  double *As = sm;                  // [kT][kT + 1]
  double *Vs = As + kT * (kT + 1);  // [kT][k]
  double *Ws = Vs + kT * k;         // [kT][k]
  double *Us = Ws + kT * k;         // [kT][k]
  double *Acc = Us + kT * k;        // [k][k]
  for (int idx = tid; idx < k * k; idx += kThreads) Acc[idx] = 0.0;
  constexpr int NW = kT * kKMax / kThreads;
  const int nout = kT * k;
  for (int r0 = 0; r0 < mi; r0 += kT) {
    double w[NW];
#pragma unroll
    for (int u = 0; u < NW; ++u) w[u] = 0.0;
    for (int c0 = 0; c0 < mj; c0 += kT) {
      __syncthreads();
      for (int idx = tid; idx < kT * kT; idx += kThreads) {
        const int rr = idx / kT, cc = idx % kT;
        double v = 0.0;
        if (r0 + rr < mi && c0 + cc < mj) v = op((int64_t)oi + r0 + rr, (int64_t)oj + c0 + cc);
        As[rr * (kT + 1) + cc] = v;
      }
      for (int idx = tid; idx < nout; idx += kThreads) {
        const int cc = idx / k, t = idx % k;
        Vs[idx] = (c0 + cc < mj) ? V[((int64_t)oj + c0 + cc) * k + t] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < NW; ++u) {
        const int idx = tid + kThreads * u;
        if (idx < nout) {
          const int rr = idx / k, t = idx % k;
          double acc = w[u];
#pragma unroll 8
          for (int cc = 0; cc < kT; ++cc) acc = fma(As[rr * (kT + 1) + cc], Vs[cc * k + t], acc);
          w[u] = acc;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < NW; ++u) {
      const int idx = tid + kThreads * u;
      if (idx < nout) Ws[idx] = w[u];
    }
    for (int idx = tid; idx < nout; idx += kThreads) {
      const int rr = idx / k, a = idx % k;
      Us[idx] = (r0 + rr < mi) ? U[((int64_t)oi + r0 + rr) * k + a] : 0.0;
    }
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += kThreads) {
      const int a = idx / k, t = idx % k;
      double s = 0.0;
      for (int rr = 0; rr < kT; ++rr) s = fma(Us[rr * k + a], Ws[rr * k + t], s);
      Acc[idx] += s;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < k * k; idx += kThreads) {
    const int a = idx / k, t = idx % k;
    const double val = (a < ki && t < kj) ? Acc[idx] : 0.0;
    out[idx] = val;
    if (mirror) out_t[(int64_t)t * k + a] = val;
  }
}

// M_is = sum_{c in set} Atilde_ic V_c(0:m_j, :)^T  (k x m_j; rows of V_c
// beyond m_c count as zero).  M[((i*S3 + s)*k + a)*mmax + q].
__global__ void __launch_bounds__(kThreads) nf_lowrank_kernel(
    const int32_t *__restrict__ offsets, const int32_t *__restrict__ nbr,
    const int32_t *__restrict__ nnbr, const int32_t *__restrict__ colour, int b, int s3, int k,
    int mmax, int mode, const double *__restrict__ At, const double *__restrict__ V,
    double *__restrict__ M) {
  extern __shared__ int set[];
  const int i = blockIdx.x, s = blockIdx.y;
  if (s >= nnbr[i]) return;
  const int j = nbr[(int64_t)i * s3 + s];
  const int mj = offsets[j + 1] - offsets[j];
  const int ns = block_probe_set(j, mode, colour, b, set);
  double *out = M + ((int64_t)i * s3 + s) * k * mmax;
  for (int idx = threadIdx.x; idx < k * mj; idx += kThreads) {
    const int a = idx / mj, q = idx % mj;
    double acc = 0.0;
    for (int u = 0; u < ns; ++u) {
      const int c = set[u];
      const int oc = offsets[c];
      if (q >= offsets[c + 1] - oc) continue;
      const double *atr = At + (((int64_t)i * b + c) * k + a) * k;
      const double *vr = V + ((int64_t)oc + q) * k;
      for (int t = 0; t < k; ++t) acc = fma(atr[t], vr[t], acc);
    }
    out[(int64_t)a * mmax + q] = acc;
  }
}

// B_ij(p, q) = sum_{c in set, q < m_c} A(I_i[p], I_c[q]) - U_i(p, :) M_is(:, q).
template <class Op>
__global__ void __launch_bounds__(kThreads) nf_block_kernel(
    Op op, const int32_t *__restrict__ offsets, const int32_t *__restrict__ nbr,
    const int32_t *__restrict__ nnbr, const int32_t *__restrict__ colour, int b, int s3, int k,
    int mmax, int mode, const double *__restrict__ U, const double *__restrict__ M,
    const int64_t *__restrict__ nf_off, double *__restrict__ Bn) {
  extern __shared__ int set[];
  const int i = blockIdx.x, s = blockIdx.y;
  if (s >= nnbr[i]) return;
  const int j = nbr[(int64_t)i * s3 + s];
  const int oi = offsets[i], mi = offsets[i + 1] - oi;
  const int mj = offsets[j + 1] - offsets[j];
  const int ns = block_probe_set(j, mode, colour, b, set);
  const double *Mi = M + ((int64_t)i * s3 + s) * k * mmax;
  double *out = Bn + nf_off[(int64_t)i * s3 + s];
  for (int idx = threadIdx.x; idx < mi * mj; idx += kThreads) {
    const int p = idx / mj, q = idx % mj;
    const int64_t gp = (int64_t)oi + p;
    double acc = 0.0;
    for (int u = 0; u < ns; ++u) {
      const int c = set[u];
      const int oc = offsets[c];
      if (q < offsets[c + 1] - oc) acc += op(gp, (int64_t)oc + q);
    }
    const double *ur = U + gp * k;
    for (int a = 0; a < k; ++a) acc = fma(-ur[a], Mi[(int64_t)a * mmax + q], acc);
    out[idx] = acc;
  }
}

}  // namespace
}  // namespace tblr

using namespace tblr;

extern "C" size_t tblr_coupling_workspace(const tblr_problem *prob) {
  Prob P;
  if (check_problem(prob, &P) != TBLR_OK) return 0;
  return (P.precision == TBLR_MIXED && symmetric_kernel(P.kernel)) ? coupling_mixed_workspace(P)
                                                                    : 0;
}

extern "C" int tblr_coupling(const tblr_problem *prob, const tblr_layout *lay, const double *dense,
                             const double *u, const double *v, const int32_t *ranks,
                             int32_t m_max, double *at, void *ws, size_t ws_bytes,
                             void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_TRY(check_layout(P, lay));
  TBLR_REQUIRE(u && v && ranks && at, "u, v, ranks and at must be non-NULL");
  TBLR_REQUIRE(P.k <= kKMax, "coupling supports k <= %d", kKMax);
  TBLR_REQUIRE(m_max >= 0, "m_max must be >= 0");
  cudaStream_t s = as_stream(stream);
  if (P.precision == TBLR_MIXED && symmetric_kernel(P.kernel)) {
    TBLR_REQUIRE(ws != nullptr && ws_bytes >= coupling_mixed_workspace(P),
                 "coupling workspace too small");
    return coupling_mixed(P, lay, u, v, ranks, at, m_max, ws, s);
  }
  const size_t smem = sizeof(double) * (kT * (kT + 1) + 3 * kT * P.k + P.k * P.k);
  return with_operator(P, lay, dense, 0, [&](auto op) {
    auto kern = coupling_kernel<decltype(op)>;
    TBLR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<dim3((unsigned)P.b, (unsigned)P.b), kThreads, smem, s>>>(op, lay->offsets, ranks, u, v,
                                                                    P.k, (int)P.b,
                                                                    P.selfadjoint ? 1 : 0, at);
    return launch_status("coupling_kernel");
  });
}

extern "C" size_t tblr_nearfield_workspace(const tblr_problem *prob, int32_t m_max) {
  Prob P;
  if (check_problem(prob, &P) != TBLR_OK || m_max < 0) return 0;
  if (P.precision == TBLR_MIXED && symmetric_kernel(P.kernel))
    return nearfield_mixed_workspace(P, m_max);
  return align256(sizeof(double) * P.b * P.s3 * P.k * (size_t)m_max);
}

extern "C" int tblr_nearfield(const tblr_problem *prob, const tblr_layout *lay, const double *dense,
                              const double *u, const double *at, const double *v,
                              const int32_t *ranks, const int64_t *nf_off, int32_t m_max,
                              double *bnear, void *ws, size_t ws_bytes, void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_TRY(check_layout(P, lay));
  (void)ranks;
  TBLR_REQUIRE(u && at && v && nf_off && bnear, "u, at, v, nf_off and bnear must be non-NULL");
  TBLR_REQUIRE(m_max >= 0, "m_max must be >= 0");
  if (m_max == 0) return TBLR_OK;
  TBLR_REQUIRE(ws != nullptr && ws_bytes >= tblr_nearfield_workspace(prob, m_max),
               "nearfield workspace too small");
  cudaStream_t s = as_stream(stream);
  if (P.precision == TBLR_MIXED && symmetric_kernel(P.kernel))
    return nearfield_mixed(P, lay, u, at, v, nf_off, m_max, bnear, ws, s);
  double *M = static_cast<double *>(ws);
  const size_t smem = sizeof(int) * P.b;
  const dim3 grid((unsigned)P.b, (unsigned)P.s3);
  nf_lowrank_kernel<<<grid, kThreads, smem, s>>>(lay->offsets, lay->nbr, lay->nnbr, lay->colour,
                                                 (int)P.b, P.s3, P.k, m_max, P.nearfield, at, v, M);
  TBLR_TRY(launch_status("nf_lowrank_kernel"));
  return with_operator(P, lay, dense, 0, [&](auto op) {
    nf_block_kernel<<<grid, kThreads, smem, s>>>(op, lay->offsets, lay->nbr, lay->nnbr, lay->colour,
                                                 (int)P.b, P.s3, P.k, m_max, P.nearfield, u, M,
                                                 nf_off, bnear);
    return launch_status("nf_block_kernel");
  });
}
