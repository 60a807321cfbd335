// Whole-pipeline entry points: tblr_compress (device buffers) and
// tblr_compress_host (host buffers, end to end), reconstruct_tag of Table 1.
#include <mutex>
#include <vector>

#include "common.cuh"

using namespace tblr;

namespace {

struct WsPlan {
  size_t omega, s, r, col, sketch, cpl, nf, total;
};

WsPlan plan_workspace(const Prob &P, const tblr_problem *prob, int32_t m_max) {
  WsPlan w;
  const bool tagged = P.tagged;
  w.omega = tagged ? 0 : align256(sizeof(double) * 2 * P.C * P.n);
  w.s = align256(sizeof(double) * P.n * P.r);
  w.r = P.selfadjoint ? 0 : w.s;
  w.col = align256(tblr_col_workspace(prob));
  w.sketch = align256(tagged ? tblr_tagged_sketch_workspace(prob) : tblr_sketch_workspace(prob));
  w.cpl = align256(tblr_coupling_workspace(prob));
  w.nf = align256(tblr_nearfield_workspace(prob, m_max));
  w.total = w.omega + w.s + w.r + w.col + w.sketch + w.cpl + w.nf;
  return w;
}

}  // namespace

extern "C" size_t tblr_compress_workspace(const tblr_problem *prob, int32_t m_max) {
  Prob P;
  if (check_problem(prob, &P) != TBLR_OK) return 0;
  return plan_workspace(P, prob, m_max).total;
}

extern "C" int tblr_compress(const tblr_problem *prob, const tblr_layout *lay, const double *dense,
                             const double *T, const double *G, const double *H, double *yz,
                             double *z, double *tau, double *rho, double *u, double *v,
                             int32_t *ranks, double *at, const int64_t *nf_off, int32_t m_max,
                             double *bnear, void *ws, size_t ws_bytes, void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_TRY(check_layout(P, lay));
  const bool tagged = P.tagged;
  TBLR_REQUIRE(T && G && H && (yz || tagged) && z && tau && rho && u && v && ranks && at &&
                   nf_off && bnear,
               "every input and output pointer must be non-NULL");
  const WsPlan w = plan_workspace(P, prob, m_max);
  TBLR_REQUIRE(ws != nullptr && ws_bytes >= w.total, "compress workspace too small (%zu < %zu)",
               ws_bytes, w.total);
  char *base = static_cast<char *>(ws);
  double *omega = reinterpret_cast<double *>(base);
  double *S = reinterpret_cast<double *>(base + w.omega);
  double *R = reinterpret_cast<double *>(base + w.omega + w.s);
  char *colws = base + w.omega + w.s + w.r;
  char *skws = colws + w.col;
  char *cplws = skws + w.sketch;
  char *nfws = cplws + w.cpl;
  // Step I (Algorithm 2): test matrices, sketch, decode, combine, col.  The
  // tag-factored sketch decodes first and forms S and R without Y and Z.
  if (tagged) {
    TBLR_TRY(tblr_decode(prob, lay, T, z, tau, rho, stream));
    TBLR_TRY(tblr_tagged_sketch(prob, lay, dense, tau, G, H, S, R, skws, w.sketch, stream));
  } else {
    TBLR_TRY(tblr_test_matrices(prob, lay, T, G, H, omega, stream));
    TBLR_TRY(tblr_sketch(prob, lay, dense, omega, yz, skws, w.sketch, stream));
    TBLR_TRY(tblr_decode(prob, lay, T, z, tau, rho, stream));
    TBLR_TRY(tblr_combine(prob, lay, yz, z, S, R, stream));
  }
  TBLR_TRY(tblr_col(prob, lay, S, u, ranks, colws, w.col, stream));
  if (P.selfadjoint) {
    // A = A^T and H = G give R = S, hence V = U.
    TBLR_CUDA(cudaMemcpyAsync(v, u, sizeof(double) * P.n * P.k, cudaMemcpyDeviceToDevice,
                              as_stream(stream)));
  } else {
    TBLR_TRY(tblr_col(prob, lay, R, v, ranks, colws, w.col, stream));
  }
  // Step II (Table 1): Atilde = U^T (A V).
  TBLR_TRY(tblr_coupling(prob, lay, dense, u, v, ranks, m_max, at, cplws, w.cpl, stream));
  // Step III (Table 1): near field from the identity probes.
  return tblr_nearfield(prob, lay, dense, u, at, v, ranks, nf_off, m_max, bnear, nfws, w.nf, stream);
}

// ------------------------------------------------------------ host buffers
namespace {

struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
};

struct DeviceCache {
  std::mutex mu;
  int device = -1;
  DevBuf b[24];
};

DeviceCache &cache() {
  static DeviceCache c;
  return c;
}

int ensure(DevBuf &d, size_t bytes) {
  bytes = align256(bytes == 0 ? 256 : bytes);
  if (d.cap >= bytes) return TBLR_OK;
  if (d.p) TBLR_CUDA(cudaFree(d.p));
  d.p = nullptr;
  d.cap = 0;
  TBLR_CUDA(cudaMalloc(&d.p, bytes));
  d.cap = bytes;
  return TBLR_OK;
}

}  // namespace

extern "C" int tblr_compress_host(const tblr_problem *prob, const double *points_h,
                                  const double *T_h, const double *G_h, const double *H_h,
                                  const double *dense_h, int32_t *perm_h, int32_t *offsets_h,
                                  int32_t *nbr_h, int32_t *ranks_h, double *u_h, double *v_h,
                                  double *at_h, double *bnear_h, int64_t bnear_capacity,
                                  int64_t *bnear_size, void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_REQUIRE(points_h && T_h && G_h && H_h && perm_h && offsets_h && nbr_h && ranks_h && u_h &&
                   v_h && at_h && bnear_size,
               "host pointers must be non-NULL");
  TBLR_REQUIRE(P.kernel != TBLR_KERNEL_DENSE || dense_h != nullptr, "dense operator needs dense_h");
  DeviceCache &dc = cache();
  std::lock_guard<std::mutex> lock(dc.mu);
  int dev = 0;
  TBLR_CUDA(cudaGetDevice(&dev));
  if (dc.device != dev) {
    for (auto &x : dc.b)
      if (x.p) cudaFree(x.p), x.p = nullptr, x.cap = 0;
    dc.device = dev;
  }
  cudaStream_t s = as_stream(stream);
  const int64_t n = P.n, b = P.b, k = P.k, r = P.r, s3 = P.s3, ell = P.ell, C = P.C;
  enum { PTS, T_, G_, H_, DN, PERM, BOX, OFF, NBR, NNBR, COL, SPTS, TWS, NFOFF, MMAX, YZ, Z, TAU,
         RHO, U, V, RANKS, AT, BN };
  TBLR_TRY(ensure(dc.b[PTS], sizeof(double) * n * P.d));
  TBLR_TRY(ensure(dc.b[T_], sizeof(double) * b * ell));
  TBLR_TRY(ensure(dc.b[G_], sizeof(double) * n * r));
  TBLR_TRY(ensure(dc.b[H_], sizeof(double) * n * r));
  if (P.kernel == TBLR_KERNEL_DENSE) TBLR_TRY(ensure(dc.b[DN], sizeof(double) * n * n));
  TBLR_TRY(ensure(dc.b[PERM], sizeof(int32_t) * n));
  TBLR_TRY(ensure(dc.b[BOX], sizeof(int32_t) * n));
  TBLR_TRY(ensure(dc.b[OFF], sizeof(int32_t) * (b + 1)));
  TBLR_TRY(ensure(dc.b[NBR], sizeof(int32_t) * b * s3));
  TBLR_TRY(ensure(dc.b[NNBR], sizeof(int32_t) * b));
  TBLR_TRY(ensure(dc.b[COL], sizeof(int32_t) * b));
  TBLR_TRY(ensure(dc.b[SPTS], sizeof(double) * n * P.d));
  TBLR_TRY(ensure(dc.b[TWS], tblr_tessellate_workspace(prob)));
  TBLR_TRY(ensure(dc.b[NFOFF], sizeof(int64_t) * (b * s3 + 1)));
  TBLR_TRY(ensure(dc.b[MMAX], sizeof(int32_t)));
  auto D = [&](int id) { return static_cast<double *>(dc.b[id].p); };
  auto I32 = [&](int id) { return static_cast<int32_t *>(dc.b[id].p); };
  TBLR_CUDA(cudaMemcpyAsync(D(PTS), points_h, sizeof(double) * n * P.d, cudaMemcpyHostToDevice, s));
  TBLR_CUDA(cudaMemcpyAsync(D(T_), T_h, sizeof(double) * b * ell, cudaMemcpyHostToDevice, s));
  TBLR_CUDA(cudaMemcpyAsync(D(G_), G_h, sizeof(double) * n * r, cudaMemcpyHostToDevice, s));
  TBLR_CUDA(cudaMemcpyAsync(D(H_), H_h, sizeof(double) * n * r, cudaMemcpyHostToDevice, s));
  if (P.kernel == TBLR_KERNEL_DENSE)
    TBLR_CUDA(cudaMemcpyAsync(D(DN), dense_h, sizeof(double) * n * n, cudaMemcpyHostToDevice, s));
  tblr_layout lay{I32(PERM), I32(BOX), I32(OFF), I32(NBR), I32(NNBR), I32(COL), D(SPTS)};
  TBLR_TRY(tblr_tessellate(prob, D(PTS), &lay, dc.b[TWS].p, dc.b[TWS].cap, stream));
  int64_t *nf_off = static_cast<int64_t *>(dc.b[NFOFF].p);
  TBLR_TRY(tblr_nearfield_offsets(prob, &lay, nf_off, I32(MMAX), stream));
  int64_t total = 0;
  int32_t m_max = 0;
  TBLR_CUDA(cudaMemcpyAsync(&total, nf_off + b * s3, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaMemcpyAsync(&m_max, I32(MMAX), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaStreamSynchronize(s));
  *bnear_size = total;
  if (total > bnear_capacity || (total > 0 && bnear_h == nullptr)) {
    set_error("near-field output needs %lld doubles, capacity %lld", (long long)total,
              (long long)bnear_capacity);
    return TBLR_EWORKSPACE;
  }
  TBLR_TRY(ensure(dc.b[YZ], sizeof(double) * n * 2 * C));
  TBLR_TRY(ensure(dc.b[Z], sizeof(double) * b * ell));
  TBLR_TRY(ensure(dc.b[TAU], sizeof(double) * b * b));
  TBLR_TRY(ensure(dc.b[RHO], sizeof(double) * b));
  TBLR_TRY(ensure(dc.b[U], sizeof(double) * n * k));
  TBLR_TRY(ensure(dc.b[V], sizeof(double) * n * k));
  TBLR_TRY(ensure(dc.b[RANKS], sizeof(int32_t) * b));
  TBLR_TRY(ensure(dc.b[AT], sizeof(double) * b * b * k * k));
  TBLR_TRY(ensure(dc.b[BN], sizeof(double) * total));
  const size_t wsb = tblr_compress_workspace(prob, m_max);
  TBLR_TRY(ensure(dc.b[TWS], wsb > dc.b[TWS].cap ? wsb : dc.b[TWS].cap));
  TBLR_TRY(tblr_compress(prob, &lay, P.kernel == TBLR_KERNEL_DENSE ? D(DN) : nullptr, D(T_), D(G_),
                         D(H_), D(YZ), D(Z), D(TAU), D(RHO), D(U), D(V), I32(RANKS), D(AT), nf_off,
                         m_max, D(BN), dc.b[TWS].p, dc.b[TWS].cap, stream));
  TBLR_CUDA(cudaMemcpyAsync(perm_h, I32(PERM), sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaMemcpyAsync(offsets_h, I32(OFF), sizeof(int32_t) * (b + 1), cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaMemcpyAsync(nbr_h, I32(NBR), sizeof(int32_t) * b * s3, cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaMemcpyAsync(ranks_h, I32(RANKS), sizeof(int32_t) * b, cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaMemcpyAsync(u_h, D(U), sizeof(double) * n * k, cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaMemcpyAsync(v_h, D(V), sizeof(double) * n * k, cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaMemcpyAsync(at_h, D(AT), sizeof(double) * b * b * k * k, cudaMemcpyDeviceToHost, s));
  if (total > 0)
    TBLR_CUDA(cudaMemcpyAsync(bnear_h, D(BN), sizeof(double) * total, cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaStreamSynchronize(s));
  return TBLR_OK;
}

extern "C" int tblr_release_device_cache(void) {
  DeviceCache &dc = cache();
  std::lock_guard<std::mutex> lock(dc.mu);
  for (auto &x : dc.b)
    if (x.p) {
      TBLR_CUDA(cudaFree(x.p));
      x.p = nullptr;
      x.cap = 0;
    }
  dc.device = -1;
  return TBLR_OK;
}
