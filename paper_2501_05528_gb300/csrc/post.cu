// Batched per-box post-processing, all FP64:
//   a4 tag decode   z_i in null(T(N_i,:)), tau_i = T z_i, rho_i   (§4.1, §5.1, §5.3)
//   a5 combine      S_i = sum_j z_ij Y_j(I_i,:)                   (Algorithm 2; eq. projected_tags)
//   a6 col          U_i = k_i dominant left singular vectors of S_i (§2.3, §2.4)
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace tblr {

// Boxes whose aspect-ratio LP stopped without an optimum (read and reset by
// tblr_decode_lp_failures); such boxes keep the projected vector.
__device__ unsigned int g_lp_failures;

namespace {

// ---------------------------------------------------------------- a4 decode
// One warp per box; lane j holds component j of ell-vectors (ell <= 32).
// The rows of T(N_i,:) are orthonormalised by modified Gram-Schmidt with one
// reorthogonalisation pass, then w = 1/sqrt(ell) is projected onto the
// orthogonal complement (the null space) twice and normalised.
constexpr int kDecWarps = 4;
constexpr int kMaxNbr = 27;

__global__ void __launch_bounds__(32 * kDecWarps) decode_kernel(
    const double *__restrict__ T, int b, int ell, int s3, const int32_t *__restrict__ nbr,
    const int32_t *__restrict__ nnbr, double *__restrict__ z, double *__restrict__ tau,
    double *__restrict__ rho) {
  __shared__ double Q[kDecWarps][kMaxNbr][32];
  __shared__ double zs[kDecWarps][32];
  __shared__ int rows[kDecWarps][kMaxNbr];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * kDecWarps + warp;
  if (i >= b) return;
  const int nb = nnbr[i];
  for (int a = 0; a < nb; ++a) {
    const int row = nbr[(int64_t)i * s3 + a];
    if (lane == 0) rows[warp][a] = row;
    double v = lane < ell ? T[(int64_t)row * ell + lane] : 0.0;
    for (int pass = 0; pass < 2; ++pass)
      for (int c = 0; c < a; ++c) {
        const double qc = Q[warp][c][lane];
        v -= warp_sum(qc * v) * qc;
      }
    v /= sqrt(warp_sum(v * v));
    Q[warp][a][lane] = v;
    __syncwarp();
  }
  double zv = lane < ell ? 1.0 / sqrt((double)ell) : 0.0;
  for (int pass = 0; pass < 2; ++pass)
    for (int c = 0; c < nb; ++c) {
      const double qc = Q[warp][c][lane];
      zv -= warp_sum(qc * zv) * qc;
    }
  zv /= sqrt(warp_sum(zv * zv));
  if (lane < ell) z[(int64_t)i * ell + lane] = zv;
  zs[warp][lane] = zv;
  __syncwarp();
  double amax = 0.0, amin = INFINITY;
  bool anyfar = false;
  for (int q = lane; q < b; q += 32) {
    double t = 0.0;
    for (int j = 0; j < ell; ++j) t = fma(T[(int64_t)q * ell + j], zs[warp][j], t);
    tau[(int64_t)i * b + q] = t;
    bool near = false;
    for (int a = 0; a < nb; ++a) near |= rows[warp][a] == q;
    if (!near) {
      amax = fmax(amax, fabs(t));
      amin = fmin(amin, fabs(t));
      anyfar = true;
    }
  }
  amax = warp_max(amax);
  amin = warp_min(amin);
  anyfar = __any_sync(0xffffffffu, anyfar);
  if (lane == 0) rho[i] = anyfar ? amax / amin : NAN;
}

// --------------------------------------- a4 decode, §5.3 aspect-ratio option
// Per box (one CTA), minimise eq. aspect_ratio over null(T(N_i,:)) inside the
// sign cell of the projected vector decode_kernel wrote: with X an orthonormal
// null basis (s vectors) and c_j = sigma_j X t_j (j in F_i, sigma_j the sign of
// the projected tag), the linear program in x = (a, rho) in R^(s+1)
//     minimise rho  subject to  L_j: c_j^T a >= 1,  U_j: rho - c_j^T a >= 0.
// Active-set primal simplex from the projected vector itself (scaled so its
// smallest projected tag is 1, it is feasible with L_min and U_max active): the
// direction is minus the objective gradient projected on the null space of the
// active rows; a blocking constraint joins the active set; at a vertex (or a
// zero direction) the multipliers y of A_W^T y = e_rho decide optimality, and
// the most negative one leaves.  The active rows are re-factorised (QR by
// modified Gram-Schmidt, twice) each iteration - at most 32 x 32.  The
// constraint values need only t_j^T (X^T a), so c_j is never stored.
constexpr int kLpThreads = 128;
constexpr int kLpRows = 32;  // s + 1 <= ell <= 32

__global__ void __launch_bounds__(kLpThreads) minratio_kernel(
    const double *__restrict__ T, int b, int ell, int s3, const int32_t *__restrict__ nbr,
    const int32_t *__restrict__ nnbr, int max_iter, double *__restrict__ z,
    double *__restrict__ tau, double *__restrict__ rho) {
  __shared__ double Q[kLpRows][32];      // rows of T(N_i, :), then columns of Q of A_W^T
  __shared__ double X[kLpRows][32];      // orthonormal null basis, X[c][l]
  __shared__ double Rm[kLpRows][kLpRows];
  __shared__ double xv[kLpRows], dv[kLpRows], yv[kLpRows], va[32], vd[32];
  __shared__ double rstep[kLpThreads];
  __shared__ int rid[kLpThreads], W[kLpRows + 1], nb_ids[kMaxNbr];
  __shared__ int s_dim, nW, state;  // state: 0 running, 1 optimal, 2 failed
  const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = nnbr[i];
  if (nb >= b || nb >= ell) return;  // no far field, or no null space to move in
  for (int a = tid; a < nb; a += kLpThreads) nb_ids[a] = nbr[(int64_t)i * s3 + a];
  __syncthreads();
  auto is_near = [&](int j) {
    for (int a = 0; a < nb; ++a)
      if (nb_ids[a] == j) return true;
    return false;
  };
  const double *zi = z + (int64_t)i * ell;
  const double *taui = tau + (int64_t)i * b;  // decode_kernel's projected tags (signs)
  // Null basis: warp 0 orthonormalises T(N_i, :)'s rows, then greedily takes the
  // unit vectors e_k with the largest residual off span(rows, X so far).
  if (warp == 0) {
    for (int a = 0; a < nb; ++a) {
      double val = lane < ell ? T[(int64_t)nb_ids[a] * ell + lane] : 0.0;
      for (int pass = 0; pass < 2; ++pass)
        for (int c = 0; c < a; ++c) {
          const double qc = Q[c][lane];
          val -= warp_sum(qc * val) * qc;
        }
      val /= sqrt(warp_sum(val * val));
      Q[a][lane] = val;
      __syncwarp();
    }
    int sd = 0;
    for (int round = 0; round < ell - nb && sd < kLpRows - 1; ++round) {
      double best = -1.0, bestv = 0.0;
      for (int k = 0; k < ell; ++k) {
        double val = lane == k ? 1.0 : 0.0;
        for (int pass = 0; pass < 2; ++pass) {
          for (int c = 0; c < nb; ++c) val -= warp_sum(Q[c][lane] * val) * Q[c][lane];
          for (int c = 0; c < sd; ++c) val -= warp_sum(X[c][lane] * val) * X[c][lane];
        }
        const double nrm = sqrt(warp_sum(val * val));
        if (nrm > best) {
          best = nrm;
          bestv = val;
        }
      }
      if (best < 1e-8) break;
      X[sd][lane] = bestv / best;
      ++sd;
      __syncwarp();
    }
    if (lane == 0) s_dim = sd;
  }
  __syncthreads();
  const int sd = s_dim, nv = sd + 1;
  if (sd <= 1) return;  // a line: the projected vector is already optimal
  auto sgn = [&](int j) { return taui[j] < 0.0 ? -1.0 : 1.0; };
  // t_j^T w for an ell-vector w in shared memory.
  auto tdot = [&](int j, const double *w) {
    double acc = 0.0;
    for (int l = 0; l < ell; ++l) acc = fma(T[(int64_t)j * ell + l], w[l], acc);
    return acc;
  };
  // Start: a0 = coordinates of the projected vector, scaled so min_j c_j^T a0 = 1.
  if (tid < sd) {
    double acc = 0.0;
    for (int l = 0; l < ell; ++l) acc = fma(X[tid][l], zi[l], acc);
    xv[tid] = acc;
  }
  __syncthreads();
  if (tid < ell) {  // va = X^T a
    double acc = 0.0;
    for (int c = 0; c < sd; ++c) acc = fma(X[c][tid], xv[c], acc);
    va[tid] = acc;
  }
  __syncthreads();
  {
    double lo = INFINITY, hi = -INFINITY;
    int jlo = INT_MAX, jhi = INT_MAX;
    for (int j = tid; j < b; j += kLpThreads) {
      if (is_near(j)) continue;
      const double cj = sgn(j) * tdot(j, va);
      if (cj < lo) lo = cj, jlo = j;
      if (cj > hi) hi = cj, jhi = j;
    }
    rstep[tid] = lo;
    rid[tid] = jlo;
    __syncthreads();
    if (tid == 0) {
      double best = INFINITY;
      int bid = INT_MAX;
      for (int t = 0; t < kLpThreads; ++t)
        if (rstep[t] < best || (rstep[t] == best && rid[t] < bid)) best = rstep[t], bid = rid[t];
      yv[0] = best;
      W[0] = bid;
    }
    __syncthreads();
    rstep[tid] = -hi;
    rid[tid] = jhi;
    __syncthreads();
    if (tid == 0) {
      double best = INFINITY;
      int bid = INT_MAX;
      for (int t = 0; t < kLpThreads; ++t)
        if (rstep[t] < best || (rstep[t] == best && rid[t] < bid)) best = rstep[t], bid = rid[t];
      yv[1] = -best;
      W[1] = b + bid;
      nW = 2;
      state = 0;
    }
    __syncthreads();
    const double scale = 1.0 / yv[0];
    if (tid < sd) xv[tid] *= scale;
    if (tid == 0) xv[sd] = yv[1] * scale;
    __syncthreads();
  }
  const double tol_y = 1e-12, tol_d = 1e-11;
  int iter = 0;
  for (; iter < max_iter; ++iter) {
    // QR of A_W^T (columns = active rows) by warp 0: lane = component (nv <= 32).
    if (warp == 0) {
      int w = nW;
      bool dropped = false;
      for (int attempt = 0; attempt < 2; ++attempt) {
        for (int c = 0; c < w; ++c) {
          const int id = W[c];
          const int j = id < b ? id : id - b;
          double row;  // component `lane` of the active row
          if (lane < sd) {
            double acc = 0.0;
            for (int l = 0; l < ell; ++l) acc = fma(X[lane][l], T[(int64_t)j * ell + l], acc);
            row = (id < b ? 1.0 : -1.0) * sgn(j) * acc;
          } else {
            row = lane == sd ? (id < b ? 0.0 : 1.0) : 0.0;
          }
          double val = row;
          for (int k = 0; k < c; ++k) Rm[k][c] = 0.0;
          for (int pass = 0; pass < 2; ++pass)
            for (int k = 0; k < c; ++k) {
              const double h = warp_sum(Q[k][lane] * val);
              if (lane == 0) Rm[k][c] += h;
              val -= h * Q[k][lane];
            }
          const double nrm = sqrt(warp_sum(val * val));
          if (lane == 0) Rm[c][c] = nrm;
          Q[c][lane] = nrm > 0.0 ? val / nrm : 0.0;
          __syncwarp();
        }
        // Direction: d = -(e_rho - Q Q^T e_rho), minus the objective gradient
        // projected on the null space of the active rows.
        double dcomp = lane == sd ? -1.0 : 0.0;
        for (int k = 0; k < w; ++k) dcomp += Q[k][sd] * Q[k][lane];
        const double dn = sqrt(warp_sum(dcomp * dcomp));
        if (w < nv && dn > tol_d) {
          if (lane < nv) dv[lane] = dcomp;
          break;
        }
        if (dropped) {  // a drop left no descent direction: degenerate, stop here
          if (lane == 0) state = 2;
          break;
        }
        // Multipliers: R y = Q^T e_rho (back substitution on lane 0).
        const double qe = lane < w ? Q[lane][sd] : 0.0;
        if (lane < w) yv[lane] = qe;
        __syncwarp();
        if (lane == 0) {
          for (int c = w - 1; c >= 0; --c) {
            double acc = yv[c];
            for (int k = c + 1; k < w; ++k) acc -= Rm[c][k] * yv[k];
            yv[c] = acc / Rm[c][c];
          }
        }
        __syncwarp();
        int q = -1;
        double ymin = -tol_y;
        for (int c = 0; c < w; ++c)
          if (yv[c] < ymin) ymin = yv[c], q = c;
        if (q < 0) {  // all multipliers non-negative: optimal
          if (lane == 0) state = 1;
          break;
        }
        if (lane == 0) {
          for (int c = q; c + 1 < w; ++c) W[c] = W[c + 1];
          nW = w - 1;
        }
        __syncwarp();
        w -= 1;
        dropped = true;
      }
    }
    __syncthreads();
    if (state != 0) break;
    // Ratio test along d over the inactive constraints.
    if (tid < ell) {
      double a1 = 0.0, a2 = 0.0;
      for (int c = 0; c < sd; ++c) {
        a1 = fma(X[c][tid], xv[c], a1);
        a2 = fma(X[c][tid], dv[c], a2);
      }
      va[tid] = a1;
      vd[tid] = a2;
    }
    __syncthreads();
    double dnorm = 0.0;
    for (int c = 0; c < nv; ++c) dnorm = fma(dv[c], dv[c], dnorm);
    dnorm = sqrt(dnorm);
    double best = INFINITY;
    int bid = INT_MAX;
    for (int j = tid; j < b; j += kLpThreads) {
      if (is_near(j)) continue;
      const double sg = sgn(j);
      const double cx = sg * tdot(j, va), cd = sg * tdot(j, vd);
      // L_j: slack c^T a - 1, rate c^T d;  U_j: slack rho - c^T a, rate d_rho - c^T d.
      const double sl[2] = {cx - 1.0, xv[sd] - cx}, rt[2] = {cd, dv[sd] - cd};
      for (int h = 0; h < 2; ++h) {
        const int id = h == 0 ? j : b + j;
        bool active = false;
        for (int c = 0; c < nW; ++c) active |= W[c] == id;
        if (active || rt[h] >= -1e-14 * dnorm) continue;
        const double step = fmax(sl[h], 0.0) / -rt[h];
        if (step < best || (step == best && id < bid)) best = step, bid = id;
      }
    }
    rstep[tid] = best;
    rid[tid] = bid;
    __syncthreads();
    if (tid == 0) {
      double bs = INFINITY;
      int bi = INT_MAX;
      for (int t = 0; t < kLpThreads; ++t)
        if (rstep[t] < bs || (rstep[t] == bs && rid[t] < bi)) bs = rstep[t], bi = rid[t];
      if (bi == INT_MAX || nW >= kLpRows) {
        state = 2;  // unbounded cannot happen (rho >= 1); keep the projected vector
      } else {
        for (int c = 0; c < nv; ++c) xv[c] += bs * dv[c];
        W[nW] = bi;
        nW = nW + 1;
      }
    }
    __syncthreads();
    if (state != 0) break;
  }
  if (state != 1) {  // keep the projected vector and count the failure
    if (tid == 0) atomicAdd(&g_lp_failures, 1u);
    return;
  }
  // z = X^T a / ||X^T a||, then its projected tags and aspect ratio.
  if (tid < ell) {
    double acc = 0.0;
    for (int c = 0; c < sd; ++c) acc = fma(X[c][tid], xv[c], acc);
    va[tid] = acc;
  }
  __syncthreads();
  if (tid == 0) {
    double nn = 0.0;
    for (int l = 0; l < ell; ++l) nn = fma(va[l], va[l], nn);
    yv[0] = 1.0 / sqrt(nn);
  }
  __syncthreads();
  if (tid < ell) {
    va[tid] *= yv[0];
    z[(int64_t)i * ell + tid] = va[tid];
  }
  __syncthreads();
  double amax = 0.0, amin = INFINITY;
  for (int j = tid; j < b; j += kLpThreads) {
    const double t = tdot(j, va);
    tau[(int64_t)i * b + j] = t;
    if (!is_near(j)) {
      amax = fmax(amax, fabs(t));
      amin = fmin(amin, fabs(t));
    }
  }
  amax = warp_max(amax);
  amin = warp_min(amin);
  if (lane == 0) {
    rstep[warp] = amax;
    rstep[4 + warp] = amin;
  }
  __syncthreads();
  if (tid == 0) {
    double gmax = 0.0, gmin = INFINITY;
    for (int w = 0; w < kLpThreads / 32; ++w) {
      gmax = fmax(gmax, rstep[w]);
      gmin = fmin(gmin, rstep[4 + w]);
    }
    rho[i] = gmax / gmin;
  }
}

// --------------------------------------------------------------- a5 combine
__global__ void combine_kernel(const double *__restrict__ yz, const double *__restrict__ z,
                               const int32_t *__restrict__ box_of, int64_t n, int r, int ell,
                               int64_t C, double *__restrict__ s, double *__restrict__ rr) {
  const int64_t total = n * r;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = idx / r;
    const int q = (int)(idx % r);
    const double *zi = z + (int64_t)box_of[p] * ell;
    const double *row = yz + p * 2 * C;
    double a = 0.0, c = 0.0;
    for (int j = 0; j < ell; ++j) {
      const double w = zi[j];
      a = fma(w, row[j * r + q], a);
      c = fma(w, row[C + j * r + q], c);
    }
    s[idx] = a;
    rr[idx] = c;
  }
}

// ------------------------------------------------------------------- a6 col
constexpr int kColThreads = 512;
constexpr int kRMax = 112;

__device__ double block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < kColThreads / 32; ++w) t += red[w];
  __syncthreads();
  return t;
}

// Round-robin (circle) schedule over qq (even) columns: in round rho, column
// qq-1 meets rho and (rho + k, rho - k) mod (qq - 1) meet for k = 1 .. qq/2-1.
__device__ __forceinline__ void jacobi_pair(int rho, int k, int qq, int *a, int *b) {
  const int m = qq - 1;
  if (k == 0) {
    *a = rho;
    *b = m;
  } else {
    *a = (rho + k) % m;
    *b = (rho - k + m) % m;
  }
}

// One-sided (Hestenes) Jacobi on the q columns (length r, column a at
// B[a * r]) of B, accumulating the rotations in the q x q matrix X (column a at
// X[a * q]); round-robin pair schedule, one warp per pair, sweeps until no
// pair has |gamma| > tol sqrt(alpha beta) or `max_sweeps` is reached.
template <class T>
__device__ void jacobi_sweeps(T *B, T *X, int q, int r, T tol, int max_sweeps, int *rotated) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nw = kColThreads / 32;
  const int qq = q + (q & 1);
  if (tid == 0) *rotated = 0;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int rho = 0; rho < qq - 1; ++rho) {
      for (int pr = warp; pr < qq / 2; pr += nw) {
        int a, bb;
        jacobi_pair(rho, pr, qq, &a, &bb);
        if (a >= q || bb >= q) continue;
        if (a > bb) {
          const int tt = a;
          a = bb;
          bb = tt;
        }
        T al = 0, be = 0, ga = 0;
        for (int c = lane; c < r; c += 32) {
          const T x = B[a * r + c], y = B[bb * r + c];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != T(0) && fabs(ga) > tol * sqrt(al * be)) {
          const T zeta = (be - al) / (T(2) * ga);
          const T tn = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          const T cs = T(1) / sqrt(T(1) + tn * tn), sn = cs * tn;
          for (int c = lane; c < r; c += 32) {
            const T x = B[a * r + c], y = B[bb * r + c];
            B[a * r + c] = cs * x - sn * y;
            B[bb * r + c] = sn * x + cs * y;
          }
          for (int c = lane; c < q; c += 32) {
            const T x = X[a * q + c], y = X[bb * q + c];
            X[a * q + c] = cs * x - sn * y;
            X[bb * q + c] = sn * x + cs * y;
          }
          if (lane == 0) *rotated = 1;
        }
      }
      __syncthreads();
    }
    const int any = *rotated;
    __syncthreads();
    if (!any) break;
    if (tid == 0) *rotated = 0;
    __syncthreads();
  }
}

struct ColArgs {
  const double *S;
  double *U;
  int32_t *ranks;
  double *W;  // workspace, column-major m_i x r per box at offset off_i * r
  double *E;  // workspace, column-major m_i x k per box at offset off_i * k
  const int32_t *offsets;
  const int32_t *nnbr;
  int r, k, b;
};

__global__ void __launch_bounds__(kColThreads) col_kernel(ColArgs A) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nw = kColThreads / 32;
  const int i = blockIdx.x;
  const int off = A.offsets[i], m = A.offsets[i + 1] - off;
  const int r = A.r, k = A.k;
  const int ki = (A.nnbr[i] < A.b) ? min(k, m) : 0;
  if (tid == 0) A.ranks[i] = ki;
  double *U = A.U + (int64_t)off * k;
  if (ki == 0) {
    for (int idx = tid; idx < m * k; idx += kColThreads) U[idx] = 0.0;
    return;
  }
  const int q = min(m, r);
  double *W = A.W + (int64_t)off * r;
  double *E = A.E + (int64_t)off * k;
  double *tauh = sm;             // [kRMax]
  double *red = tauh + kRMax;    // [kColThreads / 32]
  double *B = red + kColThreads / 32;  // [q][r]: column a of R^T (= row a of R)
  double *X = B + q * r;         // [q][q]: column-major rotations
  double *sig = X + q * q;       // [q]
  int *order = reinterpret_cast<int *>(sig + q);  // [q]
  __shared__ int rotated;

  // Working copy of S_i, column-major.
  for (int idx = tid; idx < m * r; idx += kColThreads) {
    const int p = idx / r, c = idx % r;
    W[(int64_t)c * m + p] = A.S[((int64_t)off + p) * r + c];
  }
  __syncthreads();

  // Householder QR (§2.2), reflector j: H_j = I - tau_j v v^T, v_j = 1,
  // v below the diagonal stored in column j, beta on the diagonal.
  for (int j = 0; j < q; ++j) {
    double part = 0.0;
    for (int p = j + 1 + tid; p < m; p += kColThreads) {
      const double v = W[(int64_t)j * m + p];
      part += v * v;
    }
    const double sigma = block_sum(part, red);
    const double alpha = W[(int64_t)j * m + j];
    double t = 0.0, beta = alpha, scale = 0.0;
    if (sigma != 0.0) {
      beta = -copysign(sqrt(alpha * alpha + sigma), alpha);
      t = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    __syncthreads();
    for (int p = j + 1 + tid; p < m; p += kColThreads) W[(int64_t)j * m + p] *= scale;
    if (tid == 0) {
      W[(int64_t)j * m + j] = beta;
      tauh[j] = t;
    }
    __syncthreads();
    if (t != 0.0) {
      for (int c = j + 1 + warp; c < r; c += nw) {
        double d = lane == 0 ? W[(int64_t)c * m + j] : 0.0;
        for (int p = j + 1 + lane; p < m; p += 32) d += W[(int64_t)j * m + p] * W[(int64_t)c * m + p];
        const double wv = warp_sum(d) * t;
        if (lane == 0) W[(int64_t)c * m + j] -= wv;
        for (int p = j + 1 + lane; p < m; p += 32) W[(int64_t)c * m + p] -= wv * W[(int64_t)j * m + p];
      }
    }
    __syncthreads();
  }

  // SVD of R through one-sided Jacobi on B = R^T (column a of B = row a of
  // R): R^T X = B with orthogonal columns, so R = X diag(|B_a|) (B_a/|B_a|)^T
  // and the columns of X are R's left singular vectors.  GB300's FP64 pipe is
  // ~60x slower than FP32, so the sweeps first run in FP32 (in the same
  // shared memory), then B = R^T X is formed in FP64 from the FP32 rotations
  // and FP64 sweeps polish it from that nearly orthogonal start (quadratic
  // convergence: typically one rotating sweep and one that confirms).
  {
    float *Bf = reinterpret_cast<float *>(B);
    float *Xf = reinterpret_cast<float *>(X);
    for (int idx = tid; idx < q * r; idx += kColThreads) {
      const int a = idx / r, c = idx % r;
      Bf[idx] = (c >= a) ? (float)W[(int64_t)c * m + a] : 0.f;
    }
    for (int idx = tid; idx < q * q; idx += kColThreads) Xf[idx] = (idx / q == idx % q) ? 1.f : 0.f;
    __syncthreads();
    jacobi_sweeps<float>(Bf, Xf, q, r, 4.f * r * 1.1920929e-7f, 30, &rotated);
    // Widen X: park the FP32 rotations in the free upper half of B's space
    // (Bf uses the lower half; q <= r), then write them back as FP64.
    float *Xp = Bf + q * r;
    for (int idx = tid; idx < q * q; idx += kColThreads) Xp[idx] = Xf[idx];
    __syncthreads();
    for (int idx = tid; idx < q * q; idx += kColThreads) X[idx] = (double)Xp[idx];
    __syncthreads();
  }
  // The FP32 rotations are orthogonal to ~1e-6 only and rotations cannot fix
  // that, so re-orthonormalise X's columns in FP64 (classical Gram-Schmidt,
  // twice per column; the projections of a column use the Bf space as
  // scratch).
  {
    double *proj = reinterpret_cast<double *>(B);  // [q] coefficients
    for (int a = 0; a < q; ++a) {
      double *xa = X + a * q;
      for (int pass = 0; pass < 2; ++pass) {
        for (int bcol = warp; bcol < a; bcol += nw) {
          double d = 0.0;
          for (int c = lane; c < q; c += 32) d += X[bcol * q + c] * xa[c];
          d = warp_sum(d);
          if (lane == 0) proj[bcol] = d;
        }
        __syncthreads();
        for (int c = tid; c < q; c += kColThreads) {
          double v = xa[c];
          for (int bcol = 0; bcol < a; ++bcol) v -= proj[bcol] * X[bcol * q + c];
          xa[c] = v;
        }
        __syncthreads();
      }
      if (warp == 0) {
        double nn = 0.0;
        for (int c = lane; c < q; c += 32) nn += xa[c] * xa[c];
        nn = warp_sum(nn);
        if (lane == 0) proj[q] = 1.0 / sqrt(nn);
      }
      __syncthreads();
      for (int c = tid; c < q; c += kColThreads) xa[c] *= proj[q];
      __syncthreads();
    }
  }
  // B = R^T X in FP64 (R upper triangular: R(t, c) = W[c m + t], t <= c).
  for (int idx = tid; idx < q * r; idx += kColThreads) {
    const int a = idx / r, c = idx % r;
    const int tmax = min(c, q - 1);
    double acc = 0.0;
    for (int t = 0; t <= tmax; ++t) acc += W[(int64_t)c * m + t] * X[a * q + t];
    B[idx] = acc;
  }
  __syncthreads();
  jacobi_sweeps<double>(B, X, q, r, 4.0 * r * 2.220446049250313e-16, 12, &rotated);

  // Singular values and their descending order (ties: lower index first).
  for (int a = warp; a < q; a += nw) {
    double s2 = 0.0;
    for (int c = lane; c < r; c += 32) s2 += B[a * r + c] * B[a * r + c];
    s2 = warp_sum(s2);
    if (lane == 0) sig[a] = sqrt(s2);
  }
  __syncthreads();
  for (int a = tid; a < q; a += kColThreads) {
    int rank = 0;
    for (int c = 0; c < q; ++c) rank += (sig[c] > sig[a]) || (sig[c] == sig[a] && c < a);
    order[rank] = a;
  }
  __syncthreads();

  // E = Q [X(:, order[0:ki]); 0], Q = H_0 H_1 ... H_{q-1}.
  for (int idx = tid; idx < ki * m; idx += kColThreads) {
    const int tcol = idx / m, p = idx % m;
    E[(int64_t)tcol * m + p] = (p < q) ? X[order[tcol] * q + p] : 0.0;
  }
  __syncthreads();
  for (int j = q - 1; j >= 0; --j) {
    const double t = tauh[j];
    if (t != 0.0) {
      for (int tcol = warp; tcol < ki; tcol += nw) {
        double *e = E + (int64_t)tcol * m;
        double d = lane == 0 ? e[j] : 0.0;
        for (int p = j + 1 + lane; p < m; p += 32) d += W[(int64_t)j * m + p] * e[p];
        const double wv = warp_sum(d) * t;
        if (lane == 0) e[j] -= wv;
        for (int p = j + 1 + lane; p < m; p += 32) e[p] -= wv * W[(int64_t)j * m + p];
      }
    }
    __syncthreads();
  }

  // Sign rule, then write U_i (zero columns beyond k_i).
  for (int tcol = warp; tcol < k; tcol += nw) {
    double sgn = 1.0;
    if (tcol < ki) {
      const double *e = E + (int64_t)tcol * m;
      double best = -1.0;
      int bi = 0x7fffffff;
      for (int p = lane; p < m; p += 32) {
        const double v = fabs(e[p]);
        if (v > best) {
          best = v;
          bi = p;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      sgn = (e[bi] < 0.0) ? -1.0 : 1.0;
    }
    for (int p = lane; p < m; p += 32)
      U[(int64_t)p * k + tcol] = (tcol < ki) ? sgn * E[(int64_t)tcol * m + p] : 0.0;
  }
}

size_t col_smem(int r) {
  const int q = r;  // q <= r
  return sizeof(double) * (kRMax + kColThreads / 32 + (size_t)q * r + (size_t)q * q + q) +
         sizeof(int) * q;
}

}  // namespace
}  // namespace tblr

using namespace tblr;

extern "C" int tblr_decode(const tblr_problem *prob, const tblr_layout *lay, const double *T,
                           double *z, double *tau, double *rho, void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_TRY(check_layout(P, lay));
  TBLR_REQUIRE(T && z && tau && rho, "T, z, tau and rho must be non-NULL");
  TBLR_REQUIRE(P.ell <= 32, "tag decode supports ell <= 32 (got %d)", P.ell);
  decode_kernel<<<(unsigned)cdiv(P.b, kDecWarps), 32 * kDecWarps, 0, as_stream(stream)>>>(
      T, (int)P.b, P.ell, P.s3, lay->nbr, lay->nnbr, z, tau, rho);
  TBLR_TRY(launch_status("decode_kernel"));
  if (P.zrule != TBLR_Z_MINRATIO) return TBLR_OK;
  // §5.3: minimise the aspect ratio inside the projected vector's sign cell.
  const int max_iter = 16 * P.ell + 200;
  minratio_kernel<<<(unsigned)P.b, kLpThreads, 0, as_stream(stream)>>>(
      T, (int)P.b, P.ell, P.s3, lay->nbr, lay->nnbr, max_iter, z, tau, rho);
  return launch_status("minratio_kernel");
}

namespace tblr {
// tau[i*b + c] = 0 for c in N_i, 1 otherwise (Algorithm 3's far-field mask).
__global__ void far_indicator_kernel(const int32_t *__restrict__ nbr, const int32_t *__restrict__ nnbr,
                                     int b, int s3, double *__restrict__ tau) {
  const int64_t total = (int64_t)b * b;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / b), c = (int)(t % b);
    bool near = false;
    for (int s = 0; s < nnbr[i]; ++s) near = near || nbr[(int64_t)i * s3 + s] == c;
    tau[t] = near ? 0.0 : 1.0;
  }
}
}  // namespace tblr

extern "C" int tblr_far_indicator(const tblr_problem *prob, const tblr_layout *lay, double *tau,
                                  void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_TRY(check_layout(P, lay));
  TBLR_REQUIRE(tau != nullptr, "tau must be non-NULL");
  far_indicator_kernel<<<(unsigned)std::min<int64_t>(cdiv(P.b * P.b, 256), 4096), 256, 0,
                         as_stream(stream)>>>(lay->nbr, lay->nnbr, (int)P.b, P.s3, tau);
  return launch_status("far_indicator_kernel");
}

extern "C" int tblr_decode_lp_failures(unsigned int *count) {
  TBLR_REQUIRE(count != nullptr, "count is NULL");
  unsigned int zero = 0;
  TBLR_CUDA(cudaDeviceSynchronize());
  TBLR_CUDA(cudaMemcpyFromSymbol(count, tblr::g_lp_failures, sizeof(unsigned int)));
  TBLR_CUDA(cudaMemcpyToSymbol(tblr::g_lp_failures, &zero, sizeof(unsigned int)));
  return TBLR_OK;
}

extern "C" int tblr_combine(const tblr_problem *prob, const tblr_layout *lay, const double *yz,
                            const double *z, double *s, double *rr, void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_TRY(check_layout(P, lay));
  TBLR_REQUIRE(yz && z && s && rr, "yz, z, s and rr must be non-NULL");
  const int64_t total = P.n * P.r;
  const unsigned blocks = (unsigned)std::min<int64_t>(cdiv(total, 256), 152 * 16);
  combine_kernel<<<blocks, 256, 0, as_stream(stream)>>>(yz, z, lay->box_of, P.n, P.r, P.ell, P.C,
                                                        s, rr);
  return launch_status("combine_kernel");
}

extern "C" size_t tblr_col_workspace(const tblr_problem *prob) {
  Prob P;
  if (check_problem(prob, &P) != TBLR_OK) return 0;
  return align256(sizeof(double) * P.n * P.r) + align256(sizeof(double) * P.n * P.k);
}

extern "C" int tblr_col(const tblr_problem *prob, const tblr_layout *lay, const double *s,
                        double *u, int32_t *ranks, void *ws, size_t ws_bytes, void *stream) {
  Prob P;
  TBLR_TRY(check_problem(prob, &P));
  TBLR_TRY(check_layout(P, lay));
  TBLR_REQUIRE(s && u && ranks, "s, u and ranks must be non-NULL");
  TBLR_REQUIRE(P.r <= kRMax, "col supports r <= %d (got %d)", kRMax, P.r);
  TBLR_REQUIRE(ws != nullptr && ws_bytes >= tblr_col_workspace(prob), "col workspace too small");
  ColArgs A;
  A.S = s;
  A.U = u;
  A.ranks = ranks;
  A.W = static_cast<double *>(ws);
  A.E = reinterpret_cast<double *>(static_cast<char *>(ws) + align256(sizeof(double) * P.n * P.r));
  A.offsets = lay->offsets;
  A.nnbr = lay->nnbr;
  A.r = P.r;
  A.k = P.k;
  A.b = (int)P.b;
  const size_t smem = col_smem(P.r);
  TBLR_CUDA(cudaFuncSetAttribute(col_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  col_kernel<<<(unsigned)P.b, kColThreads, smem, as_stream(stream)>>>(A);
  return launch_status("col_kernel");
}
