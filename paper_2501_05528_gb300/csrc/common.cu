// Status strings, thread-local error messages and problem validation.
#include <stdarg.h>
#include <stdio.h>

#include "common.cuh"

namespace tblr {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int launch_status(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("launch of %s failed: %s", what, cudaGetErrorString(e));
    return TBLR_ECUDA;
  }
  return TBLR_OK;
}

int check_problem(const tblr_problem *in, Prob *P) {
  TBLR_REQUIRE(in != nullptr, "problem is NULL");
  TBLR_REQUIRE(in->d >= 1 && in->d <= 3, "d must be 1, 2 or 3 (got %d)", in->d);
  TBLR_REQUIRE(in->n >= 1 && in->n <= INT32_MAX, "n out of range (%lld)", (long long)in->n);
  TBLR_REQUIRE(in->k >= 1 && in->p >= 0 && in->e >= 0, "need k >= 1, p >= 0, e >= 0");
  TBLR_REQUIRE(in->kernel == TBLR_KERNEL_LAPLACE2D || in->kernel == TBLR_KERNEL_LAPLACE3D ||
                   in->kernel == TBLR_KERNEL_DENSE,
               "unknown kernel %d", in->kernel);
  TBLR_REQUIRE(in->kernel != TBLR_KERNEL_LAPLACE2D || in->d == 2, "laplace2d needs d = 2");
  TBLR_REQUIRE(in->kernel != TBLR_KERNEL_LAPLACE3D || in->d == 3, "laplace3d needs d = 3");
  TBLR_REQUIRE(in->precision == TBLR_FP64 || in->precision == TBLR_MIXED, "bad precision");
  TBLR_REQUIRE(in->nearfield == TBLR_NEARFIELD_PROBE || in->nearfield == TBLR_NEARFIELD_EXACT,
               "bad nearfield mode");
  TBLR_REQUIRE(in->sketch == TBLR_SKETCH_BLACKBOX || in->sketch == TBLR_SKETCH_TAGGED ||
                   in->sketch == (TBLR_SKETCH_TAGGED | TBLR_SKETCH_SELFADJOINT),
               "bad sketch mode %d (the self-adjoint flag needs the tag-factored sketch)",
               in->sketch);
  P->d = in->d;
  P->kernel = in->kernel;
  P->n = in->n;
  P->k = in->k;
  P->p = in->p;
  P->e = in->e;
  P->r = in->k + in->p;
  P->precision = in->precision;
  P->nearfield = in->nearfield;
  TBLR_REQUIRE(in->zrule == TBLR_Z_PROJECT || in->zrule == TBLR_Z_MINRATIO, "bad zrule %d",
               in->zrule);
  P->zrule = in->zrule;
  P->tagged = (in->sketch & TBLR_SKETCH_TAGGED) != 0;
  P->selfadjoint = (in->sketch & TBLR_SKETCH_SELFADJOINT) != 0;
  int s3 = 1;
  for (int a = 0; a < in->d; ++a) s3 *= 3;
  P->s3 = s3;
  P->ell = s3 + 1 + in->e;
  int64_t b = 1;
  for (int a = 0; a < 3; ++a) {
    P->grid[a] = in->grid[a];
    P->lo[a] = in->lo[a];
    P->hi[a] = in->hi[a];
    if (a < in->d) {
      TBLR_REQUIRE(in->grid[a] >= 1, "grid[%d] must be >= 1", a);
      TBLR_REQUIRE(in->hi[a] > in->lo[a], "hi[%d] must exceed lo[%d]", a, a);
      b *= in->grid[a];
    } else {
      TBLR_REQUIRE(in->grid[a] == 1, "grid[%d] must be 1 for d = %d", a, in->d);
    }
  }
  TBLR_REQUIRE(b <= 16384, "at most 16384 boxes (got %lld)", (long long)b);
  P->b = b;
  P->C = (int64_t)P->ell * P->r;
  return TBLR_OK;
}

int check_layout(const Prob &P, const tblr_layout *lay) {
  (void)P;
  TBLR_REQUIRE(lay != nullptr, "layout is NULL");
  TBLR_REQUIRE(lay->perm && lay->box_of && lay->offsets && lay->nbr && lay->nnbr && lay->colour &&
                   lay->pts,
               "every layout array must be non-NULL");
  return TBLR_OK;
}

}  // namespace tblr

extern "C" const char *tblr_status_string(int status) {
  switch (status) {
    case TBLR_OK: return "ok";
    case TBLR_EINVAL: return "invalid argument";
    case TBLR_ECUDA: return "CUDA error";
    case TBLR_EUNSUPPORTED: return "unsupported";
    case TBLR_EWORKSPACE: return "workspace or capacity too small";
    case TBLR_ETIMEOUT: return "device-side wait timed out";
  }
  return "unknown status";
}

extern "C" const char *tblr_last_error(void) { return tblr::g_err; }

extern "C" int tblr_sizes_of(const tblr_problem *prob, tblr_sizes *out) {
  tblr::Prob P;
  TBLR_TRY(tblr::check_problem(prob, &P));
  TBLR_REQUIRE(out != nullptr, "out is NULL");
  out->b = P.b;
  out->ell = P.ell;
  out->r = P.r;
  out->s3 = P.s3;
  out->reserved = 0;
  out->sketch_cols = 2 * P.C;
  return TBLR_OK;
}
