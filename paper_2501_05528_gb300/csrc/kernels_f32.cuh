// FP32 kernel-matrix entries from double-float coordinates, shared by the
// mixed-precision kernels.  A coordinate x is carried as hi = fl32(x) and
// lo = fl32(x - hi), so differences (hi_p - hi_q) + (lo_p - lo_q) keep ~48
// bits: the hi difference is exact for close points (Sterbenz) and the lo
// parts restore the rest for far ones.  Entry error is ~2^-23 relative.
#pragma once
#include "common.cuh"

namespace tblr {

// The MUFU approximations (rsqrt.approx, lg2.approx: ~2^-22 relative) with
// subnormal inputs flushed to zero.  Squared distances of distinct points are
// never subnormal, and the flushing forms skip the input range scaling that
// the plain forms carry.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_ftz(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int KERNEL>
__device__ __forceinline__ float entry_f32(const float (&ph)[3], const float (&pl)[3],
                                           const float (&qh)[3], const float (&ql)[3]) {
  if (KERNEL == TBLR_KERNEL_LAPLACE2D) {
    const float dx = (ph[0] - qh[0]) + (pl[0] - ql[0]);
    const float dy = (ph[1] - qh[1]) + (pl[1] - ql[1]);
    const float r2 = fmaf(dx, dx, dy * dy);
    return 0.34657359027997264f * lg2_ftz(r2);  // 0.5 ln(2) log2(r^2) = log r
  } else {
    const float dx = (ph[0] - qh[0]) + (pl[0] - ql[0]);
    const float dy = (ph[1] - qh[1]) + (pl[1] - ql[1]);
    const float dz = (ph[2] - qh[2]) + (pl[2] - ql[2]);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    return 0.07957747154594767f * rsqrt_ftz(r2);  // 1 / (4 pi r)
  }
}

// The same entry without its constant factor: log2(r^2) in 2-D (times
// 0.5 ln 2 gives log r), 1/r in 3-D (times 1/(4 pi)).  Callers fold the factor
// into one multiplier per row.
template <int KERNEL>
__device__ __forceinline__ float entry_f32_raw(const float (&ph)[3], const float (&pl)[3],
                                               const float (&qh)[3], const float (&ql)[3]) {
  if (KERNEL == TBLR_KERNEL_LAPLACE2D) {
    const float dx = (ph[0] - qh[0]) + (pl[0] - ql[0]);
    const float dy = (ph[1] - qh[1]) + (pl[1] - ql[1]);
    return lg2_ftz(fmaf(dx, dx, dy * dy));
  } else {
    const float dx = (ph[0] - qh[0]) + (pl[0] - ql[0]);
    const float dy = (ph[1] - qh[1]) + (pl[1] - ql[1]);
    const float dz = (ph[2] - qh[2]) + (pl[2] - ql[2]);
    return rsqrt_ftz(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
  }
}
// The raw entry from the squared distance r2 (FP32).
template <int KERNEL>
__device__ __forceinline__ float entry_f32_of_r2(float r2) {
  return KERNEL == TBLR_KERNEL_LAPLACE2D ? lg2_ftz(r2) : rsqrt_ftz(r2);
}
template <int KERNEL>
__host__ __device__ constexpr float entry_f32_factor() {
  return KERNEL == TBLR_KERNEL_LAPLACE2D ? 0.34657359027997264f : 0.07957747154594767f;
}

// Split one FP64 coordinate into its double-float pair.
__device__ __forceinline__ void split_coord(double x, float &hi, float &lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// Kahan-compensated accumulation: sum ~ hi - c.
__device__ __forceinline__ void kahan_add(float &hi, float &c, float v) {
  const float y = v - c;
  const float t = hi + y;
  c = (t - hi) - y;
  hi = t;
}

// The same on 2 x 16 values in packed FP32x2 arithmetic (a - b is the exactly
// rounded fma(b, -1, a)), so every result is bitwise the scalar one.
__device__ __forceinline__ void kahan_add16(float (&hi)[16], float (&c)[16], const float (&v)[16]) {
  const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
  for (int e = 0; e < 16; e += 2) {
    const float2 h2 = make_float2(hi[e], hi[e + 1]), c2 = make_float2(c[e], c[e + 1]);
    const float2 y = __ffma2_rn(c2, m1, make_float2(v[e], v[e + 1]));  // v - c
    const float2 t = __fadd2_rn(h2, y);                                 // hi + y
    const float2 cn = __ffma2_rn(y, m1, __ffma2_rn(h2, m1, t));         // (t - hi) - y
    hi[e] = t.x;
    hi[e + 1] = t.y;
    c[e] = cn.x;
    c[e + 1] = cn.y;
  }
}

}  // namespace tblr
