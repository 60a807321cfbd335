// Pieces shared by the warp-specialised tcgen05 kernels (the mixed-precision
// apply and the tensor-core coupling): bounded mbarrier waits that turn a
// stalled pipeline into an error status instead of a hang, the three-way BF16
// split of operand values, and the TMA descriptor of a BF16 operand plane.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tc_utils.cuh"

namespace tblr {
namespace pipe {

constexpr long long kWaitBudget = 1000000000LL;  // clock cycles (~0.5 s) per wait
constexpr uint32_t kSleepNs = 200000;            // suspend hint of one try_wait (0.2 ms)

// Waits for phase `parity` of `bar`.  Gives up when another role of the CTA
// (S.abort) or another CTA of the launch (*status) has given up, or after
// kWaitBudget cycles; a timeout bumps *timeouts and raises both flags.
template <class SM>
__device__ __forceinline__ bool wait_or_abort(SM &S, volatile int *status, uint64_t *bar,
                                              uint32_t parity, unsigned int *timeouts) {
  if (tc::mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    // Suspended in the barrier rather than polling, so a waiting role takes
    // no issue slots from the warps that share its scheduler.
    if (tc::mbar_try_wait_sleep(bar, parity, kSleepNs)) return true;
    if (S.abort || *status) {
      S.abort = 1;
      return false;
    }
    if (clock64() - t0 > kWaitBudget) {
      atomicAdd(timeouts, 1u);
      *status = 1;
      S.abort = 1;
      return false;
    }
  }
}

// Warp-uniform bounded wait: lane 0 polls, every lane gets its verdict (so a
// warp never splits on a timeout), and the warp barrier orders the lanes'
// later accesses after the observed phase.
template <class SM>
__device__ __forceinline__ bool warp_wait(SM &S, volatile int *status, uint64_t *bar,
                                          uint32_t parity, unsigned int *timeouts) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = wait_or_abort(S, status, bar, parity, timeouts);
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok;
}
template <class SM>
__device__ __forceinline__ bool warp_aborted(SM &S) {
  return __shfl_sync(0xffffffffu, S.abort, 0) != 0;
}

// Drains a barrier whose copies may still be in flight before the CTA exits
// (bounded like every other wait).
__device__ __forceinline__ void drain(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!tc::mbar_try_wait_sleep(bar, parity, kSleepNs) && clock64() - t0 < kWaitBudget) {
  }
}

// Three-way BF16 split of two FP32 values, packed as K-adjacent pairs.  The
// remainders v - h and (v - h) - m are exact in FP32.
__device__ __forceinline__ void split3(float v0, float v1, uint32_t &h, uint32_t &m, uint32_t &l) {
  const __nv_bfloat162 bh = __floats2bfloat162_rn(v0, v1);
  const float2 fh = __bfloat1622float2(bh);
  const float r0 = v0 - fh.x, r1 = v1 - fh.y;
  const __nv_bfloat162 bm = __floats2bfloat162_rn(r0, r1);
  const float2 fm = __bfloat1622float2(bm);
  const __nv_bfloat162 bl = __floats2bfloat162_rn(r0 - fm.x, r1 - fm.y);
  h = *reinterpret_cast<const uint32_t *>(&bh);
  m = *reinterpret_cast<const uint32_t *>(&bm);
  l = *reinterpret_cast<const uint32_t *>(&bl);
}

// Three-way BF16 split of an FP64 value (remainders exact in FP64), so
// |x - h - m - l| <= 2^-24 |x|.
__device__ __forceinline__ void split3_fp64(double x, __nv_bfloat16 &h, __nv_bfloat16 &m,
                                            __nv_bfloat16 &l) {
  h = __double2bfloat16(x);
  const double r1 = x - (double)__bfloat162float(h);
  m = __double2bfloat16(r1);
  l = __double2bfloat16(r1 - (double)__bfloat162float(m));
}

inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// Tensor map of a BF16 plane [rows][npad] (npad contiguous, a multiple of 8):
// tiles of 64 points (128 bytes, 128-byte swizzle) x box_rows rows.
inline int make_plane_map(CUtensorMap *map, const __nv_bfloat16 *base, int64_t npad, int64_t rows,
                          int box_rows) {
  auto fn = encode_fn();
  TBLR_REQUIRE(fn != nullptr, "cuTensorMapEncodeTiled is unavailable");
  cuuint64_t dims[2] = {(cuuint64_t)npad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)npad * sizeof(__nv_bfloat16)};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base),
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return TBLR_ECUDA;
  }
  return TBLR_OK;
}

}  // namespace pipe
}  // namespace tblr
