// Tensor-core coupling blocks Atilde_ij = U_i^T (A_ij V_j) for the
// mixed-precision path (three-part BF16 operands on tcgen05); see coupling_tc.cu.
#pragma once
#include "common.cuh"

namespace tblr {
size_t coupling_tc_workspace(const Prob &P);
// v = u in the self-adjoint mode.  Built-in Laplace kernels, 1 <= k <= 64.
int coupling_tc(const Prob &P, const tblr_layout *lay, const double *u, const double *v,
                const int32_t *ranks, double *at, void *ws, size_t ws_bytes, cudaStream_t s);
// Timed-out waits of the coupling kernel since the last call (then reset).
unsigned int coupling_tc_take_timeouts();
}  // namespace tblr
