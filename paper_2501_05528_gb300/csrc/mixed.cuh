// Mixed-precision black-box apply (three-part BF16 operands on tcgen05 tensor cores,
// FP32 accumulation in TMEM); see mixed.cu.
#pragma once
#include "common.cuh"

namespace tblr {
size_t mixed_workspace(const Prob &P, int64_t ncols);
int apply_mixed(const Prob &P, const tblr_layout *lay, const double *xt, int64_t ncols, double *y,
                int64_t ldy, void *ws, size_t ws_bytes, cudaStream_t s);
size_t tagged_mixed_workspace(const Prob &P);
int tagged_sketch_mixed(const Prob &P, const tblr_layout *lay, const double *tau, const double *G,
                        const double *H, double *S, double *R, void *ws, size_t ws_bytes,
                        cudaStream_t s);
int apply_any(const Prob &P, const tblr_layout *lay, const double *dense, const double *xt,
              int64_t ncols, double *y, int64_t ldy, int adjoint, int precision, void *ws,
              size_t ws_bytes, cudaStream_t s);
}  // namespace tblr
