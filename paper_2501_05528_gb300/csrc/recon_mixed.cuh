// Mixed-precision (FP32 pipe) steps II and III; see recon_mixed.cu.
#pragma once
#include <algorithm>

#include "common.cuh"

namespace tblr {
size_t coupling_mixed_workspace(const Prob &P);
int coupling_mixed(const Prob &P, const tblr_layout *lay, const double *u, const double *v,
                   const int32_t *ranks, double *at, int mmax, void *ws, cudaStream_t s);
size_t nearfield_mixed_workspace(const Prob &P, int mmax);
int nearfield_mixed(const Prob &P, const tblr_layout *lay, const double *u, const double *at,
                    const double *v, const int64_t *nf_off, int mmax, double *bnear, void *ws,
                    cudaStream_t s);
}  // namespace tblr
