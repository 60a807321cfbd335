// Mixed-precision apply: not yet available in this build.
#include "mixed.cuh"

namespace tblr {
size_t mixed_workspace(const Prob &, int64_t) { return 0; }
int apply_mixed(const Prob &, const tblr_layout *, const double *, int64_t, double *, int64_t,
                void *, size_t, cudaStream_t) {
  set_error("mixed precision apply is not built");
  return TBLR_EUNSUPPORTED;
}
}  // namespace tblr
