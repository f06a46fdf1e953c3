// Instantiations of the pass kernels with E = 4 values per thread: single-precision
// transforms, group 'h' (split for parallel compilation).
#include "gpe_passes.cuh"
namespace gpe {
cudaError_t launch_group_f32_h_e4(Pass pass, const PassArgs& a, cudaStream_t st) {
  switch (pass) {
    case P_HX: return launch_role<0, P_HX, 4>(a, st);
    case P_HMID: return launch_role<0, P_HMID, 4>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace gpe
