// Instantiations of the pass kernels: double transforms, group 'h' (split for parallel compilation).
#include "gpe_passes.cuh"
namespace gpe {
cudaError_t launch_group_f64_h(Pass pass, const PassArgs& a, cudaStream_t st) {
  switch (pass) {
    case P_HX: return launch_role<1, P_HX>(a, st);
    case P_HMID: return launch_role<1, P_HMID>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace gpe
