// Instantiations of the pass kernels: double transforms, group 'a' (split for parallel compilation).
#include "gpe_passes.cuh"
namespace gpe {
cudaError_t launch_group_f64_a(Pass pass, const PassArgs& a, cudaStream_t st) {
  switch (pass) {
    case P_AX: return launch_role<1, P_AX>(a, st);
    case P_AMID: return launch_role<1, P_AMID>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace gpe
