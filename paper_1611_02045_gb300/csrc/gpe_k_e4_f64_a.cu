// Instantiations of the pass kernels with E = 4 values per thread: double-precision
// transforms, group 'a' (split for parallel compilation).
#include "gpe_passes.cuh"
namespace gpe {
cudaError_t launch_group_f64_a_e4(Pass pass, const PassArgs& a, cudaStream_t st) {
  switch (pass) {
    case P_AX: return launch_role<1, P_AX, 4>(a, st);
    case P_AMID: return launch_role<1, P_AMID, 4>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace gpe
