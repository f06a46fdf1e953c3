// Instantiations of the pass kernels with E = 4 values per thread: double-precision
// transforms, group 'c' (split for parallel compilation).
#include "gpe_passes.cuh"
namespace gpe {
cudaError_t launch_group_f64_c_e4(Pass pass, const PassArgs& a, cudaStream_t st) {
  switch (pass) {
    case P_C1: return launch_role<1, P_C1, 4>(a, st);
    case P_CFWD: return launch_role<1, P_CFWD, 4>(a, st);
    case P_CCORE: return launch_role<1, P_CCORE, 4>(a, st);
    case P_CINV: return launch_role<1, P_CINV, 4>(a, st);
    case P_C3: return launch_role<1, P_C3, 4>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace gpe
