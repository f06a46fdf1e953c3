// Instantiations of the refinement-phase passes: double-single state (phi,
// H phi, r, V) and H phi transforms, FP32 direction fields (P_C workspace, p).
#include "gpe_passes.cuh"
namespace gpe {
cudaError_t launch_group_split(Pass pass, const PassArgs& a, cudaStream_t st) {
  switch (pass) {
    case P_HX: return launch_role<2, P_HX>(a, st);
    case P_HMID: return launch_role<2, P_HMID>(a, st);
    case P_C1: return launch_role<2, P_C1>(a, st);
    case P_C3: return launch_role<2, P_C3>(a, st);
    case P_AX: return launch_role<2, P_AX>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace gpe
