// Instantiations of the refinement-phase passes (double-single state and H phi
// transforms, FP32 direction) with E = 4 values per thread.
#include "gpe_passes.cuh"
namespace gpe {
cudaError_t launch_group_split_e4(Pass pass, const PassArgs& a, cudaStream_t st) {
  switch (pass) {
    case P_HX: return launch_role<2, P_HX, 4>(a, st);
    case P_HMID: return launch_role<2, P_HMID, 4>(a, st);
    case P_C1: return launch_role<2, P_C1, 4>(a, st);
    case P_C3: return launch_role<2, P_C3, 4>(a, st);
    case P_AX: return launch_role<2, P_AX, 4>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace gpe
