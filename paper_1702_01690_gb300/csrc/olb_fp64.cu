// olb_fp64.cu -- FP64 instances of the stage kernel (all tile shapes) and of
// the initialisation / output kernels.
#include "olb_fused.cuh"

namespace olb {
OLB_DEFINE_FUSED(double)
OLB_DEFINE_AUX_LAUNCHERS(double)
}  // namespace olb
