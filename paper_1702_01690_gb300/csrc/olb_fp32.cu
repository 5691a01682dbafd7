// olb_fp32.cu -- FP32 instances of the stage kernel (populations, fluxes and
// stencils in FP32; Kahan-compensated moment sums; T and Delta p recovered
// in FP64) and of the initialisation / output kernels.
#include "olb_fused.cuh"

namespace olb {
OLB_DEFINE_FUSED(float)
OLB_DEFINE_AUX_LAUNCHERS(float)
}  // namespace olb
