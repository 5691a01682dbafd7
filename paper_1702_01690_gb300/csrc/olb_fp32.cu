// olb_fp32.cu -- FP32 instantiation of the stage kernels (populations, fluxes
// and stencils in FP32; Kahan-compensated moment sums; T and Delta p in FP64).
#include "olb_kernels.cuh"

namespace olb {
OLB_DEFINE_LAUNCHERS(float, 32, 8)
}  // namespace olb
