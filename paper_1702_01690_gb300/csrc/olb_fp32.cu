// olb_fp32.cu -- FP32 instances of the stage kernel (FP32 arithmetic on
// populations stored as hi + lo pairs of floats; moments, T and Delta p in
// double-float arithmetic) and of the initialisation / output kernels.
#include "olb_fused.cuh"

namespace olb {
OLB_DEFINE_FUSED(float)
OLB_DEFINE_AUX_LAUNCHERS(float)
}  // namespace olb
