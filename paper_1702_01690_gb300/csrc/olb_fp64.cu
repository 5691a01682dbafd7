// olb_fp64.cu -- FP64 instantiation of the stage kernels (32 x 8 node tiles).
#include "olb_kernels.cuh"

namespace olb {
OLB_DEFINE_LAUNCHERS(double, 32, 8)
}  // namespace olb
