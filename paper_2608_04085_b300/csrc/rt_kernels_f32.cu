// rt_kernels_f32.cu -- FP32-state instantiation of the kernels (compiled with
// FMA contraction and fast approximate division / square root; reductions
// stay FP64).
#include "rt_launch_impl.cuh"

namespace rt {
RT_INSTANTIATE_LAUNCHERS(float)
}  // namespace rt
