// dsmc_ops_f32.cu -- FP32 (padded cell bins, fused step) instantiation.
#include "dsmc_ops.cuh"

namespace dsmc {
template struct Ops<float>;
}  // namespace dsmc
