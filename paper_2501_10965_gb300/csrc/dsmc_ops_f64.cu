// dsmc_ops_f64.cu -- FP64-deterministic instantiation of the step kernels.
// Built with -fmad=false so that every FP64 expression rounds as written.
#include "dsmc_ops.cuh"

namespace dsmc {
template struct Ops<double>;
}  // namespace dsmc
