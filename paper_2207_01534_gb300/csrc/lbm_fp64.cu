// FP64 populations, FP64 arithmetic.
#include "lbm_kernels.cuh"
#include "lbm_pipe.cuh"
#include "lbm_flow.cuh"
#include "lbm_ops.inl"

namespace lbm {
template struct Ops<double>;
}
