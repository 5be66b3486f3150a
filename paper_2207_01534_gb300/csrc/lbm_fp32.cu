// FP32 populations, FP32 arithmetic.
#include "lbm_kernels.cuh"
#include "lbm_pipe.cuh"
#include "lbm_flow.cuh"
#include "lbm_ops.inl"

namespace lbm {
template struct Ops<float>;
}
