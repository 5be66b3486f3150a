// BF16 deviation storage of the moving populations, FP32 arithmetic.
#include "lbm_kernels.cuh"
#include "lbm_pipe.cuh"
#include "lbm_flow.cuh"
#include "lbm_ops.inl"

namespace lbm {
template struct Ops<__nv_bfloat16>;
}
