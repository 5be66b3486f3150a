// Reverse pass for FP32 storage.
#include "lbm_adjoint.cuh"

namespace lbm {
template struct Adj<float>;
}
