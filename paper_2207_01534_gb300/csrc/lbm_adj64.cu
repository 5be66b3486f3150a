// Reverse pass for FP64 storage.
#include "lbm_adjoint.cuh"

namespace lbm {
template struct Adj<double>;
}
