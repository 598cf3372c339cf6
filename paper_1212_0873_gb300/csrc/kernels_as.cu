// Active-set coordinate-descent kernels (derivatives and the polish of x) for
// the three precision pairs.
#include "active_set_kernels.cuh"

namespace pcdm {
template struct ActiveSetKernels<double, double>;
template struct ActiveSetKernels<float, float>;
template struct ActiveSetKernels<bf16_t, float>;
}  // namespace pcdm
