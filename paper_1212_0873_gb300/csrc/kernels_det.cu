// The deterministic two-kernel form (det_kernels.cuh) for the three precision pairs.
#include "det_kernels.cuh"

namespace pcdm {
template struct DetKernels<double, double>;
template struct DetKernels<float, float>;
template struct DetKernels<bf16_t, float>;
}  // namespace pcdm
