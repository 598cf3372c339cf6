// Batched (several right-hand sides) kernels for stored values of type float with FP32 residuals.
#include "batch_kernels.cuh"

namespace pcdm {
template struct BatchKernels<float, float>;
}  // namespace pcdm
