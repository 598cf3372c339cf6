// Batched (several right-hand sides) kernels for stored values of type bf16_t with FP32 residuals.
#include "batch_kernels.cuh"

namespace pcdm {
template struct BatchKernels<bf16_t, float>;
}  // namespace pcdm
