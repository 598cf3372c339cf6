// Batched (several right-hand sides) kernels for stored values of type double with FP64 residuals.
#include "batch_kernels.cuh"

namespace pcdm {
template struct BatchKernels<double, double>;
}  // namespace pcdm
