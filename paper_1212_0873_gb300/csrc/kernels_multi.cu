// One-block-per-problem kernels for the three precision pairs.
#include "multi_kernels.cuh"

namespace pcdm {
template struct MultiKernels<double, double>;
template struct MultiKernels<float, float>;
template struct MultiKernels<bf16_t, float>;
}  // namespace pcdm
