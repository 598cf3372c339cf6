// Column kernels for stored values of type bf16_t with x, g and the accumulator in float.
#include "pcdm_kernels.cuh"

namespace pcdm {
template struct Kernels<bf16_t, float>;
}  // namespace pcdm
