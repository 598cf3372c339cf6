// Column kernels for stored values of type float with x, g and the accumulator in float.
#include "pcdm_kernels.cuh"

namespace pcdm {
template struct Kernels<float, float>;
}  // namespace pcdm
