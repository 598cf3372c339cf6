// Column kernels for stored values of type double with x, g and the accumulator in double.
#include "pcdm_kernels.cuh"

namespace pcdm {
template struct Kernels<double, double>;
}  // namespace pcdm
