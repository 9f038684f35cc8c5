// z pass of the transposed product in FP64.
#include "zmac.cuh"

namespace vc {
template int zmac_launch<double, true>(const Handle&, C_t<double>*, int, cudaStream_t, int, int);
}  // namespace vc
