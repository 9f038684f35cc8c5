// z pass of the transposed product in FP32.
#include "zmac.cuh"

namespace vc {
template int zmac_launch<float, true>(const Handle&, C_t<float>*, int, cudaStream_t, int, int);
}  // namespace vc
