// z pass of the forward product in FP32.
#include "zmac.cuh"

namespace vc {
template int zmac_launch<float, false>(const Handle&, C_t<float>*, int, cudaStream_t, int, int);
}  // namespace vc
