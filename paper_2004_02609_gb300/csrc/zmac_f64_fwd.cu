// z pass of the forward product in FP64.
#include "zmac.cuh"

namespace vc {
template int zmac_launch<double, false>(const Handle&, C_t<double>*, int, cudaStream_t, int, int);
}  // namespace vc
