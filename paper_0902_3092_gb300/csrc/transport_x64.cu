// transport_x64.cu -- FP64 transport with polarization or with the mean-intensity tally (compiled
// without FMA contraction, like the FP64 debug kernels, so that it follows the CPU oracle).
#include "transport_x.cuh"

namespace mcrt {
MCRT_TRANSPORT_X(double)
}  // namespace mcrt
