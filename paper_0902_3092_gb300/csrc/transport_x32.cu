// transport_x32.cu -- FP32 transport with polarization or with the mean-intensity tally (compiled
// like the FP32 production kernels).
#include "transport_x.cuh"

namespace mcrt {
MCRT_TRANSPORT_X(float)
}  // namespace mcrt
