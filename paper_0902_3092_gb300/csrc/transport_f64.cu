// transport_f64.cu -- FP64 debug instantiations of the transport kernel. Compiled without FMA
// contraction so that its arithmetic follows the FP64 CPU oracle operation by operation.
#include "internal.h"

namespace mcrt {

template <>
cudaError_t launch_transport<double>(const KParams<double>& P, bool trace, bool batch, int grid, int block,
                                     cudaStream_t st) {
  if (batch) return cudaErrorInvalidValue;
  if (trace) transport_kernel<double, true, false><<<grid, block, 0, st>>>(P);
  else transport_kernel<double, false, false><<<grid, block, 0, st>>>(P);
  return cudaGetLastError();
}

template <>
int transport_blocks_per_sm<double>(bool trace, bool batch, int block) {
  int n = 0;
  if (batch) return 0;
  if (trace) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transport_kernel<double, true, false>, block, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transport_kernel<double, false, false>, block, 0);
  return n;
}

}  // namespace mcrt
