// transport_f64.cu -- FP64 debug instantiations of the transport kernel. Compiled without FMA
// contraction so that its arithmetic follows the FP64 CPU oracle operation by operation.
#include "internal.h"

namespace mcrt {

template <>
cudaError_t launch_transport<double>(const KParams<double>& P, bool trace, bool batch, bool gray, int grid, int block,
                                     cudaStream_t st) {
  if (batch) return cudaErrorInvalidValue;
  if (trace) {
    if (gray) transport_kernel<double, true, false, true><<<grid, block, 0, st>>>(P);
    else transport_kernel<double, true, false, false><<<grid, block, 0, st>>>(P);
  } else {
    if (gray) transport_kernel<double, false, false, true><<<grid, block, 0, st>>>(P);
    else transport_kernel<double, false, false, false><<<grid, block, 0, st>>>(P);
  }
  return cudaGetLastError();
}

template <>
cudaError_t launch_transport_tail<double>(const KParams<double>& P, bool trace, bool batch, bool gray, int sms,
                                          int warps_per_sm, cudaStream_t st) {
  if (batch) return cudaErrorInvalidValue;
  const int grid = sms * (warps_per_sm > 0 ? warps_per_sm : kTailBlocksPerSm);
  if (trace) {
    if (gray) transport_tail_kernel<double, true, true, false><<<grid, 32, 0, st>>>(P);
    else transport_tail_kernel<double, true, false, false><<<grid, 32, 0, st>>>(P);
  } else {
    if (gray) transport_tail_kernel<double, false, true, false><<<grid, 32, 0, st>>>(P);
    else transport_tail_kernel<double, false, false, false><<<grid, 32, 0, st>>>(P);
  }
  return cudaGetLastError();
}

template <>
int transport_blocks_per_sm<double>(bool trace, bool batch, bool gray, int block) {
  int n = 0;
  if (batch) return 0;
  if (trace) {
    if (gray) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transport_kernel<double, true, false, true>, block, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transport_kernel<double, true, false, false>, block, 0);
  } else {
    if (gray) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transport_kernel<double, false, false, true>, block, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transport_kernel<double, false, false, false>, block, 0);
  }
  return n;
}

}  // namespace mcrt
