// transport_f32.cu -- FP32 production instantiations of the transport kernel: single disk (gray dust
// fixed at compile time, or not) and batches.
#include "internal.h"

namespace mcrt {

template <>
cudaError_t launch_transport<float>(const KParams<float>& P, bool trace, bool batch, bool gray, int grid, int block,
                                    cudaStream_t st) {
  if (trace) return cudaErrorInvalidValue;
  if (batch) transport_kernel<float, false, true, false><<<grid, block, 0, st>>>(P);
  else if (gray) transport_kernel<float, false, false, true><<<grid, block, 0, st>>>(P);
  else transport_kernel<float, false, false, false><<<grid, block, 0, st>>>(P);
  return cudaGetLastError();
}

template <>
cudaError_t launch_transport_tail<float>(const KParams<float>& P, bool trace, bool batch, bool gray, int sms,
                                         int warps_per_sm, cudaStream_t st) {
  if (trace) return cudaErrorInvalidValue;
  const int grid = sms * (warps_per_sm > 0 ? warps_per_sm : kTailBlocksPerSm);
  if (batch) transport_tail_kernel<float, false, false, true><<<grid, 32, 0, st>>>(P);
  else if (gray) transport_tail_kernel<float, false, true, false><<<grid, 32, 0, st>>>(P);
  else transport_tail_kernel<float, false, false, false><<<grid, 32, 0, st>>>(P);
  return cudaGetLastError();
}

template <>
int transport_blocks_per_sm<float>(bool trace, bool batch, bool gray, int block) {
  int n = 0;
  if (trace) return 0;
  if (batch) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transport_kernel<float, false, true, false>, block, 0);
  else if (gray) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transport_kernel<float, false, false, true>, block, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transport_kernel<float, false, false, false>, block, 0);
  return n;
}

}  // namespace mcrt
