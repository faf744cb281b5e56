// transport_x.cuh -- launchers of the transport variants that keep extra tallies: polarization (the
// Mueller matrix of each scattering, Sect. 2.3) and the path-length estimator of the mean intensity
// (the scattering field of the observables). Single disk, no event trace; gray dust fixed at compile
// time or not. Each precision has its own translation unit, apart from the production kernels.
#pragma once
#include "internal.h"

namespace mcrt {

template <class R, bool POL, bool JT>
cudaError_t launch_x(const KParams<R>& P, bool gray, int grid, int block, cudaStream_t st) {
  if (gray) transport_kernel<R, false, false, true, POL, JT><<<grid, block, 0, st>>>(P);
  else transport_kernel<R, false, false, false, POL, JT><<<grid, block, 0, st>>>(P);
  return cudaGetLastError();
}

template <class R, bool POL, bool JT>
cudaError_t launch_tail_x(const KParams<R>& P, bool gray, int sms, int warps_per_sm, cudaStream_t st) {
  const int grid = sms * (warps_per_sm > 0 ? warps_per_sm : kTailBlocksPerSm);
  if (gray) transport_tail_kernel<R, false, true, false, POL, JT><<<grid, 32, 0, st>>>(P);
  else transport_tail_kernel<R, false, false, false, POL, JT><<<grid, 32, 0, st>>>(P);
  return cudaGetLastError();
}

template <class R, bool POL, bool JT>
int blocks_per_sm_x(bool gray, int block) {
  int n = 0;
  if (gray) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transport_kernel<R, false, false, true, POL, JT>, block, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transport_kernel<R, false, false, false, POL, JT>, block, 0);
  return n;
}

}  // namespace mcrt

// the six launchers of one precision R
#define MCRT_TRANSPORT_X(R)                                                                                  \
  template <>                                                                                                \
  cudaError_t launch_transport_pol<R>(const KParams<R>& P, bool gray, int grid, int block, cudaStream_t st) { \
    return launch_x<R, true, false>(P, gray, grid, block, st);                                               \
  }                                                                                                          \
  template <>                                                                                                \
  cudaError_t launch_transport_tail_pol<R>(const KParams<R>& P, bool gray, int sms, int wps, cudaStream_t st) { \
    return launch_tail_x<R, true, false>(P, gray, sms, wps, st);                                             \
  }                                                                                                          \
  template <>                                                                                                \
  int transport_blocks_per_sm_pol<R>(bool gray, int block) { return blocks_per_sm_x<R, true, false>(gray, block); } \
  template <>                                                                                                \
  cudaError_t launch_transport_j<R>(const KParams<R>& P, bool gray, int grid, int block, cudaStream_t st) {   \
    return launch_x<R, false, true>(P, gray, grid, block, st);                                               \
  }                                                                                                          \
  template <>                                                                                                \
  cudaError_t launch_transport_tail_j<R>(const KParams<R>& P, bool gray, int sms, int wps, cudaStream_t st) { \
    return launch_tail_x<R, false, true>(P, gray, sms, wps, st);                                             \
  }                                                                                                          \
  template <>                                                                                                \
  int transport_blocks_per_sm_j<R>(bool gray, int block) { return blocks_per_sm_x<R, false, true>(gray, block); }
