// Host build of the Planck bin integrals of the CUDA library (planck.cuh), for a CPU test against the
// oracle.
#define __host__
#define __device__
#include <cmath>

#include "planck.cuh"

extern "C" void planck_bins_host(const double* lam_e, int nlam, double T, double* B, double* dB) {
  mcrt::planck_bins(lam_e, nlam, T, B, dB);
}
