// source.cuh -- the source function of the ray-traced observables and the mean intensity of the
// path-length tally (Sect. 2.3): per cell and wavelength bin, thermal emission kappa_b Bbar_b(T) / chi_b
// plus the scattered light (sigma_b / chi_b) J_b. Included by raytrace.cu; compiled for the host in the
// tests too.
#pragma once
#include "common.cuh"
#include "planck.cuh"

namespace mcrt {

// E_pkt / (4 pi l^2): turns a path length per cell volume, both in internal units (l = r_faces[0] cm),
// into the mean intensity; 0 before any packet ran
__host__ __device__ inline double j_factor_of(double L_pkt, double n_total, double l_unit,
                                              unsigned long long packets_done) {
  if (!packets_done || !(n_total > 0)) return 0.0;
  return L_pkt / n_total / (4.0 * kPi * l_unit * l_unit);
}

// Volume of cell c (internal units): (2 pi / 3) (r1^3 - r0^3) (cos theta0 - cos theta1).
__host__ __device__ inline double cell_volume(const double* rf, const double* cf, int nt, int c) {
  const int i = c / nt, j = c - i * nt;
  const double r0 = rf[i], r1 = rf[i + 1];
  return (2.0 * kPi / 3.0) * (r1 * r1 * r1 - r0 * r0 * r0) * (cf[j] - cf[j + 1]);
}

// The mean intensity of the path-length estimator, J[c][b] = jfac jlen[c][b] / V_c with
// jfac = E_pkt / (4 pi l^2) (erg s^-1 cm^-2 sr^-1, integrated over the bin; jlen and V in internal units).
static __global__ void k_mean_intensity(int nc, int nt, int nlam, const double* __restrict__ rf, const double* __restrict__ cf,
                                 const double* __restrict__ jlen, double jfac, double* __restrict__ J) {
  const size_t n = (size_t)nc * nlam;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(k / nlam);
    J[k] = jfac * jlen[k] / cell_volume(rf, cf, nt, c);
  }
}

// Source function per cell and bin: S[c][b] = kappa_b Bbar_b(T_c) / chi_b (FP64 bin integrals), plus
// the scattered light (sigma_b / chi_b) J_b of the mean-intensity tally when jlen is given (isotropic
// scattering); one warp per cell, lanes over bins.
template <class R>
__global__ void k_source(int nc, int nlam, const double* __restrict__ T, const double* __restrict__ lam_e,
                         const double* __restrict__ kabs, const double* __restrict__ chi, R* __restrict__ S,
                         const double* __restrict__ jlen, double jfac, const double* __restrict__ alb,
                         const double* __restrict__ rf, const double* __restrict__ cf, int nt) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const double k4 = kKB * kKB * kKB * kKB;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nc; c += nw) {
    const double t = T[c];
    const double pref3 = 2.0 * k4 * t * t * t * t / (kH * kH * kH * kC * kC);
    for (int b = lane; b < nlam; b += 32) {
      double v = 0.0;
      if (t > 0.0) {
        // bin b spans lam_e[b] .. lam_e[b+1]; G3 at the short edge is 0 for the first bin (lambda -> 0),
        // at the long edge G3(0) for the last one (lambda -> infinity)
        double g_short = 0.0, g_long, g4;
        if (b > 0) tails(kH * kC / (lam_e[b] * 1e-4 * kKB * t), g_short, g4);
        if (b + 1 == nlam) tails(0.0, g_long, g4);
        else tails(kH * kC / (lam_e[b + 1] * 1e-4 * kKB * t), g_long, g4);
        v = pref3 * (g_long - g_short) * kabs[b] / chi[b];
      }
      if (jlen) v += alb[b] * (jfac * jlen[(size_t)c * nlam + b] / cell_volume(rf, cf, nt, c));
      S[(size_t)c * nlam + b] = (R)v;
    }
  }
}

}  // namespace mcrt
