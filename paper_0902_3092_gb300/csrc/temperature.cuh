// temperature.cuh -- the radiative-equilibrium temperature of a cell (Sect. 2.1): the T that solves
// Q(T) = 4 pi sum_b kappa_b Bbar_b(T) = q, q the absorbed luminosity per unit mass, in FP64 on the exact
// bin integrals. Host and device code (the temperature kernel; compiled for the host in the tests too).
#pragma once
#include <cmath>

#include "common.cuh"
#include "planck.cuh"

namespace mcrt {

// Q(T) and dQ/dT (erg s^-1 g^-1 and per K) from the bin integrals of Bbar and of T dBbar/dT
__host__ __device__ inline void q_sum(const double* lam_e, const double* kabs, int nlam, double T, double& Q, double& dQ) {
  const double k4 = kKB * kKB * kKB * kKB;
  const double p3 = 2.0 * k4 * T * T * T * T / (kH * kH * kH * kC * kC);
  const double p4 = 2.0 * k4 * T * T * T / (kH * kH * kH * kC * kC);
  double g3p = 0.0, g4p = 0.0, s3 = 0.0, s4 = 0.0;
  for (int b = 0; b < nlam; ++b) {
    double g3, g4;
    if (b + 1 == nlam) tails(0.0, g3, g4);
    else tails(kH * kC / (lam_e[b + 1] * 1e-4 * kKB * T), g3, g4);
    s3 += kabs[b] * (g3 - g3p);
    s4 += kabs[b] * (g4 - g4p);
    g3p = g3;
    g4p = g4;
  }
  Q = 4.0 * kPi * p3 * s3;
  dQ = 4.0 * kPi * p4 * s4;
}

// T with Q(T) = q > 0: gray dust in closed form, otherwise bracketed Newton from a cubic Hermite guess on
// the tabulated grid (lQk: log Q(T_k), slQ: d log Q / d log T at T_k, T_k = Tmin exp((k-1) dlnT), k >= 1)
__host__ __device__ inline double cell_temperature(double q, int gray, double kabs0, int nlam, const double* lam_e,
                                                   const double* kabs, const double* lQk, const double* slQ, int nT,
                                                   double Tmin, double dlnT) {
  if (gray) {
    return pow(q / (4.0 * MCRT_SIGMA * kabs0), 0.25);
  }
  // initial guess from the log-spaced grid: log T as a cubic Hermite function of log Q between the two
  // grid temperatures that bracket q (slopes d log T / d log Q from the table; beyond the grid Q ~ T^4),
  // then bracketed Newton on the exact bin integrals (about two evaluations from this guess)
  const double lq = log(q);
  double Tk;
  if (lq < lQk[1]) {
    Tk = Tmin * exp(0.25 * (lq - lQk[1]));
  } else if (lq >= lQk[nT - 1]) {
    Tk = Tmin * exp((nT - 2) * dlnT) * exp(0.25 * (lq - lQk[nT - 1]));
  } else {
    int lo_k = 1, hi_k = nT - 1;  // lQk[lo_k] <= lq < lQk[hi_k]
    while (hi_k - lo_k > 1) {
      const int mid = (lo_k + hi_k) >> 1;
      if (lQk[mid] <= lq) lo_k = mid; else hi_k = mid;
    }
    const double x0 = lQk[lo_k], x1 = lQk[lo_k + 1], h = x1 - x0;
    const double y0 = (lo_k - 1) * dlnT, y1 = lo_k * dlnT;
    const double m0 = 1.0 / slQ[lo_k], m1 = 1.0 / slQ[lo_k + 1];
    double y = y0;
    if (h > 0) {
      const double t = (lq - x0) / h, t2 = t * t, t3 = t2 * t;
      y = (2 * t3 - 3 * t2 + 1) * y0 + (t3 - 2 * t2 + t) * h * m0 + (-2 * t3 + 3 * t2) * y1 + (t3 - t2) * h * m1;
    }
    Tk = Tmin * exp(y);
  }
  double lo = 0.0, hi = INFINITY;
  double x = Tk;
  for (int it = 0; it < 100; ++it) {
    double Q, dQ;
    q_sum(lam_e, kabs, nlam, x, Q, dQ);
    const double f = Q - q;
    if (f > 0) hi = x; else lo = x;
    double xn = x - f / dQ;
    // Q is smooth and increasing in T, so a Newton step of relative size s leaves a relative error of
    // order s^2: below 1e-8 the new point is the root to rounding (this also ends a guess that is the
    // root already, where f may be 0 and the step would not lie strictly inside the bracket)
    if (fabs(xn - x) <= 1e-8 * x) {
      x = xn;
      break;
    }
    if (!(xn > lo && xn < hi)) xn = isinf(hi) ? 2.0 * x : 0.5 * (lo + hi);
    if (fabs(xn - x) <= 1e-15 * x) {
      x = xn;
      break;
    }
    x = xn;
  }
  return x;
}

}  // namespace mcrt
