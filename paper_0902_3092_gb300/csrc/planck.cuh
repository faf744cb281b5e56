// planck.cuh -- Planck function integrated over wavelength bins, host and device (FP64).
//
// int_bin B_nu(T) dnu = (2 k^4 T^4 / (h^3 c^2)) [F3(x_hi) - F3(x_lo)],  F3(x) = int_0^x t^3/(e^t-1) dt,
// int_bin dB_nu/dT dnu = (2 k^4 T^3 / (h^3 c^2)) [F4(x_hi) - F4(x_lo)], F4(x) = int_0^x t^4 e^t/(e^t-1)^2 dt,
// with x = h nu / (k T). For x <= 2 the integrals are evaluated by 20-point Gauss-Legendre quadrature
// on [0, x] (the integrands are analytic there); above, from their complements
// int_x^inf t^3 e^{-nt} dt and int_x^inf t^4 n e^{-nt} dt summed over n (geometric expansion of
// 1/(e^t-1) and e^t/(e^t-1)^2). The first bin extends to lambda -> 0 and the last to infinity.
#pragma once
#include <cmath>

namespace mcrt {

constexpr double kH = 6.62607015e-27;
constexpr double kC = 2.99792458e10;
constexpr double kKB = 1.380649e-16;
// 2 pi^5 k^4 / (15 h^3 c^2)
#define MCRT_SIGMA (2.0 * 3.14159265358979323846 * 3.14159265358979323846 * 3.14159265358979323846 * \
                    3.14159265358979323846 * 3.14159265358979323846 * kKB * kKB * kKB * kKB /       \
                    (15.0 * kH * kH * kH * kC * kC))

// 20-point Gauss-Legendre nodes and weights on [-1, 1] (positive half; symmetric)
__host__ __device__ inline void gl20(int i, double& x, double& w) {
  const double X[10] = {0.0765265211334973337546, 0.2277858511416450780805, 0.3737060887154195606726,
                        0.5108670019508270980044, 0.6360536807265150254528, 0.7463319064601507926143,
                        0.8391169718222188233945, 0.9122344282513259058678, 0.9639719272779137912677,
                        0.9931285991850949247861};
  const double W[10] = {0.1527533871307258506981, 0.1491729864726037467878, 0.1420961093183820513293,
                        0.1316886384491766268985, 0.1181945319615184173124, 0.1019301198172404350368,
                        0.0832767415767047487248, 0.0626720483341090635695, 0.0406014298003869413310,
                        0.0176140071391521183119};
  x = X[i];
  w = W[i];
}

// F3, F4 on [0, x] for x <= 2 by quadrature; t^3/(e^t - 1) = t^3 / expm1(t)
__host__ __device__ inline void f34_small(double x, double& f3, double& f4) {
  f3 = 0.0;
  f4 = 0.0;
  const double h = 0.5 * x;
  for (int i = 0; i < 10; ++i) {
    double xi, wi;
    gl20(i, xi, wi);
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      const double t = h * (1.0 + sgn * xi);
      const double em = expm1(t);
      const double a = t * t * t / em;
      f3 += wi * a;
      f4 += wi * a * t * (em + 1.0) / em;
    }
  }
  f3 *= h;
  f4 *= h;
}

// complements G3 = int_x^inf, G4 = int_x^inf for x > 2
__host__ __device__ inline void g34_large(double x, double& g3, double& g4) {
  g3 = 0.0;
  g4 = 0.0;
  const double x2 = x * x, x3 = x2 * x, x4 = x3 * x;
  const double e1 = exp(-x);
  double e = e1;  // exp(-n x) as a running product: one exponential per call
  for (int n = 1; n < 200; ++n) {
    const double q = 1.0 / (double)n, q2 = q * q, q3 = q2 * q, q4 = q3 * q;
    const double t3 = e * (x3 * q + 3.0 * x2 * q2 + 6.0 * x * q3 + 6.0 * q4);
    const double t4 = e * (x4 + 4.0 * x3 * q + 12.0 * x2 * q2 + 24.0 * x * q3 + 24.0 * q4);
    g3 += t3;
    g4 += t4;
    if (t4 <= 1e-18 * g4 && t3 <= 1e-18 * g3) break;  // also ends at once where exp(-x) underflows to 0
    e *= e1;
  }
}

// Tail integrals from x to infinity, both kinds.
__host__ __device__ inline void tails(double x, double& g3, double& g4) {
  const double pi4 = 3.14159265358979323846 * 3.14159265358979323846 * 3.14159265358979323846 *
                     3.14159265358979323846;
  if (!(x > 0.0)) {
    g3 = pi4 / 15.0;
    g4 = 4.0 * pi4 / 15.0;
    return;
  }
  if (x > 2.0) {
    g34_large(x, g3, g4);
    return;
  }
  double f3, f4;
  f34_small(x, f3, f4);
  g3 = pi4 / 15.0 - f3;
  g4 = 4.0 * pi4 / 15.0 - f4;
}

// Bbar_b(T) and dBbar_b/dT for all bins; lam_e in micron (nlam+1 edges). Either output may be null.
__host__ __device__ inline void planck_bins(const double* lam_e, int nlam, double T, double* B, double* dB) {
  if (!(T > 0.0)) {
    for (int b = 0; b < nlam; ++b) {
      if (B) B[b] = 0.0;
      if (dB) dB[b] = 0.0;
    }
    return;
  }
  const double k4 = kKB * kKB * kKB * kKB;
  const double pref3 = 2.0 * k4 * T * T * T * T / (kH * kH * kH * kC * kC);
  const double pref4 = 2.0 * k4 * T * T * T / (kH * kH * kH * kC * kC);
  double g3p = 0.0, g4p = 0.0;  // tails at edge 0 (lambda -> 0, x -> inf)
  for (int b = 0; b < nlam; ++b) {
    double g3, g4;
    if (b + 1 == nlam) {
      tails(0.0, g3, g4);
    } else {
      const double x = kH * kC / (lam_e[b + 1] * 1e-4 * kKB * T);
      tails(x, g3, g4);
    }
    if (B) B[b] = pref3 * (g3 - g3p);
    if (dB) dB[b] = pref4 * (g4 - g4p);
    g3p = g3;
    g4p = g4;
  }
}

// Rosseland mean of chi' = kappa + (1-g) sigma at T (Eq. 3 with Eq. 16), exact bin integrals
__host__ __device__ inline double rosseland(const double* lam_e, const double* chip, int nlam, double T) {
  double g4p = 0.0, s1 = 0.0, s2 = 0.0;
  for (int b = 0; b < nlam; ++b) {
    double g3, g4;
    if (b + 1 == nlam) tails(0.0, g3, g4);
    else tails(kH * kC / (lam_e[b + 1] * 1e-4 * kKB * T), g3, g4);
    const double db = g4 - g4p;
    s1 += db;
    s2 += db / chip[b];
    g4p = g4;
  }
  return s1 / s2;
}

}  // namespace mcrt
