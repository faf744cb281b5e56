// tables.h -- the arrays and tables the kernels read, built on the host: the grid geometry, the density
// arrays, the dust per wavelength bin and its tables on the temperature grid, the inverse MRW
// escape-time table, and the sampling table of a Mueller matrix. Host code, compiled for the host in the
// tests too.
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "planck.cuh"

namespace mcrt {

struct TGridTables {
  std::vector<float> lQk;    // nT: log Q(T_k), Q = 4 pi sum_b kappa_b Bbar_b(T) (erg/s/g); lQk[0] = -inf
  std::vector<float> cbw;    // nT * nlam: cumulative kappa_b Bbar_b(T_k) (row 0 zero): BW re-emission
  std::vector<float> cexit;  // nT * nlam: cumulative dBbar_b/dT / chi'_b: the MRW exit spectrum
  std::vector<float> chiRk;  // nT: Rosseland mean of chi' (Eq. 12-15 at the fixed point of Eq. 13)
  std::vector<float> kbark;  // nT: kappa_bar of Eq. 10 at the fixed point of Eq. 13
  std::vector<float> jw;     // nT * nlam: Eq. 10 weights of the J tally, dBbar_b/dT normalised
  std::vector<double> lQ64;  // nT: FP64 log Q (temperature guesses)
  std::vector<double> slQ64; // nT: d log Q / d log T
};

// Temperature grid T_0 = Tmin (standing for 0), T_k = Tmin (Tmax/Tmin)^((k-1)/(nT-2)) for k >= 1.
// The eta of Eq. 13 has the closed-form fixed point eta_b = a chi'_b dBbar_b/dT, so the averages of
// Eq. 10 and 12-15 are weighted by dBbar_b/dT: kappa_bar = sum kappa dB / sum dB and
// chi_R = sum dB / sum (dB / chi').
inline void build_T_tables(int nlam, const double* lam_e, const double* kabs, const double* chip, int nT, double Tmin,
                           double Tmax, TGridTables& t) {
  const double dlnT = std::log(Tmax / Tmin) / (nT - 2);
  t.lQk.assign(nT, 0.f);
  t.cbw.assign((size_t)nT * nlam, 0.f);
  t.cexit.assign((size_t)nT * nlam, 0.f);
  t.chiRk.assign(nT, 0.f);
  t.kbark.assign(nT, 0.f);
  t.jw.assign((size_t)nT * nlam, 0.f);
  t.lQ64.assign(nT, -INFINITY);
  t.slQ64.assign(nT, 4.0);
  std::vector<double> B(nlam), dB(nlam);
  t.lQk[0] = -INFINITY;
  for (int k = 0; k < nT; ++k) {
    const double T = (k == 0) ? Tmin : Tmin * std::exp((k - 1) * dlnT);
    planck_bins(lam_e, nlam, T, B.data(), dB.data());
    double q = 0, c1 = 0, c2 = 0, sdb = 0, sdbc = 0, skdb = 0;
    for (int b = 0; b < nlam; ++b) {
      q += kabs[b] * B[b];
      c1 += kabs[b] * B[b];
      c2 += dB[b] / chip[b];
      sdb += dB[b];
      sdbc += dB[b] / chip[b];
      skdb += kabs[b] * dB[b];
      if (k > 0) t.cbw[(size_t)k * nlam + b] = (float)c1;
      t.cexit[(size_t)k * nlam + b] = (float)c2;
    }
    if (k > 0) {
      t.lQk[k] = (float)std::log(4.0 * kPi * q);
      t.lQ64[k] = std::log(4.0 * kPi * q);
      t.slQ64[k] = q > 0 ? T * skdb / q : 4.0;
    }
    t.chiRk[k] = (float)(sdb / sdbc);
    t.kbark[k] = (float)(skdb / sdb);
    if (sdb > 0)
      for (int b = 0; b < nlam; ++b) t.jw[(size_t)k * nlam + b] = (float)(dB[b] / sdb);
  }
}

// Geometry of the grid in units of r_faces[0] (FP64; the FP32 copies are cast from these): radial faces
// and their squares, per polar face cos, sin, their squares and its kind (2 the axis, 0 the midplane
// plane, +1 / -1 a cone opening up / down).
struct GeomArrays {
  std::vector<double> rf, rf2, c2, s2, cf, sf;
  std::vector<signed char> fk;
};
inline void geometry_arrays(int nr, int nt, const double* rf_cm, const double* tf, GeomArrays& g) {
  const double l = rf_cm[0];
  g.rf.resize(nr + 1);
  g.rf2.resize(nr + 1);
  g.c2.resize(nt + 1);
  g.s2.resize(nt + 1);
  g.cf.resize(nt + 1);
  g.sf.resize(nt + 1);
  g.fk.resize(nt + 1);
  for (int i = 0; i <= nr; ++i) {
    g.rf[i] = rf_cm[i] / l;
    g.rf2[i] = g.rf[i] * g.rf[i];
  }
  for (int j = 0; j <= nt; ++j) {
    const double t = tf[j];
    g.cf[j] = std::cos(t);
    g.sf[j] = std::sin(t);
    g.c2[j] = g.cf[j] * g.cf[j];
    g.s2[j] = g.sf[j] * g.sf[j];
    if (j == 0 || j == nt) g.fk[j] = 2;
    else if (std::fabs(t - 0.5 * kPi) < 1e-12) g.fk[j] = 0;
    else g.fk[j] = t < 0.5 * kPi ? 1 : -1;
  }
}

// Density-dependent arrays: rho * l_unit (extinction per internal length unit per cm^2/g), the cell
// masses (g) and log(1 / m) (FP32, 0 for empty cells).
struct DensityArrays {
  std::vector<double> rhol, mass;
  std::vector<float> lqm;
};
inline void density_arrays(int nr, int nt, const double* rf_cm, const double* tf, const double* rho, DensityArrays& d) {
  const size_t ncell = (size_t)nr * nt;
  d.rhol.resize(ncell);
  d.mass.resize(ncell);
  d.lqm.resize(ncell);
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nt; ++j) {
      const size_t c = (size_t)i * nt + j;
      d.rhol[c] = rho[c] * rf_cm[0];
      const double r1 = rf_cm[i], r2 = rf_cm[i + 1];
      const double V = 2.0 * kPi / 3.0 * (r2 * r2 * r2 - r1 * r1 * r1) * (std::cos(tf[j]) - std::cos(tf[j + 1]));
      d.mass[c] = rho[c] * V;
      d.lqm[c] = d.mass[c] > 0 ? (float)(-std::log(d.mass[c])) : 0.f;
    }
}

// Dust per wavelength bin: extinction chi = kappa + sigma, albedo sigma / chi, chi' = kappa + (1 - g) sigma,
// and the cumulative stellar spectrum (unnormalised Bbar_b(T_star)).
struct DustArrays {
  std::vector<double> chi, alb, chip, star;
};
inline void dust_arrays(int nlam, const double* lam_e, const double* kabs, const double* ksca, const double* g,
                        double Tstar, DustArrays& o) {
  o.chi.resize(nlam);
  o.alb.resize(nlam);
  o.chip.resize(nlam);
  o.star.resize(nlam);
  for (int b = 0; b < nlam; ++b) {
    o.chi[b] = kabs[b] + ksca[b];
    o.alb[b] = ksca[b] / o.chi[b];
    o.chip[b] = kabs[b] + (1.0 - g[b]) * ksca[b];
  }
  std::vector<double> B(nlam);
  planck_bins(lam_e, nlam, Tstar, B.data(), nullptr);
  double acc = 0.0;
  for (int b = 0; b < nlam; ++b) {
    acc += B[b];
    o.star[b] = acc;
  }
}

// Geometric half-cell resistances of the PDA (Sect. 2.2.1; multiply by 1/D), per cell (cgs faces): from the
// cell's centre to its inner / outer radial face, (1/a - 1/b) / Omega over the radial half [a, b] of solid
// angle Omega, and to its lower / upper polar face, (ln tan(t2/2) - ln tan(t1/2)) / (2 pi (r2 - r1)) over
// the polar half [t1, t2] (infinite towards the axis); ell: the cell's smallest extent, min(dr, r_c dtheta).
struct HalfResistances {
  std::vector<double> hr_in, hr_out, ht_lo, ht_hi, ell;
};
inline void half_resistances(int nr, int nt, const double* rf, const double* tf, HalfResistances& h) {
  const size_t n = (size_t)nr * nt;
  h.hr_in.resize(n);
  h.hr_out.resize(n);
  h.ht_lo.resize(n);
  h.ht_hi.resize(n);
  h.ell.resize(n);
  for (int i = 0; i < nr; ++i) {
    const double r1 = rf[i], r2 = rf[i + 1], rc = 0.5 * (r1 + r2);
    for (int j = 0; j < nt; ++j) {
      const double t1 = tf[j], t2 = tf[j + 1], tc = 0.5 * (t1 + t2);
      const double om = 2.0 * kPi * (std::cos(t1) - std::cos(t2));
      const size_t c = (size_t)i * nt + j;
      h.hr_in[c] = (1.0 / r1 - 1.0 / rc) / om;
      h.hr_out[c] = (1.0 / rc - 1.0 / r2) / om;
      const double ltc = std::log(std::tan(0.5 * tc));
      h.ht_lo[c] = (t1 > 0 ? ltc - std::log(std::tan(0.5 * t1)) : INFINITY) / (2.0 * kPi * (r2 - r1));
      h.ht_hi[c] = (t2 < kPi ? std::log(std::tan(0.5 * t2)) - ltc : INFINITY) / (2.0 * kPi * (r2 - r1));
      h.ell[c] = std::min(r2 - r1, rc * (t2 - t1));
    }
  }
}

// MRW escape-time law (Eq. 7-8): P(x) = 2 sum (-1)^{n+1} exp(-n^2 pi^2 x), the probability that a walker
// started at the centre of a sphere is still inside at x = D c t / R0^2. For x < 0.1 the series is
// slow; there its Jacobi-theta transform 1 - P = (2 / sqrt(pi x)) sum_{n>=0} exp(-(n + 1/2)^2 / x)
// converges in a few terms.
inline double mrw_survival(double x) {
  if (x <= 0) return 1.0;
  if (x >= 0.1) {
    double s = 0.0;
    for (int n = 1; n < 64; ++n) {
      const double t = std::exp(-(double)n * n * kPi * kPi * x);
      s += (n & 1) ? t : -t;
      if (t < 1e-20) break;
    }
    return 2.0 * s;
  }
  double s = 0.0;
  for (int n = 0; n < 16; ++n) {
    const double a = n + 0.5;
    const double t = std::exp(-a * a / x);
    s += t;
    if (t < 1e-20 * s) break;
  }
  return 1.0 - 2.0 / std::sqrt(kPi * x) * s;
}

// x with P(x) = P0 by bisection in log x; complement: solve 1 - P(x) = Q0 instead (accurate when P0
// is close to 1)
inline double mrw_survival_inverse(double P0, bool complement, double Q0) {
  double lo = 1e-5, hi = 64.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = std::sqrt(lo * hi);
    const double v = mrw_survival(mid);
    const bool above = complement ? (1.0 - v < Q0) : (v > P0);  // still inside: move right
    if (above) lo = mid; else hi = mid;
    if (hi / lo - 1.0 < 1e-15) break;
  }
  return std::sqrt(lo * hi);
}

// The inverse tables read by the transport kernels: node i at u = exp(t0 + i dt), u from 2^-24 to 1/2;
// tab[i] = x with P(x) = u, tab[kMrwTab + i] = 1 / x with P(x) = 1 - u (the kernel interpolates linearly
// in log u and takes the second table for u > 1/2).
inline float mrw_table_t0() { return (float)(-24.0 * 0.69314718055994530942); }  // ln 2^-24
inline float mrw_table_dt() {
  return (float)((-0.69314718055994530942 + 24.0 * 0.69314718055994530942) / (kMrwTab - 1));
}
inline void build_mrw_table(float* tab) {
  const float t0 = mrw_table_t0(), dt = mrw_table_dt();
  for (int i = 0; i < kMrwTab; ++i) {
    const double t = (double)t0 + (double)i * (double)dt;
    const double u = std::exp(t);
    tab[i] = (float)mrw_survival_inverse(u, false, 0.0);                     // P(x) = u, u <= 1/2
    tab[kMrwTab + i] = (float)(1.0 / mrw_survival_inverse(1.0 - u, true, u));  // P(x) = 1-u
  }
}

// Sampling table of the scattering angle of a Mueller matrix (Sect. 2.3): the cumulative S11 sin(theta)
// on theta_k = k pi / (nmu - 1) by the trapezoid rule, normalised to 1 (the kernels interpolate S11
// linearly, so theta follows from a quadratic within an interval). False when S11 sin(theta) vanishes.
inline bool mueller_cdf(const double* S11, int nmu, double* c) {
  const double h = kPi / (nmu - 1);
  c[0] = 0.0;
  for (int k = 1; k < nmu; ++k)
    c[k] = c[k - 1] + 0.5 * h * (S11[k - 1] * std::sin((double)(k - 1) * h) + S11[k] * std::sin((double)k * h));
  if (!(c[nmu - 1] > 0)) return false;
  const double tot = c[nmu - 1];
  for (int k = 0; k < nmu; ++k) c[k] /= tot;
  return true;
}

}  // namespace mcrt
