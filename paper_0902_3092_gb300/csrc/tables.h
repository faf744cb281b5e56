// tables.h -- the dust tables on the temperature grid that the transport and temperature kernels read
// (built on the host when the opacities are set; host code, compiled for the host in the tests too).
#pragma once
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

}  // namespace mcrt
