// Host build of the temperature kernel's per-cell solve (temperature.cuh: q_sum, cell_temperature) over
// the library's temperature-grid tables (tables.h), and the Rosseland mean the PDA kernels read
// (planck.cuh: rosseland), for CPU tests against the oracle.
#include <algorithm>
#include <vector>

#include "tables.h"
#include "temperature.cuh"

// T (K) with 4 pi sum_b kappa_b Bbar_b(T) = q for each of the n values q (erg s^-1 g^-1)
extern "C" void host_temperatures(int nlam, const double* lam_e, const double* kabs, const double* ksca,
                                  const double* g, double Tstar, int n, const double* q, double* T) {
  mcrt::DustArrays dust;
  mcrt::dust_arrays(nlam, lam_e, kabs, ksca, g, Tstar, dust);
  bool gray = true;
  for (int b = 1; b < nlam; ++b)
    if (kabs[b] != kabs[0] || ksca[b] != ksca[0] || g[b] != g[0]) gray = false;
  const int nT = 1024;
  const double Tmin = 1.0, Tmax = std::max(1e4, 2.0 * Tstar);
  mcrt::TGridTables tt;
  mcrt::build_T_tables(nlam, lam_e, kabs, dust.chip.data(), nT, Tmin, Tmax, tt);
  const double dlnT = std::log(Tmax / Tmin) / (nT - 2);
  for (int i = 0; i < n; ++i)
    T[i] = mcrt::cell_temperature(q[i], gray ? 1 : 0, kabs[0], nlam, lam_e, kabs, tt.lQ64.data(), tt.slQ64.data(), nT,
                                  Tmin, dlnT);
}

// Rosseland mean of chi' at each of the n temperatures (planck.cuh: rosseland, read by the PDA kernels)
extern "C" void host_rosseland(int nlam, const double* lam_e, const double* chip, int n, const double* T, double* out) {
  for (int i = 0; i < n; ++i) out[i] = mcrt::rosseland(lam_e, chip, nlam, T[i]);
}
