// Host build of the library's temperature-grid dust tables (tables.h), for a CPU test against the oracle.
#include <cstring>

#include "tables.h"

extern "C" void tables_host(int nlam, const double* lam_e, const double* kabs, const double* chip, int nT, double Tmin,
                            double Tmax, float* lQk, float* cbw, float* cexit, float* chiR, float* kbar, float* jw,
                            double* lQ64, double* slQ64) {
  mcrt::TGridTables t;
  mcrt::build_T_tables(nlam, lam_e, kabs, chip, nT, Tmin, Tmax, t);
  const size_t m = (size_t)nT * nlam;
  std::memcpy(lQk, t.lQk.data(), nT * sizeof(float));
  std::memcpy(cbw, t.cbw.data(), m * sizeof(float));
  std::memcpy(cexit, t.cexit.data(), m * sizeof(float));
  std::memcpy(chiR, t.chiRk.data(), nT * sizeof(float));
  std::memcpy(kbar, t.kbark.data(), nT * sizeof(float));
  std::memcpy(jw, t.jw.data(), m * sizeof(float));
  std::memcpy(lQ64, t.lQ64.data(), nT * sizeof(double));
  std::memcpy(slQ64, t.slQ64.data(), nT * sizeof(double));
}

extern "C" int mrw_table_host(float* tab, float* t0, float* dt) {
  mcrt::build_mrw_table(tab);
  *t0 = mcrt::mrw_table_t0();
  *dt = mcrt::mrw_table_dt();
  return mcrt::kMrwTab;
}

// PDA half-cell resistances and cell extents (nr*nt each), as the PDA set-up builds them
extern "C" void half_resistances_host(int nr, int nt, const double* rf, const double* tf, double* hr_in, double* hr_out,
                                      double* ht_lo, double* ht_hi, double* ell) {
  mcrt::HalfResistances h;
  mcrt::half_resistances(nr, nt, rf, tf, h);
  const size_t n = (size_t)nr * nt * sizeof(double);
  std::memcpy(hr_in, h.hr_in.data(), n);
  std::memcpy(hr_out, h.hr_out.data(), n);
  std::memcpy(ht_lo, h.ht_lo.data(), n);
  std::memcpy(ht_hi, h.ht_hi.data(), n);
  std::memcpy(ell, h.ell.data(), n);
}
