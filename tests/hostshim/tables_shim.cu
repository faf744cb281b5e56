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
