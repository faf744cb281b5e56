// Host build of the wavelength sampling and the MRW escape-time lookup of the transport kernels
// (transport.cuh: qpos, sample_bw, sample_exit, sample_star, mrw_x) over the library's own tables
// (tables.h), for CPU tests against the oracle. One cell, log(1/m) = 0: log q = log(tally) + lq_run.
#include <cstring>
#include <vector>

#include "tables.h"
#include "transport.cuh"

using namespace mcrt;

namespace {
struct HostModel {
  TGridTables t;
  std::vector<float> lqm;
  std::vector<double> star;
  DevModel<double> M;
};
HostModel* H = nullptr;
}  // namespace

extern "C" void sampling_setup(int nlam, const double* lam_e, const double* kabs, const double* chip, int nT, double Tmin,
                               double Tmax, const double* star_cum, float lq_run) {
  delete H;
  H = new HostModel();
  build_T_tables(nlam, lam_e, kabs, chip, nT, Tmin, Tmax, H->t);
  H->lqm.assign(1, 0.f);
  H->star.assign(star_cum, star_cum + nlam);
  std::memset(&H->M, 0, sizeof(H->M));
  H->M.nlam = nlam;
  H->M.nT = nT;
  H->M.lQk = H->t.lQk.data();
  H->M.cbw = H->t.cbw.data();
  H->M.cexit = H->t.cexit.data();
  H->M.lqm = H->lqm.data();
  H->M.lq_run = lq_run;
  H->M.star_cum = H->star.data();
}

// re-emission bin after an absorption raised the cell's tally from t_old to t_new
extern "C" int bw_bin_host(unsigned long long t_old, unsigned long long t_new, float u) {
  int ko, kn;
  float wo, wn;
  qpos(H->M, t_old, 0, ko, wo);
  qpos(H->M, t_new, 0, kn, wn);
  return sample_bw(H->M, ko, wo, kn, wn, u);
}

// MRW exit bin at the cell's tally
extern "C" int exit_bin_host(unsigned long long tally, float u) {
  int k;
  float w;
  qpos(H->M, tally, 0, k, w);
  return sample_exit(H->M, k, w, u);
}

extern "C" int star_bin_host(double u) { return sample_star(H->M, u); }

// MRW escape time x with P(x) = u (Eq. 7-8) as the kernels look it up, FP32 (prec 32) or FP64
extern "C" double mrw_x_host(double u, int prec) {
  static std::vector<float> tab;
  if (tab.empty()) {
    tab.resize(2 * kMrwTab);
    build_mrw_table(tab.data());
  }
  if (prec == 32) {
    KParams<float> P;
    std::memset(&P, 0, sizeof(P));
    P.mrw_tab = tab.data();
    P.mrw_t0 = mrw_table_t0();
    P.mrw_dt = mrw_table_dt();
    return mrw_x(P, (float)u);
  }
  KParams<double> P;
  std::memset(&P, 0, sizeof(P));
  P.mrw_tab = tab.data();
  P.mrw_t0 = mrw_table_t0();
  P.mrw_dt = mrw_table_dt();
  return mrw_x(P, u);
}
