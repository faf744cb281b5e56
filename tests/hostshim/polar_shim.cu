// Host build of the polarization functions of the CUDA library (transport.cuh) and of its sampling
// table of the scattering angle (tables.h, as mcrt_set_mueller builds it), for a CPU test against the
// oracle: one scattering and the sky-frame Stokes of a packet, in FP32 and FP64.
#include <cmath>
#include <cstring>
#include <vector>

#include "tables.h"
#include "transport.cuh"

using namespace mcrt;

template <class R>
static void scatter(int nmu, const double* table, double* u, double* e, double* st, double w1, double w2) {
  std::vector<double> cdf((size_t)nmu);
  mueller_cdf(table, nmu, cdf.data());
  std::vector<R> t(4 * (size_t)nmu), c((size_t)nmu);
  for (size_t k = 0; k < t.size(); ++k) t[k] = (R)table[k];
  for (int k = 0; k < nmu; ++k) c[k] = (R)cdf[k];
  DevModel<R> M;
  std::memset(&M, 0, sizeof(M));
  M.mtab = t.data();
  M.mcdf = c.data();
  M.nmu = nmu;
  Pkt<R> s;
  std::memset(&s, 0, sizeof(s));
  s.lam = 0;
  s.ux = (R)u[0]; s.uy = (R)u[1]; s.uz = (R)u[2];
  s.ex = (R)e[0]; s.ey = (R)e[1]; s.ez = (R)e[2];
  s.sq = (R)st[0]; s.su = (R)st[1]; s.sv = (R)st[2];
  pol_scatter(M, s, (R)w1, (R)w2);
  u[0] = s.ux; u[1] = s.uy; u[2] = s.uz;
  e[0] = s.ex; e[1] = s.ey; e[2] = s.ez;
  st[0] = s.sq; st[1] = s.su; st[2] = s.sv;
}

template <class R>
static void observer(const double* u, const double* e, const double* st, double* q, double* uu) {
  Pkt<R> s;
  std::memset(&s, 0, sizeof(s));
  s.ux = (R)u[0]; s.uy = (R)u[1]; s.uz = (R)u[2];
  s.ex = (R)e[0]; s.ey = (R)e[1]; s.ez = (R)e[2];
  s.sq = (R)st[0]; s.su = (R)st[1]; s.sv = (R)st[2];
  R a, b;
  pol_observer(s, a, b);
  *q = a;
  *uu = b;
}

extern "C" void pol_scatter_f(int nmu, const double* t, double* u, double* e, double* st, double w1, double w2) {
  scatter<float>(nmu, t, u, e, st, w1, w2);
}
extern "C" void pol_scatter_d(int nmu, const double* t, double* u, double* e, double* st, double w1, double w2) {
  scatter<double>(nmu, t, u, e, st, w1, w2);
}
extern "C" void pol_observer_f(const double* u, const double* e, const double* st, double* q, double* uu) {
  observer<float>(u, e, st, q, uu);
}
extern "C" void pol_observer_d(const double* u, const double* e, const double* st, double* q, double* uu) {
  observer<double>(u, e, st, q, uu);
}
