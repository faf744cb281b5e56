// Host build of the transport kernels' cell geometry (common.cuh: next_face, dmin_cell, theta_cell, with
// the branch-free FP32 versions), for a CPU test against the oracle. Lengths in the grid's unit.
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

using namespace mcrt;

template <class R>
struct Grid {
  std::vector<R> rf, rf2, c2, s2, cf, sf;
  std::vector<signed char> fk;
  DevModel<R> M;
  Grid(int nr, int nt, const double* rfd, const double* tfd) {
    for (int i = 0; i <= nr; ++i) {
      rf.push_back((R)rfd[i]);
      rf2.push_back((R)(rfd[i] * rfd[i]));
    }
    for (int j = 0; j <= nt; ++j) {
      const double c = std::cos(tfd[j]), s = std::sin(tfd[j]);
      cf.push_back((R)c);
      sf.push_back((R)s);
      c2.push_back((R)(c * c));
      s2.push_back((R)(s * s));
      fk.push_back(j == 0 || j == nt ? 2 : (std::fabs(tfd[j] - 1.5707963267948966) < 1e-12 ? 0 : (tfd[j] < 1.5707963267948966 ? 1 : -1)));
    }
    std::memset(&M, 0, sizeof(M));
    M.nr = nr;
    M.nt = nt;
    M.rf = rf.data();
    M.rf2 = rf2.data();
    M.c2 = c2.data();
    M.s2 = s2.data();
    M.cf = cf.data();
    M.sf = sf.data();
    M.fk = fk.data();
  }
};

template <class R>
static double face_dist(int nr, int nt, const double* rf, const double* tf, int ir, int it, const double* p,
                        const double* u, int* face) {
  Grid<R> G(nr, nt, rf, tf);
  return (double)next_face(G.M, ir, it, (R)p[0], (R)p[1], (R)p[2], (R)u[0], (R)u[1], (R)u[2], *face);
}

template <class R>
static double dmin(int nr, int nt, const double* rf, const double* tf, int ir, int it, const double* p) {
  Grid<R> G(nr, nt, rf, tf);
  return (double)dmin_cell(G.M, ir, it, (R)p[0], (R)p[1], (R)p[2]);
}

extern "C" double next_face_f(int nr, int nt, const double* rf, const double* tf, int ir, int it, const double* p,
                              const double* u, int* face) {
  return face_dist<float>(nr, nt, rf, tf, ir, it, p, u, face);
}
extern "C" double next_face_d(int nr, int nt, const double* rf, const double* tf, int ir, int it, const double* p,
                              const double* u, int* face) {
  return face_dist<double>(nr, nt, rf, tf, ir, it, p, u, face);
}
extern "C" double dmin_f(int nr, int nt, const double* rf, const double* tf, int ir, int it, const double* p) {
  return dmin<float>(nr, nt, rf, tf, ir, it, p);
}
extern "C" double dmin_d(int nr, int nt, const double* rf, const double* tf, int ir, int it, const double* p) {
  return dmin<double>(nr, nt, rf, tf, ir, it, p);
}
extern "C" int theta_cell_f(int nr, int nt, const double* rf, const double* tf, const double* p) {
  Grid<float> G(nr, nt, rf, tf);
  return theta_cell(G.M, (float)p[0], (float)p[1], (float)p[2]);
}
