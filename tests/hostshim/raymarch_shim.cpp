// Host build of the ray march of the CUDA library (raymarch.cuh), for a CPU test against the oracle.
#include <vector>

#include "raymarch.cuh"
using namespace mcrt;
template <class R>
static int run(int nr, int nt, const R* rf2, const R* c2, const R* s2, const R* cf, const signed char* fk, R p, R q,
               R si, R ci, int maxn, int* cells, double* L, int cap) {
  std::vector<FaceCoef<R>> fc(nt + 1);
  for (int j = 0; j <= nt; ++j) fc[j] = face_coef<R>(c2[j], s2[j], fk[j], si, ci);
  RayGrid<R> G{nr, nt, rf2, cf, fc.data()};
  int m = 0;
  int rc = march_ray(G, p, q, si, ci, maxn, [&](int ir, int it, R l) {
    if (m < cap) { cells[m] = ir * nt + it; L[m] = (double)l; }
    ++m;
  });
  return rc < 0 ? -1 : m;
}
extern "C" int march_d(int nr, int nt, const double* rf2, const double* c2, const double* s2, const double* cf,
                       const signed char* fk, double p, double q, double si, double ci, int maxn, int* cells, double* L, int cap) {
  return run<double>(nr, nt, rf2, c2, s2, cf, fk, p, q, si, ci, maxn, cells, L, cap);
}
extern "C" int march_f(int nr, int nt, const float* rf2, const float* c2, const float* s2, const float* cf,
                       const signed char* fk, float p, float q, float si, float ci, int maxn, int* cells, double* L, int cap) {
  return run<float>(nr, nt, rf2, c2, s2, cf, fk, p, q, si, ci, maxn, cells, L, cap);
}
