// Host build of the ray tracer's source function and the mean-intensity read-out (source.cuh:
// k_source, k_mean_intensity, j_factor_of) over the library's own host builders (tables.h), for a CPU
// test against the oracle. The kernels' bodies run lane by lane (cuda_host_stubs.h).
#include <vector>

#include "cuda_host_stubs.h"
#include "tables.h"
#include "source.cuh"

using namespace mcrt;

// J (nr*nt*nlam) from path lengths jlen in internal units (l = r_faces[0]), as mcrt_mean_intensity reads it
extern "C" void host_mean_intensity(int nr, int nt, int nlam, const double* rf_cm, const double* tf,
                                    const double* jlen, double L_pkt, double n_total, double* J) {
  GeomArrays geo;
  geometry_arrays(nr, nt, rf_cm, tf, geo);
  host_blockIdx.x = host_threadIdx.x = 0;
  host_blockDim.x = host_gridDim.x = 1;
  k_mean_intensity(nr * nt, nt, nlam, geo.rf.data(), geo.cf.data(), jlen, j_factor_of(L_pkt, n_total, rf_cm[0], 1), J);
}

// S (nr*nt*nlam) as mcrt_raytrace builds it, FP32 (prec 32) or FP64; jlen NULL: no scattered light
extern "C" void host_source(int nr, int nt, int nlam, const double* rf_cm, const double* tf, const double* T,
                            const double* lam_e, const double* kabs, const double* ksca, const double* g, double Tstar,
                            const double* jlen, double L_pkt, double n_total, int prec, double* S) {
  GeomArrays geo;
  geometry_arrays(nr, nt, rf_cm, tf, geo);
  DustArrays dust;
  dust_arrays(nlam, lam_e, kabs, ksca, g, Tstar, dust);
  const int nc = nr * nt;
  const double f = j_factor_of(L_pkt, n_total, rf_cm[0], 1);
  std::vector<float> s32((size_t)nc * nlam);
  host_blockIdx.x = 0;
  host_blockDim.x = 32;  // one warp: lane t takes bins t, t + 32, ... of every cell
  host_gridDim.x = 1;
  for (unsigned t = 0; t < 32; ++t) {
    host_threadIdx.x = t;
    if (prec == 32)
      k_source<float>(nc, nlam, T, lam_e, kabs, dust.chi.data(), s32.data(), jlen, f, dust.alb.data(), geo.rf.data(),
                      geo.cf.data(), nt);
    else
      k_source<double>(nc, nlam, T, lam_e, kabs, dust.chi.data(), S, jlen, f, dust.alb.data(), geo.rf.data(),
                       geo.cf.data(), nt);
  }
  if (prec == 32)
    for (size_t k = 0; k < s32.size(); ++k) S[k] = s32[k];
}
