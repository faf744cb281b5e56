// hydro.cu -- vertical hydrostatic structure of the disk (Sect. 2.5, Eq. 20).
//
// dP/dz = -rho G M_star z / R^3 with P = k_B rho T / (mu m_u), at fixed surface density, with the
// temperatures of the last Monte Carlo (+ PDA) solution. Each radial shell of the (r, theta) grid is
// one column: at the cell centres z = r_c cos theta_c, R = r_c sin theta_c, and
//   d ln(rho c^2) / dz = -G M z / (R^3 c^2),   c^2 = k_B T / (mu m_u),
// is integrated with the trapezoid rule between consecutive cell centres from theta = 0 to pi, so
// rho_j is proportional to exp(Phi_j) / T_j; each shell keeps its dust mass, cells without dust stay
// without dust, and temperatures below T_floor (cells no packet heated) are raised to it.
// One thread per shell, FP64 (a shell is a sequential sweep of a few hundred cells).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "hydro.cuh"
#include "internal.h"

namespace mcrt {
namespace {

constexpr double kG = 6.67430e-8;  // cm^3 g^-1 s^-2

__global__ void k_hydro(int nr, int nt, const double* __restrict__ rf, const double* __restrict__ tf,
                        const double* __restrict__ T, const double* __restrict__ rho_cur,
                        const double* __restrict__ shell_mass, double GM, double mu, double T_floor,
                        const double* __restrict__ relax, double* __restrict__ rho_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  hydro_shell(i, nt, rf, tf, T, rho_cur, shell_mass, GM, mu, T_floor, rho_out);
  if (relax) hydro_relax(i, nt, rf, tf, rho_cur, relax[i], shell_mass, rho_out);
}

}  // namespace
}  // namespace mcrt

using namespace mcrt;

#define CK(call, what)                                    \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(d, e_, what); \
  } while (0)

extern "C" {

void mcrt_default_hydro_opts(mcrt_hydro_opts* o) {
  if (!o) return;
  o->M_star_g = 2.5 * 1.98892e33;
  o->mu = 2.3;
  o->T_floor_K = 10.0;
  o->which = MCRT_T_PDA;
  o->shell_mass_g = nullptr;
  o->relax = nullptr;
}

mcrt_status mcrt_hydrostatic_density(mcrt_disk* d, const mcrt_hydro_opts* o, double* rho_out) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!o || !rho_out) return set_error(d, MCRT_EINVAL, "NULL argument");
  if (!(o->M_star_g > 0 && std::isfinite(o->M_star_g)) || !(o->mu > 0 && std::isfinite(o->mu)) ||
      !(o->T_floor_K > 0 && std::isfinite(o->T_floor_K)))
    return set_error(d, MCRT_EINVAL, "M_star, mu and T_floor must be positive");
  if (o->which != MCRT_T_MC && o->which != MCRT_T_PDA) return set_error(d, MCRT_EINVAL, "which");
  if (!d->has_opacity) return set_error(d, MCRT_ESTATE, "mcrt_set_opacity must come first");
  if (o->which == MCRT_T_PDA && !d->have_pda) return set_error(d, MCRT_ESTATE, "no PDA solution");
  const int nr = d->nr, nt = d->nt;
  const size_t n = (size_t)nr * nt;
  std::vector<double> M(nr, 0.0);
  if (o->shell_mass_g) {
    for (int i = 0; i < nr; ++i) {
      if (!(o->shell_mass_g[i] >= 0 && std::isfinite(o->shell_mass_g[i])))
        return set_error(d, MCRT_EINVAL, "shell masses must be finite and >= 0");
      M[i] = o->shell_mass_g[i];
    }
  } else {
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j < nt; ++j) M[i] += d->mass[(size_t)i * nt + j];
  }
  if (o->relax)
    for (int i = 0; i < nr; ++i)
      if (!(o->relax[i] > 0.0 && o->relax[i] <= 2.0)) return set_error(d, MCRT_EINVAL, "relax must be in (0, 2]");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  if (!d->have_T) {
    mcrt_status s = compute_temperatures(d);
    if (s != MCRT_OK) return s;
  }
  DBuf rf, tf, Md, out, rl;
  if (o->relax) {
    CK(rl.alloc(nr * 8), "cudaMalloc");
    CK(cudaMemcpyAsync(rl.p, o->relax, nr * 8, cudaMemcpyHostToDevice, d->stream), "copy");
  }
  CK(rf.alloc((nr + 1) * 8), "cudaMalloc");
  CK(tf.alloc((nt + 1) * 8), "cudaMalloc");
  CK(Md.alloc(nr * 8), "cudaMalloc");
  CK(out.alloc(n * 8), "cudaMalloc");
  cudaStream_t st = d->stream;
  CK(cudaMemcpyAsync(rf.p, d->rf.data(), (nr + 1) * 8, cudaMemcpyHostToDevice, st), "copy");
  CK(cudaMemcpyAsync(tf.p, d->tf.data(), (nt + 1) * 8, cudaMemcpyHostToDevice, st), "copy");
  CK(cudaMemcpyAsync(Md.p, M.data(), nr * 8, cudaMemcpyHostToDevice, st), "copy");
  const double* T = (o->which == MCRT_T_PDA ? d->T_pda : d->T_mc).as<double>();
  k_hydro<<<(nr + 127) / 128, 128, 0, st>>>(nr, nt, rf.as<double>(), tf.as<double>(), T, d->rho_cgs_d.as<double>(),
                                            Md.as<double>(), kG * o->M_star_g, o->mu, o->T_floor_K,
                                            o->relax ? rl.as<double>() : nullptr, out.as<double>());
  d->launches++;
  CK(cudaGetLastError(), "hydrostatic kernel");
  CK(cudaMemcpyAsync(rho_out, out.p, n * 8, cudaMemcpyDeviceToHost, st), "copy");
  CK(cudaStreamSynchronize(st), "synchronize");
  return MCRT_OK;
}

}  // extern "C"
