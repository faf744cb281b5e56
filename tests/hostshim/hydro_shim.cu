// Host build of the hydrostatic kernel's column sweep (hydro.cuh: hydro_shell), for a CPU test against
// the oracle: every shell of the grid in turn, cgs inputs as the kernel takes them.
#include "hydro.cuh"

extern "C" void host_hydro(int nr, int nt, const double* rf, const double* tf, const double* T, const double* rho_cur,
                           const double* shell_mass, double GM, double mu, double T_floor, double* rho_out) {
  for (int i = 0; i < nr; ++i) mcrt::hydro_shell(i, nt, rf, tf, T, rho_cur, shell_mass, GM, mu, T_floor, rho_out);
}

// the relaxed step of every shell (hydro.cuh: hydro_relax) applied to rho_h in place
extern "C" void host_hydro_relax(int nr, int nt, const double* rf, const double* tf, const double* rho_cur,
                                 const double* a, const double* shell_mass, double* rho_h) {
  for (int i = 0; i < nr; ++i) mcrt::hydro_relax(i, nt, rf, tf, rho_cur, a[i], shell_mass, rho_h);
}
