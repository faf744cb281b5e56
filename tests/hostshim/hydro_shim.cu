// Host build of the hydrostatic kernel's column sweep (hydro.cuh: hydro_shell), for a CPU test against
// the oracle: every shell of the grid in turn, cgs inputs as the kernel takes them.
#include "hydro.cuh"

extern "C" void host_hydro(int nr, int nt, const double* rf, const double* tf, const double* T, const double* rho_cur,
                           const double* shell_mass, double GM, double mu, double T_floor, double* rho_out) {
  for (int i = 0; i < nr; ++i) mcrt::hydro_shell(i, nt, rf, tf, T, rho_cur, shell_mass, GM, mu, T_floor, rho_out);
}
