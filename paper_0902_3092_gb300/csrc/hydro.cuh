// hydro.cuh -- one radial shell of the vertical hydrostatic structure (Sect. 2.5, Eq. 20): the column
// sweep of the hydrostatic kernel (host and device code; compiled for the host in the tests too).
#pragma once
#include <cmath>

#include "common.cuh"

namespace mcrt {

// Shell i (cgs: rf, tf the grid faces, T the temperatures, rho_cur the current density, shell_mass its
// mass): at the cell centres z = r_c cos theta_c, R = r_c sin theta_c, d ln(rho c^2)/dz = -G M z / (R^3 c^2)
// with c^2 = k_B T / (mu m_u), by the trapezoid rule from theta = 0 to pi; rho_j ~ exp(Phi_j) / T_j scaled
// to the shell's mass; cells without dust stay without dust, T below T_floor is raised to it.
__host__ __device__ inline void hydro_shell(int i, int nt, const double* rf, const double* tf, const double* T,
                                            const double* rho_cur, const double* shell_mass, double GM, double mu,
                                            double T_floor, double* rho_out) {
  constexpr double kKB = 1.380649e-16;       // erg / K
  constexpr double kMU = 1.66053906660e-24;  // g
  const double rc = 0.5 * (rf[i] + rf[i + 1]);
  const size_t row = (size_t)i * nt;
  double phi = 0.0, a_prev = 0.0, z_prev = 0.0, lgmax = -INFINITY;
  bool any = false;
  for (int j = 0; j < nt; ++j) {
    const double th = 0.5 * (tf[j] + tf[j + 1]);
    const double z = rc * cos(th), R = rc * sin(th);
    const double Tc = fmax(T[row + j], T_floor);
    const double a = GM * z / (R * R * R) * (mu * kMU / (kKB * Tc));  // G M z / (R^3 c^2)
    if (j > 0) phi = phi - 0.5 * (a + a_prev) * (z - z_prev);
    a_prev = a;
    z_prev = z;
    const double lg = phi - log(Tc);
    rho_out[row + j] = lg;
    if (rho_cur[row + j] > 0.0) {
      any = true;
      lgmax = fmax(lgmax, lg);
    }
  }
  const double M = shell_mass[i];
  if (!any || !(M > 0.0)) {
    for (int j = 0; j < nt; ++j) rho_out[row + j] = 0.0;
    return;
  }
  const double r1 = rf[i], r2 = rf[i + 1];
  const double sh = 2.0 * kPi / 3.0 * (r2 * r2 * r2 - r1 * r1 * r1);
  double sum = 0.0;
  for (int j = 0; j < nt; ++j) {
    double p = 0.0;
    if (rho_cur[row + j] > 0.0) {
      p = exp(rho_out[row + j] - lgmax);
      sum += p * (sh * (cos(tf[j]) - cos(tf[j + 1])));
    }
    rho_out[row + j] = p;
  }
  const double s = M / sum;
  for (int j = 0; j < nt; ++j) rho_out[row + j] *= s;
}

// Relaxed update of shell i: log rho_new = (1 - a) log rho_cur + a log rho_h in the cells with dust, then
// the shell rescaled to its mass (a damped step of the structure iteration; a = 1 leaves rho_h as it is).
// rho_h: in the Eq. 20 density of the shell (hydro_shell), out the relaxed one.
__host__ __device__ inline void hydro_relax(int i, int nt, const double* rf, const double* tf, const double* rho_cur,
                                            double a, const double* shell_mass, double* rho_h) {
  if (a == 1.0) return;
  const size_t row = (size_t)i * nt;
  const double r1 = rf[i], r2 = rf[i + 1];
  const double sh = 2.0 * kPi / 3.0 * (r2 * r2 * r2 - r1 * r1 * r1);
  double sum = 0.0;
  for (int j = 0; j < nt; ++j) {
    const double c = rho_cur[row + j], h = rho_h[row + j];
    const double v = (c > 0.0 && h > 0.0) ? exp((1.0 - a) * log(c) + a * log(h)) : 0.0;
    rho_h[row + j] = v;
    sum += v * (sh * (cos(tf[j]) - cos(tf[j + 1])));
  }
  const double M = shell_mass[i];
  const double s = sum > 0.0 ? M / sum : 0.0;
  for (int j = 0; j < nt; ++j) rho_h[row + j] *= s;
}

}  // namespace mcrt
