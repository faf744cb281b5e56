"""Plain FP64 CPU oracle for the vertical hydrostatic structure of Min et al. 2009, Sect. 2.5 ("Vertical
structure", Eq. 20).

TEST INFRASTRUCTURE. Only the test suite uses this module. It shares no code with the CUDA library.

Eq. 20: dP/dz = -rho G M_star z / R^3 with P = k_B rho T / (mu m_u), mu = 2.3, at fixed surface
density; the temperatures come from the Monte Carlo (+ PDA) solution and the iteration stops when the
mean difference of two consecutive temperature fields is below 3 sigma of their statistical errors.

Readings (the paper gives no discretisation):

* Columns are the polar rows of one radial shell of the (r, theta) grid: at the cell centres
  (r_c = (r_i + r_i+1) / 2, theta_c = (theta_j + theta_j+1) / 2), z = r_c cos theta_c and
  R = r_c sin theta_c. Eq. 20 is integrated along the shell in z,
  d ln(rho c^2) / dz = -G M z / (R^3 c^2),  c^2 = k_B T / (mu m_u),
  with the trapezoid rule between consecutive cell centres, from the pole at theta = 0 to the pole
  at theta = pi; so rho_j is proportional to exp(Phi_j) / T_j.
* "Surface density kept fixed": each shell keeps its dust mass, sum_j rho_j V_j = M_shell.
* Cells without dust stay without dust (the disk's inner and outer truncation); dust and gas
  share one temperature; temperatures below T_floor (cells the packets never heated) are raised
  to it.
* Convergence: mean over the cells that have a Monte Carlo error estimate in both iterations of
  |T_new - T_old| / sqrt(sigma_new^2 + sigma_old^2) with sigma = T * (relative error), < 3.
"""
from __future__ import annotations

import numpy as np

G_CGS = 6.67430e-8          # cm^3 g^-1 s^-2
K_B = 1.380649e-16          # erg / K
M_U = 1.66053906660e-24     # g
M_SUN = 1.98892e33          # g


def cell_volumes(r_faces, theta_faces):
    """Volumes of the (r, theta) cells of an axisymmetric grid (cm^3)."""
    rf = np.asarray(r_faces, np.float64)
    tf = np.asarray(theta_faces, np.float64)
    r1, r2 = rf[:-1], rf[1:]
    return (2.0 * np.pi / 3.0) * (r2 ** 3 - r1 ** 3)[:, None] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :]


def shell_masses(r_faces, theta_faces, rho):
    return (np.asarray(rho, np.float64) * cell_volumes(r_faces, theta_faces)).sum(axis=1)


def hydrostatic_density(r_faces, theta_faces, rho_mask, T, shell_mass, M_star=2.5 * M_SUN, mu=2.3, T_floor=1.0):
    """New density (g/cm^3) of every cell from Eq. 20 with the temperatures T (K), keeping each radial
    shell's mass and the cells where rho_mask is False empty."""
    rf = np.asarray(r_faces, np.float64)
    tf = np.asarray(theta_faces, np.float64)
    nr, nt = len(rf) - 1, len(tf) - 1
    V = cell_volumes(rf, tf)
    rho = np.zeros((nr, nt))
    GM = G_CGS * M_star
    for i in range(nr):
        rc = 0.5 * (rf[i] + rf[i + 1])
        Tc = np.maximum(np.asarray(T[i], np.float64), T_floor)
        phi = np.zeros(nt)
        a_prev = z_prev = None
        for j in range(nt):
            th = 0.5 * (tf[j] + tf[j + 1])
            z, R = rc * np.cos(th), rc * np.sin(th)
            a = GM * z / R ** 3 * (mu * M_U / (K_B * Tc[j]))  # G M z / (R^3 c^2)
            if j > 0:
                phi[j] = phi[j - 1] - 0.5 * (a + a_prev) * (z - z_prev)
            a_prev, z_prev = a, z
        lg = phi - np.log(Tc)
        m = np.asarray(rho_mask[i], bool)
        if not m.any() or not shell_mass[i] > 0:
            continue
        prof = np.where(m, np.exp(lg - lg[m].max()), 0.0)
        rho[i] = prof * (shell_mass[i] / (prof * V[i]).sum())
    return rho


def relaxed_density(r_faces, theta_faces, rho_cur, rho_h, a, shell_mass):
    """A damped step of the structure iteration (a reading: the paper iterates without damping): per radial
    shell i, log rho = (1 - a_i) log rho_cur + a_i log rho_h in the cells where both are positive (zero
    elsewhere), rescaled so that the shell keeps its mass. a_i = 1 returns rho_h."""
    V = cell_volumes(r_faces, theta_faces)
    rho_cur, rho_h = np.asarray(rho_cur, np.float64), np.asarray(rho_h, np.float64)
    out = np.array(rho_h, copy=True)
    for i, ai in enumerate(np.asarray(a, np.float64)):
        if ai == 1.0:
            continue
        ok = (rho_cur[i] > 0) & (rho_h[i] > 0)
        v = np.zeros_like(rho_h[i])
        v[ok] = np.exp((1.0 - ai) * np.log(rho_cur[i][ok]) + ai * np.log(rho_h[i][ok]))
        tot = (v * V[i]).sum()
        out[i] = v * (shell_mass[i] / tot) if tot > 0 else 0.0
    return out


def isothermal_shell_density(r_faces, theta_faces, i, T, M_star=2.5 * M_SUN, mu=2.3):
    """Closed form of Eq. 20 along shell i at constant T: integrating z / R^3 dz at fixed r gives
    1 / (r sin theta), so rho is proportional to exp(-(G M / (c^2 r)) (1 / sin theta - 1)), whose
    small-z limit is the Gaussian of scale height c (r^3 / (G M))^(1/2). Unnormalised (1 at the
    midplane)."""
    rf = np.asarray(r_faces, np.float64)
    tf = np.asarray(theta_faces, np.float64)
    rc = 0.5 * (rf[i] + rf[i + 1])
    th = 0.5 * (tf[:-1] + tf[1:])
    c2 = K_B * T / (mu * M_U)
    return np.exp(-(G_CGS * M_star / (c2 * rc)) * (1.0 / np.sin(th) - 1.0))


def convergence(T_old, err_old, T_new, err_new):
    """Mean of |T_new - T_old| / sigma over the cells with an error estimate in both fields; the
    structure is converged when it is below 3."""
    T_old, T_new = np.asarray(T_old), np.asarray(T_new)
    s_old, s_new = T_old * np.asarray(err_old), T_new * np.asarray(err_new)
    ok = (T_old > 0) & (T_new > 0) & np.isfinite(s_old) & np.isfinite(s_new) & (s_old > 0) & (s_new > 0)
    if not ok.any():
        return float("inf")
    return float(np.mean(np.abs(T_new[ok] - T_old[ok]) / np.sqrt(s_old[ok] ** 2 + s_new[ok] ** 2)))
