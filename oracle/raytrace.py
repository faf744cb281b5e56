"""Plain FP64 CPU oracle for the ray-traced observables of Min et al. 2009: the SED, images and
interferometric visibilities obtained by integrating the source function along straight rays through
the axisymmetric (r, theta) grid (Sect. 2.3, description of MCMax; Sect. 4.1 for the SED at 45 degrees
and the N-band visibilities at a 100 m baseline and 150 pc).

TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the benchmark's CPU-baseline leg
use this module. It shares no code with the CUDA library.

Readings (the paper states what is computed, not how):

* Temperatures: the Monte Carlo ones (the paper does not use the PDA temperatures for the observables,
  Sect. 4.1); the caller passes T.
* Source function per cell and wavelength bin: thermal emission over the total extinction,
  S_b = kappa_b Bbar_b(T) / (kappa_b + sigma_b), with Bbar_b the Planck function integrated over the
  bin; with the mean intensity J_b of a Monte Carlo run (path-length estimator) the scattered light
  sigma_b J_b / (kappa_b + sigma_b) is added (isotropic scattering). Without J, scattering removes light
  from a ray and adds none.
* Within a cell S and the extinction are constant, so the integral along a segment of optical depth
  dtau is exact: a segment adds S (1 - exp(-dtau)), dimmed by exp(-tau) of everything between it and
  the observer.
* The star is a point source at the origin: flux pi R*^2 Bbar_b(T*) / d^2, dimmed by the optical depth
  along the radial line from the origin towards the observer. Rays are not occulted by the star.
* Observer direction o = (sin i, 0, cos i) for inclination i from the disk axis; sky-plane axes
  e1 = (0, 1, 0) (along the major axis of the projected disk) and e2 = (-cos i, 0, sin i), so a ray
  is X(s) = p e1 + q e2 + s o and s grows towards the observer.
* Visibility at a baseline of length B and position angle PA (from e1 towards e2) at wavelength bin b:
  spatial frequency (u, v) = B (cos PA, sin PA) / lambda_b, lambda_b = sqrt(lambda_lo lambda_hi);
  V = |sum_k w_k I_kb exp(-2 pi i (u p_k + v q_k) / d) / d^2 + F*_b| / (sum_k w_k I_kb / d^2 + F*_b),
  the star's flux entering with phase 0.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as O

C_LIGHT = 2.99792458e10


def observer_axes(incl):
    """Unit vectors (o, e1, e2) of the observer direction and the sky plane (reading above)."""
    si, ci = math.sin(incl), math.cos(incl)
    o = np.array([si, 0.0, ci])
    e1 = np.array([0.0, 1.0, 0.0])
    e2 = np.array([-ci, 0.0, si])
    return o, e1, e2


def _cell_of(disk, X):
    """(ir, it) of the points X (n x 3); ir = -1 inside r_in or nr outside r_out."""
    r = np.sqrt((X * X).sum(axis=1))
    th = np.arccos(np.clip(X[:, 2] / np.where(r > 0, r, 1.0), -1.0, 1.0))
    ir = np.searchsorted(disk.r_faces_cm, r, side="right") - 1
    ir = np.where(r >= disk.r_faces_cm[-1], disk.nr, ir)
    it = np.clip(np.searchsorted(disk.theta_faces, th, side="right") - 1, 0, disk.ntheta - 1)
    return ir, it


def segments(disk, incl, p, q):
    """Cells and path lengths (cm) of the ray through sky point (p, q), in order of increasing s (towards
    the observer): every crossing of a radial sphere and of a polar cone is found in closed form, the
    crossings are sorted, and each piece between two consecutive crossings belongs to the cell of its
    midpoint. Returns (flat cell indices, lengths)."""
    o, e1, e2 = observer_axes(incl)
    X0 = p * e1 + q * e2
    b2 = p * p + q * q
    rf, tf = disk.r_faces_cm, disk.theta_faces
    if b2 >= rf[-1] ** 2:
        return np.zeros(0, np.int64), np.zeros(0)
    s_list = []
    # spheres |X0 + s o|^2 = r^2 with X0 . o = 0
    h = rf[rf * rf > b2]
    d = np.sqrt(h * h - b2)
    s_list += [d, -d]
    # cones: (x^2 + y^2) cos^2 t = z^2 sin^2 t on the nappe sign(z) = sign(cos t); plane z = 0 at t = pi/2
    for t in tf[1:-1]:
        ct, st = math.cos(t), math.sin(t)
        if abs(ct) < 1e-15:
            if o[2] != 0.0:
                s_list.append(np.array([-X0[2] / o[2]]))
            continue
        A = ct * ct * (o[0] ** 2 + o[1] ** 2) - st * st * o[2] ** 2
        B = ct * ct * (X0[0] * o[0] + X0[1] * o[1]) - st * st * X0[2] * o[2]
        Cc = ct * ct * (X0[0] ** 2 + X0[1] ** 2) - st * st * X0[2] ** 2
        if abs(A) < 1e-300:
            roots = [-Cc / (2 * B)] if B != 0 else []
        else:
            disc = B * B - A * Cc
            if disc < 0:
                continue
            sq = math.sqrt(disc)
            roots = [(-B - sq) / A, (-B + sq) / A]
        for s in roots:
            z = X0[2] + s * o[2]
            if z * ct > 0:
                s_list.append(np.array([s]))
    s_all = np.unique(np.concatenate(s_list))
    s_out = math.sqrt(rf[-1] ** 2 - b2)
    s_all = s_all[(s_all >= -s_out) & (s_all <= s_out)]
    s_all = np.unique(np.concatenate([[-s_out, s_out], s_all]))
    mid = 0.5 * (s_all[:-1] + s_all[1:])
    L = np.diff(s_all)
    ir, it = _cell_of(disk, X0[None, :] + mid[:, None] * o[None, :])
    ok = (ir >= 0) & (ir < disk.nr) & (L > 0)
    return (ir * disk.ntheta + it)[ok], L[ok]


def source(disk, T, J=None):
    """S[c, b] = kappa_b Bbar_b(T_c) / chi_b (erg s^-1 cm^-2 sr^-1 per bin), cells r-major; with the mean
    intensity J (nr, ntheta, nlam) of a Monte Carlo run, the isotropic scattering term sigma_b J_b / chi_b
    is added (the scattered light; exact for isotropic scattering)."""
    op = disk.opacity
    chi = op.kappa_abs + op.kappa_sca
    T = np.asarray(T, np.float64).ravel()
    S = np.zeros((T.size, op.nlam))
    for c, t in enumerate(T):
        if t > 0:
            S[c] = op.kappa_abs * O.planck_bins(op.lam_edges_um, t) / chi
    if J is not None:
        S += np.asarray(J, np.float64).reshape(T.size, op.nlam) * (op.kappa_sca / chi)[None, :]
    return S


def intensity(disk, T, incl, p, q, S=None):
    """Emergent intensity per wavelength bin of the ray through (p, q): the sum over segments of
    S (1 - exp(-dtau)) exp(-tau between the segment and the observer)."""
    if S is None:
        S = source(disk, T)
    cells, L = segments(disk, incl, p, q)
    op = disk.opacity
    chi = op.kappa_abs + op.kappa_sca
    if cells.size == 0:
        return np.zeros(op.nlam)
    rho = disk.rho.ravel()[cells]
    dtau = (rho * L)[:, None] * chi[None, :]
    front = np.cumsum(dtau[::-1], axis=0)[::-1] - dtau  # optical depth between each segment and the observer
    return (S[cells] * (1.0 - np.exp(-dtau)) * np.exp(-front)).sum(axis=0)


def image(disk, T, incl, p, q, J=None):
    S = source(disk, T, J)
    return np.array([intensity(disk, T, incl, pk, qk, S) for pk, qk in zip(p, q)])


def star_tau(disk, incl):
    """Optical depth per bin along the radial line from the origin towards the observer (polar angle
    incl), through the cells of the polar row that holds that angle."""
    it = int(np.clip(np.searchsorted(disk.theta_faces, incl, side="right") - 1, 0, disk.ntheta - 1))
    op = disk.opacity
    col = (disk.rho[:, it] * np.diff(disk.r_faces_cm)).sum()
    return col * (op.kappa_abs + op.kappa_sca)


def star_flux(disk, incl, dist):
    """Stellar flux per bin at distance dist (erg s^-1 cm^-2), dimmed along the line of sight."""
    op = disk.opacity
    Bs = O.planck_bins(op.lam_edges_um, disk.star.T_K)
    return math.pi * disk.star.R_cm ** 2 * Bs / dist ** 2 * np.exp(-star_tau(disk, incl))


def sed(disk, T, incl, dist, p, q, w, J=None):
    """Flux per bin (erg s^-1 cm^-2): sum_k w_k I_k / d^2 over the rays (w_k their sky-plane areas in
    cm^2) plus the star. Returns (total, disk part). J: add the scattered light (see source)."""
    I = image(disk, T, incl, p, q, J)
    Fd = (np.asarray(w)[:, None] * I).sum(axis=0) / dist ** 2
    return Fd + star_flux(disk, incl, dist), Fd


def bin_centre_cm(disk, b):
    e = disk.opacity.lam_edges_um
    return math.sqrt(e[b] * e[b + 1]) * 1e-4


def visibility(p, q, w, I_b, dist, lam_cm, B_cm, PA, F_star=0.0):
    """|V| of the image I_b (one wavelength) plus an unresolved star of flux F_star, at baseline B_cm and
    position angle PA (reading above)."""
    u = B_cm * math.cos(PA) / lam_cm
    v = B_cm * math.sin(PA) / lam_cm
    ph = -2.0 * math.pi * (u * np.asarray(p) + v * np.asarray(q)) / dist
    f = np.asarray(w) * np.asarray(I_b) / dist ** 2
    re = (f * np.cos(ph)).sum() + F_star
    im = (f * np.sin(ph)).sum()
    return math.hypot(re, im) / (f.sum() + F_star)
