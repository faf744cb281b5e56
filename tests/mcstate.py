"""Synthetic Monte Carlo states for the tests.

A state is the integer cell tallies (absorbed packet energy, in units of 1/65536 of a packet) and the
packet entry counts of every cell, with the packet count they are normalised by. The GPU path takes a
state through the library's checkpoint format (mcrt_restore). The oracle takes the same arrays. Neither
side computes them, so a parity test of the temperatures, the PDA solve, its adjoint or the vertical
structure starts both sides from the same inputs.

The recipes hold none of the method's arithmetic. Tallies come from a wanted temperature field through
the gray balance q = 4 kappa sigma T^4 (each side then recomputes its exact T from the integers).
Entry counts are zero where a test wants the PDA region and 1e4 elsewhere.
"""
import math
import struct

import numpy as np

from paper_0902_3092_gb300 import disks

EUNIT = 65536
MAGIC = 0x4D43525443484B31  # checkpoint magic of the library's mcrt_checkpoint format, version 1


def volumes(d):
    rf, tf = d.r_faces_cm, d.theta_faces
    return (2 * math.pi / 3) * (rf[1:] ** 3 - rf[:-1] ** 3)[:, None] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :]


def thick(d, tau=1.0):
    """Cells whose smallest extent is at least `tau` extinction lengths at the most opaque wavelength."""
    rf, tf = d.r_faces_cm, d.theta_faces
    rc = 0.5 * (rf[:-1] + rf[1:])
    ext = np.minimum((rf[1:] - rf[:-1])[:, None], rc[:, None] * (tf[1:] - tf[:-1])[None, :])
    op = d.opacity
    return d.rho * float(np.max(op.kappa_abs + (1 - op.g) * op.kappa_sca)) * ext >= tau


def wanted_T(d):
    """A smooth temperature field (K) that falls with radius and rises away from the midplane."""
    rc, tc = disks.cell_centres(d.r_faces_cm, d.theta_faces)
    return 400.0 * (rc[:, None] / disks.AU_CM) ** -0.5 * (1 + 0.3 * np.cos(tc)[None, :] ** 2)


def midplane_band(d, half_width=0.15, first_shell=3):
    rc, tc = disks.cell_centres(d.r_faces_cm, d.theta_faces)
    return (d.rho > 0) & (np.abs(tc - math.pi / 2)[None, :] < half_width) & (np.arange(d.nr)[:, None] >= first_shell)


def deep_band(d, tau_min, first_shell=3):
    """Cells whose vertical optical depth from the nearer pole (along theta at the cell's radius, at the
    most opaque wavelength) exceeds tau_min: where few packets arrive in an optically thick disk."""
    rf, tf = d.r_faces_cm, d.theta_faces
    rc = 0.5 * (rf[:-1] + rf[1:])
    op = d.opacity
    dtau = d.rho * float(np.max(op.kappa_abs + (1 - op.g) * op.kappa_sca)) * rc[:, None] * np.diff(tf)[None, :]
    from_top = np.cumsum(dtau, axis=1) - 0.5 * dtau
    from_bottom = np.cumsum(dtau[:, ::-1], axis=1)[:, ::-1] - 0.5 * dtau
    depth = np.minimum(from_top, from_bottom)
    return (d.rho > 0) & (depth > tau_min) & (np.arange(d.nr)[:, None] >= first_shell)


def state_for(d, T_wanted, pda_region, n_total=10 ** 6, visits_elsewhere=10 ** 4, thick_only=True):
    """Tallies outside `pda_region`, none inside it; entry counts zero inside the region and
    `visits_elsewhere` outside. thick_only: tallies in the thick cells, for temperatures near T_wanted
    but at least 1000 packet energies each (counting error below 1 %; light cells run hotter).
    Otherwise: tallies for T_wanted in every dusty cell heavy enough to hold one tally unit at it."""
    q = 4 * d.opacity.kappa_abs[0] * disks.SIGMA_SB * T_wanted ** 4  # L_abs / m of a gray cell at T_wanted
    m = d.rho * volumes(d)
    t = np.floor(q * m * n_total * EUNIT / d.star.L)
    if thick_only:
        t = np.where(thick(d), np.maximum(t + 1, 1000 * EUNIT), 0)
    else:
        t = np.where(d.rho > 0, t, 0)
    tally = np.where(pda_region, 0, t).astype(np.uint64).ravel()
    visits = np.where(pda_region, 0, visits_elsewhere).astype(np.uint64).ravel()
    return tally, visits


def random_tallies(d, seed, n_total, T_lo=3.0, T_hi=3000.0, empty_fraction=0.2):
    """Seeded tallies on the dusty cells for temperatures log-uniform in [T_lo, T_hi] (through the gray
    balance, so a non-gray cell lands near, not at, its draw); a fraction of the cells, and those too
    light to hold one tally unit at their draw, left empty; entry counts Poisson around the tallies."""
    rng = np.random.default_rng(seed)
    n = d.nr * d.ntheta
    T = np.exp(rng.uniform(math.log(T_lo), math.log(T_hi), n)).reshape(d.rho.shape)
    q = 4 * d.opacity.kappa_abs[0] * disks.SIGMA_SB * T ** 4
    t = np.floor(q * d.rho * volumes(d) * n_total * EUNIT / d.star.L).ravel()
    t[(rng.random(n) < empty_fraction) | (d.rho.ravel() <= 0)] = 0
    t = t.astype(np.uint64)
    v = rng.poisson(t.astype(np.float64) / EUNIT + 1.0).astype(np.uint64)
    return t, v


def blob(d, tally, visits, n_total, nabs=None):
    """The library's checkpoint image of a Monte Carlo state: header (magic, version, nr, ntheta, nlam,
    packets as an integer and as a double, reserved), then tallies, entry counts and absorption counts
    per cell (uint64), then the escaping-energy spectrum, nlam x 10 inclination bins (zero)."""
    n = d.nr * d.ntheta
    hdr = struct.pack("<8Q", MAGIC, 1, d.nr, d.ntheta, d.opacity.nlam, int(n_total),
                      struct.unpack("<Q", struct.pack("<d", float(n_total)))[0], 0)
    a = np.zeros(n, np.uint64) if nabs is None else np.asarray(nabs, np.uint64)
    return hdr + np.asarray(tally, np.uint64).tobytes() + np.asarray(visits, np.uint64).tobytes() + a.tobytes() + \
        np.zeros(d.opacity.nlam * 10, np.uint64).tobytes()
