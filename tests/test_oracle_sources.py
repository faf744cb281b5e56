"""Pins of the oracle's internal sources (viscous heating, Sect. 5): the choice of the star or a cell
in proportion to the luminosities, release points uniform in the cell's volume, the energy balance of
an optically thin disk heated from inside, and no change at all without sources."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_0902_3092_gb300 import disks


def _launch_events(oracle, d, L, n, seed=1):
    r = oracle.Run(d, sources=L).run(n, seed=seed, want_sed=False, trace_packets=n, trace_max=2)
    tr = r.trace
    assert np.all(tr["type"][:, 0] == 0)  # launch first
    return r, tr["cell"][:, 0], tr["pos"][:, 0, :], tr["type"][:, 1]


def test_source_choice_frequencies(oracle):
    """Star with probability L*/L_tot, cell c with L_c/L_tot: binomial and chi^2 checks."""
    d = disks.config_plain_gray(8, 8, 1.0)
    rng = np.random.default_rng(3)
    L = np.zeros(d.rho.shape)
    sel = (d.rho > 0) & (rng.random(d.rho.shape) < 0.5)
    L[sel] = rng.uniform(0.2, 3.0, sel.sum())
    L *= 9.0 * d.star.L / L.sum()  # the star carries 10 %
    n = 40_000
    r, cell, pos, second = _launch_events(oracle, d, L, n)
    star = cell == -1
    p_star = 0.1
    assert abs(star.mean() - p_star) < 4 * math.sqrt(p_star * (1 - p_star) / n)
    # every cell packet is released by an absorption in its cell; the star's starts in the cavity
    assert np.all(second[~star] == 3)
    counts = np.bincount(cell[~star], minlength=d.nr * d.ntheta)
    expected = (L.ravel() / L.sum()) * (~star).sum()
    assert np.all(counts[expected == 0] == 0)
    m = expected > 0
    chi2 = ((counts[m] - expected[m]) ** 2 / expected[m]).sum()
    assert stats.chi2.sf(chi2, m.sum() - 1) > 1e-4
    assert math.isclose(r.packet_lum, d.star.L + L.sum(), rel_tol=1e-12)


def test_release_points_uniform_in_cell_volume(oracle):
    """One source cell: r^3 and cos(theta) of the release points are uniform across the cell (KS), the
    points lie at azimuth 0, inside the cell."""
    d = disks.config_plain_gray(6, 6, 1.0)
    L = np.zeros(d.rho.shape)
    ir, it = 3, 2
    L[ir, it] = 1e6 * d.star.L
    _, cell, pos, _ = _launch_events(oracle, d, L, 5000, seed=7)
    src = cell == ir * d.ntheta + it
    assert src.mean() > 0.99
    p = pos[src]
    r = np.linalg.norm(p, axis=1)
    mu = p[:, 2] / r
    r1, r2 = d.r_faces_cm[ir], d.r_faces_cm[ir + 1]
    c1, c2 = math.cos(d.theta_faces[it]), math.cos(d.theta_faces[it + 1])
    assert np.all(p[:, 1] == 0) and np.all((r >= r1 * (1 - 1e-12)) & (r <= r2 * (1 + 1e-12)))
    assert stats.kstest((r ** 3 - r1 ** 3) / (r2 ** 3 - r1 ** 3), "uniform").pvalue > 1e-3
    assert stats.kstest((mu - c1) / (c2 - c1), "uniform").pvalue > 1e-3


def test_thin_disk_heated_from_inside(oracle):
    """Optically thin gray disk (tau_mid = 1e-3) whose sources outshine the star 100 times: each
    cell's energy balance is 4 m kappa sigma T^4 = L_c (absorbed light adds O(tau)); within four
    counting errors 1/(4 sqrt(N_c)) on cells that released at least 400 packets."""
    d = disks.config_plain_gray(10, 8, 1e-3)
    L = disks.viscous_sources(d)
    L *= 100.0 * d.star.L / L.sum()
    n = 200_000
    r = oracle.Run(d, sources=L).run(n, seed=5, want_sed=False)
    st = r.stats
    assert st["escaped"] + st["capped"] == n
    T, _ = r.temperatures()
    rf, tf = d.r_faces_cm, d.theta_faces
    V = (2 * math.pi / 3) * (rf[1:] ** 3 - rf[:-1] ** 3)[:, None] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :]
    kappa = d.opacity.kappa_abs[0]
    with np.errstate(invalid="ignore", divide="ignore"):
        T_exp = (L / (4 * d.rho * V * kappa * disks.SIGMA_SB)) ** 0.25
    n_c = n * L / (L.sum() + d.star.L)
    ok = n_c >= 400
    assert ok.sum() >= 10
    err = np.abs(T[ok] / T_exp[ok] - 1)
    assert np.all(err < 4 / (4 * np.sqrt(n_c[ok])) + 3e-3), err.max()


def test_zero_sources_change_nothing(oracle):
    d = disks.config_plain_gray(10, 10, 30.0)
    a = oracle.Run(d).run(3000, seed=2, mrw=True, gamma=2.0)
    b = oracle.Run(d, sources=np.zeros(d.rho.shape)).run(3000, seed=2, mrw=True, gamma=2.0)
    assert np.array_equal(a.tally, b.tally) and np.array_equal(a.visits, b.visits)
    assert a.stats == b.stats
