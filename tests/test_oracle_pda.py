"""PDA solve (Sect. 2.2.1, Eq. 4) and its adjoint: exact 1-D solutions, manufactured harmonic
solutions, the maximum principle and central finite differences."""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_0902_3092_gb300 import disks


def custom_disk(rf, tf, rho, op=None):
    return disks.Disk(np.asarray(rf, float), np.asarray(tf, float), np.asarray(rho, float), disks.paper_star(),
                      op or disks.gray_opacity(), "custom")


def run_pda(oracle, d, pda_mask, T_bnd, kappa_R=None):
    visits = np.where(pda_mask, 0, 1000)
    relerr = np.where(pda_mask, np.inf, 0.01)
    tally = np.ones(d.nr * d.ntheta, np.uint64)
    return oracle.solve_pda(d, T_bnd, tally, visits, relerr, kappa_R=kappa_R)


def test_radial_shells_exact(oracle):
    """u depends on r only: u linear in int dr / (D r^2) between the two Dirichlet shells."""
    rng = np.random.default_rng(1)
    nr, nt = 24, 4
    rf = np.geomspace(1.0, 30.0, nr + 1) * disks.AU_CM
    tf = np.linspace(0, math.pi, nt + 1)
    rho_r = 1e-10 * np.exp(rng.normal(0, 1.0, nr))
    d = custom_disk(rf, tf, np.repeat(rho_r[:, None], nt, 1))
    mask = np.zeros((nr, nt), bool)
    mask[1:-1] = True
    Tb = np.full((nr, nt), 50.0)
    Tb[0], Tb[-1] = 1200.0, 80.0
    T, m, u, info = run_pda(oracle, d, mask, Tb)
    chi = 1000.0
    D = 1 / (3 * rho_r * chi)
    rc = 0.5 * (rf[:-1] + rf[1:])

    def R(a, b):  # int_a^b dr/(D(r) r^2), D piecewise constant on cells
        tot = 0.0
        for i in range(nr):
            lo, hi = max(a, rf[i]), min(b, rf[i + 1])
            if hi > lo:
                tot += integrate.quad(lambda r: 1 / (D[i] * r * r), lo, hi, epsrel=1e-13)[0]
        return tot

    Rt = R(rc[0], rc[-1])
    u0, u1 = 1200.0 ** 4, 80.0 ** 4
    for i in range(1, nr - 1):
        ue = u0 + (u1 - u0) * R(rc[0], rc[i]) / Rt
        assert np.allclose(u[i], ue, rtol=1e-10)


def test_polar_slab_exact(oracle):
    """u depends on theta only: T^4 linear in int dtheta / (D sin theta) -- the gray slab whose T^4
    is linear in optical depth."""
    rng = np.random.default_rng(2)
    nr, nt = 5, 18
    rf = np.geomspace(1.0, 3.0, nr + 1) * disks.AU_CM
    tf = np.linspace(0, math.pi, nt + 1)
    rho_t = 1e-11 * np.exp(rng.normal(0, 1.5, nt))
    d = custom_disk(rf, tf, np.repeat(rho_t[None, :], nr, 0))
    mask = np.zeros((nr, nt), bool)
    mask[:, 1:-1] = True
    Tb = np.full((nr, nt), 10.0)
    Tb[:, 0], Tb[:, -1] = 400.0, 900.0
    T, m, u, info = run_pda(oracle, d, mask, Tb)
    D = 1 / (3 * rho_t * 1000.0)
    tc = 0.5 * (tf[:-1] + tf[1:])

    def S(a, b):
        tot = 0.0
        for j in range(nt):
            lo, hi = max(a, tf[j]), min(b, tf[j + 1])
            if hi > lo:
                tot += integrate.quad(lambda t: 1 / (D[j] * math.sin(t)), lo, hi, epsrel=1e-13)[0]
        return tot

    St = S(tc[0], tc[-1])
    for j in range(1, nt - 1):
        ue = 400.0 ** 4 + (900.0 ** 4 - 400.0 ** 4) * S(tc[0], tc[j]) / St
        assert np.allclose(u[:, j], ue, rtol=1e-10)


def _harmonic_error(oracle, n, f):
    rf = np.linspace(1.0, 2.0, n + 1) * disks.AU_CM
    tf = np.linspace(0.6, 2.4, n + 1)
    d = custom_disk(rf, tf, np.full((n, n), 1e-12))
    rc = 0.5 * (rf[:-1] + rf[1:])[:, None]
    tc = 0.5 * (tf[:-1] + tf[1:])[None, :]
    ue = f(rc / disks.AU_CM, tc) * np.ones((n, n))
    mask = np.zeros((n, n), bool)
    mask[1:-1, 1:-1] = True
    T, m, u, info = run_pda(oracle, d, mask, ue ** 0.25)
    return np.max(np.abs(u - ue)[mask]) / np.max(np.abs(ue))


def test_manufactured_harmonic(oracle):
    # a + b/r is reproduced exactly by the series-resistance radial conductance
    assert _harmonic_error(oracle, 10, lambda r, t: 2.0 + 3.0 / r) < 1e-12
    # z = r cos(theta) (+ const): second-order convergence
    f = lambda r, t: 4.0 + r * np.cos(t)
    e = [_harmonic_error(oracle, n, f) for n in (8, 16, 32)]
    assert e[0] / e[1] > 3.0 and e[1] / e[2] > 3.0, e
    # r^2 (3 cos^2 - 1)/2 + const (an l = 2 harmonic)
    g = lambda r, t: 6.0 + r ** 2 * (3 * np.cos(t) ** 2 - 1) / 2
    e = [_harmonic_error(oracle, n, g) for n in (8, 16, 32)]
    assert e[0] / e[1] > 3.0 and e[1] / e[2] > 3.0, e


def _small_disk_problem(nongray=False, n=14):
    d = disks.config_nongray(n, n, 1e5) if nongray else disks.config_plain_gray(n, n, tau_mid=1e4)
    rc, tc = disks.cell_centres(d.r_faces_cm, d.theta_faces)
    T = 300.0 * (rc[:, None] / disks.AU_CM) ** -0.5 * (1 + 0.3 * np.cos(tc)[None, :] ** 2)
    mask = (d.rho > 0) & (np.abs(tc - math.pi / 2)[None, :] < 0.12) & (np.arange(n)[:, None] > 1)
    return d, T, mask


def test_maximum_principle(oracle):
    d, Tb, mask = _small_disk_problem()
    T, m, u, info = run_pda(oracle, d, mask, Tb)
    assert not np.any(m & ~mask)
    mask = m
    assert mask.sum() > 10
    A = info["A"]
    assert abs(A - A.T).max() < 1e-12 * abs(A).max()
    bnd = (~mask) & (d.rho > 0)
    assert T[mask].min() >= Tb[bnd].min() * (1 - 1e-12)
    assert T[mask].max() <= Tb[bnd].max() * (1 + 1e-12)


@pytest.mark.parametrize("nongray", [False, True])
def test_adjoint_against_finite_differences(oracle, nongray):
    d, Tb, mask = _small_disk_problem(nongray)
    rng = np.random.default_rng(7)
    kR = np.where(d.rho > 0, 1000.0 * np.exp(rng.normal(0, 0.3, d.rho.shape)), 1.0)
    w = np.where(mask, rng.uniform(0.5, 1.5, mask.shape), 0.0)
    T, m, u, info = run_pda(oracle, d, mask, Tb, kappa_R=kR)
    g_lr, g_kR, lam = oracle.pda_adjoint(d, u, m, info, w)

    def J(rho=None, kappa=None):
        dd = d if rho is None else custom_disk(d.r_faces_cm, d.theta_faces, rho, d.opacity)
        T2, *_ = run_pda(oracle, dd, mask, Tb, kappa_R=kR if kappa is None else kappa)
        return float(np.sum(w * T2))

    cells = np.argwhere((d.rho > 0) & (np.abs(g_lr) > 0))
    sel = cells[rng.choice(len(cells), size=min(25, len(cells)), replace=False)]
    h = 1e-5
    for i, j in sel:
        rp, rm = d.rho.copy(), d.rho.copy()
        rp[i, j] *= math.exp(h)
        rm[i, j] *= math.exp(-h)
        fd = (J(rho=rp) - J(rho=rm)) / (2 * h)
        assert math.isclose(g_lr[i, j], fd, rel_tol=1e-5, abs_tol=1e-6 * abs(g_lr).max()), (i, j)
        kp, km = kR.copy(), kR.copy()
        hk = h * kR[i, j]
        kp[i, j] += hk
        km[i, j] -= hk
        fdk = (J(kappa=kp) - J(kappa=km)) / (2 * hk)
        assert math.isclose(g_kR[i, j], fdk, rel_tol=1e-5, abs_tol=1e-6 * abs(g_kR).max()), (i, j)


def test_singular_region_is_rejected(oracle):
    """Every cell thick and in the PDA region: no Monte Carlo boundary value anywhere."""
    rf = np.geomspace(1.0, 3.0, 7) * disks.AU_CM
    tf = np.linspace(0, math.pi, 7)
    d = custom_disk(rf, tf, np.full((6, 6), 1e-10))
    with pytest.raises(ValueError):
        run_pda(oracle, d, np.ones((6, 6), bool), np.full((6, 6), 100.0))


def test_thickness_threshold_of_the_pda_region(oracle):
    """Reading of Sect. 2.2.1 ("regions of high optical depth"): an unvisited cell joins the PDA region only
    if it is optically thick across its smallest extent at the most opaque wavelength, rho * max_b chi'_b *
    min(dr, r dtheta) >= 1. Cells built on both sides of the threshold: one thick radially (3) but thin
    polarly (0.5) stays out (a test of dr alone would take it in); a non-gray cell thick only at its most
    opaque wavelength (1.5 there, 0.2 at the least) comes in (a test of the smallest chi' would leave it
    out); lowering the threshold to 0.25 lets the polarly thin cell in, which is what the reading decides."""
    rf = np.array([1.0, 1.3, 1.6]) * disks.AU_CM
    tf = np.array([0.0, 1.0, 1.05, np.pi / 2, np.pi - 1.05, np.pi - 1.0, np.pi])
    nr, nt = 2, 6
    rc = 0.5 * (rf[:-1] + rf[1:])
    dr = rf[1:] - rf[:-1]
    dth = tf[1:] - tf[:-1]
    op = disks.powerlaw_opacity(nlam=8, g=0.0)
    chip = op.kappa_abs + op.kappa_sca
    cmax, cmin = float(chip.max()), float(chip.min())
    rho = np.full((nr, nt), 1e-30)
    # (0, 1): polar extent rc dth = 0.05 rc, radial 0.3 AU: their ratio sets the two optical depths
    ext = min(dr[0], rc[0] * dth[1])
    assert ext == rc[0] * dth[1] < dr[0]
    rho[0, 1] = 0.5 / (cmax * ext)            # 0.5 across the smallest extent, 0.5 dr/ext > 1 radially
    assert rho[0, 1] * cmax * dr[0] > 1.0
    ext2 = min(dr[1], rc[1] * dth[1])
    rho[1, 1] = 1.5 / (cmax * ext2)           # 1.5 at the most opaque bin
    assert rho[1, 1] * cmin * ext2 < 1.0      # thin at the least opaque one
    d = custom_disk(rf, tf, rho, op)
    visits = np.zeros((nr, nt))
    relerr = np.full((nr, nt), np.inf)
    m = oracle.pda_mask(d, visits, relerr)
    assert not m[0, 1] and m[1, 1]
    m2 = oracle.pda_mask(d, visits, relerr, min_cell_tau=0.25)
    assert m2[0, 1] and m2[1, 1]
    # a visited cell with a small error never joins, however thick
    visits[1, 1], relerr[1, 1] = 1000, 0.01
    assert not oracle.pda_mask(d, visits, relerr)[1, 1]
