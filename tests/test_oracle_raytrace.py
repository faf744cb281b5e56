"""Pins of the ray-tracing oracle (observables: SED, images, visibilities) against closed forms and
brute force."""
import math

import numpy as np
import pytest
from scipy import special

from paper_0902_3092_gb300 import disks

AU = disks.AU_CM
PC = 3.0856775814913673e18


@pytest.fixture(scope="module")
def R(oracle):
    from oracle import raytrace
    return raytrace


def shell(nr=6, nt=8, tau=2.0, nlam=12):
    """Uniform-density shell filling all polar angles, gray dust (albedo 0.5); tau = radial optical
    depth across the shell."""
    rf = np.geomspace(1.0, 3.0, nr + 1) * AU
    tf = np.linspace(0.0, math.pi, nt + 1)
    op = disks.gray_opacity(nlam=nlam)
    chi = float(op.kappa_abs[0] + op.kappa_sca[0])
    rho = np.full((nr, nt), tau / (chi * (rf[-1] - rf[0])))
    return disks.Disk(rf, tf, rho, disks.paper_star(), op, "shell"), chi


def S_of(oracle, d, T):
    op = d.opacity
    return op.kappa_abs * oracle.planck_bins(op.lam_edges_um, T) / (op.kappa_abs + op.kappa_sca)


def chord_pieces(rf, b):
    """Intervals of s (ray parameter, 0 at closest approach) inside the shell r_in <= r <= r_out."""
    so = math.sqrt(rf[-1] ** 2 - b * b)
    if b >= rf[0]:
        return [(-so, so)]
    si = math.sqrt(rf[0] ** 2 - b * b)
    return [(-so, -si), (si, so)]


def test_uniform_shell_closed_form(R, oracle):
    """Constant T and density: I = S (1 - exp(-rho chi L(b))) at any inclination, L(b) the chord through
    the shell (two pieces when the ray passes the inner cavity)."""
    d, chi = shell()
    T = np.full(d.rho.shape, 500.0)
    S = S_of(oracle, d, 500.0)
    rho = d.rho[0, 0]
    for incl in (0.0, 0.3, 1.0, math.pi / 2 - 0.2, math.pi / 2):
        for b_au, phi in ((0.0, 0.0), (0.5, 1.0), (1.0 + 1e-7, 2.0), (1.7, 0.4), (2.9, 3.5)):
            b = b_au * AU
            p, q = b * math.cos(phi), b * math.sin(phi)
            L = sum(hi - lo for lo, hi in chord_pieces(d.r_faces_cm, b))
            ref = S * (1 - np.exp(-rho * chi * L))
            got = R.intensity(d, T, incl, p, q)
            assert np.allclose(got, ref, rtol=1e-12, atol=0), (incl, b_au)


def test_hemispheres_order(R, oracle):
    """Different temperatures above and below the midplane: for 0 < i < 90 deg the ray runs from z < 0
    to z > 0, so I = S_up (1 - e^-tau_up) + S_low (1 - e^-tau_low) e^-tau_up. A reversed segment order
    or a swapped exponent fails."""
    d, chi = shell(nt=8, tau=3.0)
    tc = 0.5 * (d.theta_faces[:-1] + d.theta_faces[1:])
    T = np.where(tc[None, :] < math.pi / 2, 900.0, 300.0) * np.ones(d.rho.shape)
    Su, Sl = S_of(oracle, d, 900.0), S_of(oracle, d, 300.0)
    rho = d.rho[0, 0]
    for incl in (0.2, 0.8, 1.3):
        for b_au, phi in ((0.4, 0.7), (1.5, 2.2), (2.2, 4.0), (0.0, 0.0)):
            b = b_au * AU
            p, q = b * math.cos(phi), b * math.sin(phi)
            s_mid = -q * math.tan(incl)  # where z = q sin i + s cos i vanishes
            up = low = 0.0
            for lo, hi in chord_pieces(d.r_faces_cm, b):
                low += max(0.0, min(hi, s_mid) - lo)
                up += max(0.0, hi - max(lo, s_mid))
            tu, tl = rho * chi * up, rho * chi * low
            ref = Su * (1 - math.exp(-tu)) + Sl * (1 - math.exp(-tl)) * math.exp(-tu)
            got = R.intensity(d, T, incl, p, q)
            assert np.allclose(got, ref, rtol=1e-11, atol=0), (incl, b_au)


def test_segments_against_dense_sampling(R):
    """Path length per cell of rays through the rim-refined grid: the closed-form crossings against
    1e5 equally spaced points located one by one; total length = chord of the grid's outer sphere."""
    d = disks.config_thick_gray(30, 24, 1e3)
    rng = np.random.default_rng(3)
    rf = d.r_faces_cm
    for k in range(6):
        incl = rng.uniform(0, math.pi)
        b = rf[-1] * rng.uniform(0, 1) ** 2
        phi = rng.uniform(0, 2 * math.pi)
        p, q = b * math.cos(phi), b * math.sin(phi)
        cells, L = R.segments(d, incl, p, q)
        o, e1, e2 = R.observer_axes(incl)
        L_tot = sum(hi - lo for lo, hi in chord_pieces(rf, b))
        assert math.isclose(L.sum(), L_tot, rel_tol=1e-10)
        so = math.sqrt(rf[-1] ** 2 - b * b)
        n = 100_000
        s = -so + (np.arange(n) + 0.5) * (2 * so / n)
        X = (p * e1 + q * e2)[None, :] + s[:, None] * o[None, :]
        r = np.linalg.norm(X, axis=1)
        th = np.arccos(np.clip(X[:, 2] / r, -1, 1))
        ir = np.searchsorted(rf, r, side="right") - 1
        it = np.searchsorted(d.theta_faces, th, side="right") - 1
        ok = (ir >= 0) & (ir < d.nr)
        dense = np.bincount(ir[ok] * d.ntheta + it[ok], minlength=d.nr * d.ntheta) * (2 * so / n)
        exact = np.bincount(cells, weights=L, minlength=d.nr * d.ntheta)
        # every cell boundary moves a sample's worth of length at most
        assert np.max(np.abs(dense - exact)) <= 4 * (2 * so / n)
        assert set(np.nonzero(exact > 4 * (2 * so / n))[0]) <= set(np.nonzero(dense)[0])


def test_optically_thin_flux_limit(R, oracle):
    """tau_mid = 1e-5: the ray-traced disk flux tends to sum_c m_c kappa_b Bbar_b(T_c) / d^2 (each
    cell radiates 4 pi m kappa B into 4 pi d^2) as the rays are refined, face-on and inclined. The
    sky-plane sum is a midpoint rule in the ring radius, slowed near the outer edge by the square-root
    chord, so the bound is 1 % per bin at the finer sampling."""
    d = disks.config_plain_gray(16, 16, 1e-5)
    op = d.opacity
    rc, tc = disks.cell_centres(d.r_faces_cm, d.theta_faces)
    T = 300.0 * (rc[:, None] / AU) ** -0.5 * (1 + 0.3 * np.cos(tc)[None, :] ** 2)
    rf, tf = d.r_faces_cm, d.theta_faces
    V = (2 * math.pi / 3) * (rf[1:] ** 3 - rf[:-1] ** 3)[:, None] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :]
    m = d.rho * V
    dist = 100 * PC
    ref = sum(m.ravel()[c] * op.kappa_abs * oracle.planck_bins(op.lam_edges_um, T.ravel()[c])
              for c in range(T.size)) / dist ** 2
    sel = ref > 1e-6 * ref.max()
    for incl in (0.0, 0.7):
        errs, bol = [], []
        for n_sub, n_phi in ((2, 16), (8, 64)):
            rays = disks.polar_rays(rf, n_sub=n_sub, n_phi=n_phi, n_inner=2 * n_sub)
            _, Fd = R.sed(d, T, incl, dist, rays.p, rays.q, rays.w)
            errs.append(np.max(np.abs(Fd[sel] / ref[sel] - 1)))
            bol.append(abs(Fd.sum() / ref.sum() - 1))
        assert errs[1] < 0.01 and bol[1] < 0.006 and errs[1] < errs[0], (incl, errs, bol)
        if incl > 0:
            assert errs[1] < 0.5 * errs[0], errs


def test_star_flux(R):
    """Unattenuated: sum over the bins = sigma T*^4 R*^2 / d^2 (the bins cover the whole spectrum);
    through a uniform shell at any inclination: dimmed by exp(-rho chi (r_out - r_in))."""
    d, chi = shell(tau=0.7, nlam=40)
    dist = 140 * PC
    st = d.star
    empty = disks.Disk(d.r_faces_cm, d.theta_faces, np.zeros(d.rho.shape), st, d.opacity, "empty")
    F0 = R.star_flux(empty, 0.4, dist)
    assert math.isclose(F0.sum(), disks.SIGMA_SB * st.T_K ** 4 * st.R_cm ** 2 / dist ** 2, rel_tol=1e-12)
    for incl in (0.1, 1.0, 2.5):
        assert np.allclose(R.star_flux(d, incl, dist), F0 * math.exp(-0.7), rtol=1e-12)


def _disk_rays(a, n_rings=400, n_phi=64):
    edges = np.linspace(0.0, a, n_rings + 1)
    return disks.polar_rays(edges[1:], n_sub=1, n_phi=n_phi, n_inner=1)


def test_visibility_closed_forms(R):
    """Uniform disk of radius a: |2 J1(x) / x|, x = 2 pi (B / lambda)(a / d); Gaussian of width s:
    exp(-2 pi^2 (B / lambda)^2 (s / d)^2); an unresolved star adds with phase 0."""
    dist = 150 * PC
    a = 2.0 * AU
    lam = 10e-4
    rays = _disk_rays(a * 1.5)
    b = np.hypot(rays.p, rays.q)
    flat = (b < a).astype(float)
    # the ring edges fall on b = a only approximately: compare with the exact radius of the rings' area
    a_eff = math.sqrt(rays.w[b < a].sum() / math.pi)
    for B in (10e2, 50e2, 100e2, 130e2):
        for PA in (0.0, 0.9):
            x = 2 * math.pi * (B / lam) * (a_eff / dist)
            got = R.visibility(rays.p, rays.q, rays.w, flat, dist, lam, B, PA)
            assert abs(got - abs(2 * special.j1(x) / x)) < 2e-4, (B, got)
    s = 0.6 * AU
    gauss = np.exp(-b * b / (2 * s * s))
    for B in (20e2, 60e2, 100e2):
        ref = math.exp(-2 * math.pi ** 2 * (B / lam) ** 2 * (s / dist) ** 2)
        assert abs(R.visibility(rays.p, rays.q, rays.w, gauss, dist, lam, B, 0.3) - ref) < 1e-4
    # disk + star: (F_d V_d + F*) / (F_d + F*), V_d real for a centred symmetric image
    Fd = (rays.w * flat).sum() / dist ** 2
    B = 60e2
    x = 2 * math.pi * (B / lam) * (a_eff / dist)
    Vd = 2 * special.j1(x) / x
    got = R.visibility(rays.p, rays.q, rays.w, flat, dist, lam, B, 0.0, F_star=0.5 * Fd)
    assert abs(got - abs(Fd * Vd + 0.5 * Fd) / (1.5 * Fd)) < 2e-4
    assert R.visibility(rays.p, rays.q, rays.w, 0 * flat, dist, lam, B, 0.0, F_star=1.0) == 1.0
