"""Pins of the oracle's polarized transport (full Mueller matrix per scattering, Sect. 2.3): the
sampling of the scattering angle and of the scattering plane against the phase matrix, the Stokes
update of a Rayleigh scatterer against its closed forms, the sky-frame rotation, and the Monte Carlo
polarization of an optically thin scattering disk against an independent single-scattering
quadrature over the cells."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_0902_3092_gb300 import disks


@pytest.fixture(scope="module")
def O(oracle):
    return oracle


def test_scattering_angle_follows_S11(O):
    """Stratified uniforms through the tabulated inverse CDF of S11 sin(theta): the cosine follows
    (3/8)(1 + mu^2) for Rayleigh and the Henyey-Greenstein law for g = 0.6 (closed-form CDFs)."""
    n = 4000
    xi = (np.arange(n) + 0.5) / n
    ray = disks.rayleigh_mueller(1, 181)[0, 0]
    mu = np.cos([O.pol_sample_theta(ray, x) for x in xi])
    F = 0.375 * (mu + mu ** 3 / 3) + 0.5  # P(cos <= mu)
    assert np.max(np.abs(F - (1 - xi))) < 1e-3
    g = 0.6
    hg = disks.hg_polarized_mueller([g], [0.0], 721)[0, 0]
    mu = np.cos([O.pol_sample_theta(hg, x) for x in xi])
    F = (1 - g * g) / (2 * g) * (1 / np.sqrt(1 + g * g - 2 * g * mu) - 1 / (1 + g))
    assert np.max(np.abs(F - (1 - xi))) < 2e-3


@pytest.mark.parametrize("a,q,u", [(-1.0, 1.0, 0.0), (-0.5, 0.0, 1.0), (0.3, 0.6, -0.8)])
def test_plane_azimuth_follows_polarization(O, a, q, u):
    """The azimuth of the scattering plane has density (1 + a (q cos 2phi + u sin 2phi)) / (2 pi):
    chi^2 of 2e5 seeded draws in 36 bins against the bin integrals of that density."""
    rng = np.random.default_rng(4)
    phi = np.array([O.pol_sample_phi(a, q, u, x) for x in rng.random(200_000)])
    assert phi.min() >= 0 and phi.max() <= 2 * math.pi
    edges = np.linspace(0, 2 * math.pi, 37)
    cnt, _ = np.histogram(phi, edges)
    prim = lambda x: x + a * (q * np.sin(2 * x) + u * (1 - np.cos(2 * x))) / 2
    exp = (prim(edges[1:]) - prim(edges[:-1])) / (2 * math.pi) * phi.size
    assert stats.chisquare(cnt, exp).pvalue > 1e-4


def _frame(rng):
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    e = np.cross(u, rng.normal(size=3))
    return u, e / np.linalg.norm(e)


def test_rayleigh_scattering_stokes(O):
    """Unpolarized light scattered by angle theta: q = -(1 - mu^2)/(1 + mu^2), u = v = 0, the new
    direction at angle theta from the old one in the plane of e turned by 2 pi w2, the new reference a
    unit vector perpendicular to it. Fully polarized light stays fully polarized (a dipole), to the
    table's interpolation error: between the 721 angles, linear S11, S12, S33 keep
    S11^2 = S12^2 + S33^2 to ~1e-5."""
    rng = np.random.default_rng(9)
    tab = disks.rayleigh_mueller(1, 721)[0]
    for _ in range(200):
        u, e = _frame(rng)
        w1, w2 = rng.random(2)
        un, en, st = O.pol_scatter(tab, u, e, [0.0, 0.0, 0.0], w1, w2)
        th = O.pol_sample_theta(tab[0], w1)
        c = math.cos(th)
        assert abs(un @ u - c) < 1e-9
        assert abs(np.linalg.norm(en) - 1) < 1e-12 and abs(en @ un) < 1e-12
        phi = 2 * math.pi * w2
        ep = e * math.cos(phi) + np.cross(u, e) * math.sin(phi)
        assert np.allclose(un, u * c + ep * math.sin(th), atol=1e-9)
        assert abs(st[0] + (1 - c * c) / (1 + c * c)) < 2e-4 and st[1] == 0 and st[2] == 0
        ang = rng.uniform(0, math.pi)
        _, _, s2 = O.pol_scatter(tab, u, e, [math.cos(2 * ang), math.sin(2 * ang), 0.0], *rng.random(2))
        assert abs(math.hypot(s2[0], math.hypot(s2[1], s2[2])) - 1) < 1e-4


def test_sky_frame_rotation(O):
    """Reference along the projected disk axis: unchanged; turned by 90 degrees: q and u change sign;
    along the axis itself: unchanged."""
    u = np.array([1.0, 0.0, 0.0])
    st = [0.3, -0.2, 0.1]
    assert np.allclose(O.pol_observer(u, [0, 0, 1.0], st), (0.3, -0.2))
    assert np.allclose(O.pol_observer(u, [0, 1.0, 0], st), (-0.3, 0.2))
    s = math.sqrt(0.5)
    q, uu = O.pol_observer(u, [0, s, s], st)
    assert abs(math.hypot(q, uu) - math.hypot(0.3, 0.2)) < 1e-12
    assert np.allclose(O.pol_observer(np.array([0, 0, 1.0]), [1.0, 0, 0], st), (0.3, -0.2))


def _single_scattering_Q_over_I(d, mus_per_bin=8, nsr=4, nst=4, nph=96):
    """Q/I per |cos i| bin of a gray Rayleigh-scattering disk in the single-scattering limit: starlight
    dimmed on its way in, scattered once by every point of every cell (sub-cell quadrature), plus the
    dimmed star; Q in the frame of the projected disk axis."""
    L = d.star.L
    ksca = d.opacity.kappa_sca[0]
    chi = d.opacity.kappa_abs[0] + ksca
    rf, tf = d.r_faces_cm, d.theta_faces
    tau0 = np.zeros(d.rho.shape)
    tau0[1:] = np.cumsum((d.rho * chi * np.diff(rf)[:, None])[:-1], axis=0)
    K, W = [], []
    for i in range(d.nr):
        re = np.linspace(rf[i] ** 3, rf[i + 1] ** 3, nsr + 1) ** (1 / 3)
        rm = 0.5 * (re[1:] + re[:-1])
        for j in range(d.ntheta):
            if d.rho[i, j] <= 0:
                continue
            ce = np.linspace(math.cos(tf[j]), math.cos(tf[j + 1]), nst + 1)
            cm = 0.5 * (ce[1:] + ce[:-1])
            dv = (np.diff(re ** 3) / 3)[:, None] * (-np.diff(ce))[None, :] * (2 * math.pi / nph)
            ph = (np.arange(nph) + 0.5) * 2 * math.pi / nph
            R, Cm, P = np.meshgrid(rm, cm, ph, indexing="ij")
            S = np.sqrt(1 - Cm ** 2)
            K.append(np.stack([S * np.cos(P), S * np.sin(P), Cm], -1).reshape(-1, 3))
            tin = tau0[i, j] + d.rho[i, j] * chi * (R - rf[i])
            W.append((np.broadcast_to(dv[:, :, None], R.shape) * d.rho[i, j] * ksca * L / (4 * math.pi * R ** 2)
                      * np.exp(-tin)).ravel())
    K, W = np.concatenate(K), np.concatenate(W)
    out = []
    for k in range(10):
        Iq = Qq = Id = 0.0
        for mo in k / 10 + (np.arange(mus_per_bin) + 0.5) / (10 * mus_per_bin):
            so = math.sqrt(1 - mo * mo)
            uo = np.array([so, 0.0, mo])
            c = K @ uo
            es = K - c[:, None] * uo[None, :]
            es /= np.linalg.norm(es, axis=1)[:, None]
            n = np.array([-mo * so, 0.0, 1 - mo * mo])
            n /= np.linalg.norm(n)
            cps, sps = es @ n, np.cross(uo[None, :], es) @ n
            Iq += (W * 0.75 * (1 + c * c)).sum() / (4 * math.pi)
            Qq += (W * 0.75 * (c * c - 1) * (cps ** 2 - sps ** 2)).sum() / (4 * math.pi)
            jj = min(int(np.searchsorted(tf, math.acos(mo), side="right")) - 1, d.ntheta - 1)
            Id += L / (4 * math.pi) * math.exp(-(d.rho[:, jj] * chi * np.diff(rf)).sum())
        out.append(Qq / (Iq + Id))
    return np.array(out)


def test_thin_disk_polarization_matches_single_scattering(O):
    """Pure Rayleigh scattering (albedo 1, gray) in a disk of h/r = 0.2 and midplane optical depth
    0.05: Monte Carlo Q/I per inclination bin within four Monte Carlo errors plus 6 % of the single-
    scattering quadrature (which leaves out the dimming on the way out and second scatterings, both
    of order the optical depth); positive (polarized across the disk plane), largest edge-on; U/I
    consistent with zero."""
    op = disks.gray_opacity(nlam=4, albedo=1.0)
    d = disks.make_disk(disks.log_r_faces(0.1, 100.0, 16), disks.midplane_refined_theta_faces(16),
                        disks.paper_star(), op, 0.05, h1_au=0.2, p=1.0, name="thin_scatter")
    n = 4_000_000
    r = O.Run(d, mueller=disks.rayleigh_mueller(4, 181)).run(n, seed=11, want_sed=True)
    I, Q, U = (x.sum(axis=0) for x in r.sed_stokes())
    mc, mcu = Q / I, U / I
    ref = _single_scattering_Q_over_I(d)
    sig = math.sqrt(0.5 * r.stats["scatterings"] / 10) / (n / 10)
    assert np.all(np.abs(mc - ref) < 4 * sig + 0.06 * np.abs(ref)), (mc, ref, sig)
    assert np.all(np.abs(mcu) < 4 * sig)
    assert ref[0] > 0 and ref[0] > ref[5] > ref[9]


def test_no_mueller_matrix_changes_nothing(O):
    d = disks.config_plain_gray(10, 10, 30.0)
    a = O.Run(d).run(3000, seed=2)
    b = O.Run(d, mueller=None).run(3000, seed=2)
    assert np.array_equal(a.tally, b.tally) and a.stats == b.stats
    assert not b.sed_q.any() and not b.sed_u.any()
