"""Ray-traced observables (images, SED, visibilities) on the GPU against the FP64 oracle, through the C
ABI. Both sides take the same synthetic Monte Carlo state (restored tallies; each side computes its
temperatures from them) and the same rays.

Tolerances. FP64: the two sides find the same segments by different means (face-to-face stepping
against closed-form crossings sorted along the ray), so path lengths agree to rounding and the
intensities to 1e-9 of the bin's largest intensity. FP32: positions carry a relative error of ~6e-8
of the radius, so a segment's length is off by ~1e-7 r; in the rim-refined cells (1e-3 r_in wide) that
is 1e-4 of the length and of the cell's optical depth, and exp(-dtau) in FP32 adds ~1e-7 dtau; the
bound is 3e-4 of the bin's largest intensity and 5e-5 of the SED (which sums many rays whose errors
share a sign where they cross the same thin cells; measured 1.05e-5 on the 20 x 16 gray disk)."""
import math

import numpy as np
import pytest

import mcstate as S
from paper_0902_3092_gb300 import disks

pytestmark = pytest.mark.gpu
AU = disks.AU_CM
PC = 3.0856775814913673e18


@pytest.fixture(scope="module")
def M():
    from paper_0902_3092_gb300 import build, mcrt
    build.build()
    mcrt.lib()
    return mcrt


@pytest.fixture(scope="module")
def RT(oracle):
    from oracle import raytrace
    return raytrace


def setup(M, oracle, d, n_total=10 ** 6):
    """GPU disk and oracle temperatures from one synthetic state: tallies for a smooth field in every
    dusty cell heavy enough to hold one tally unit."""
    t, v = S.state_for(d, S.wanted_T(d), np.zeros(d.rho.shape, bool), n_total, thick_only=False)
    g = M.Disk.from_model(d)
    g.restore(S.blob(d, t, v, n_total))
    r = oracle.Run(d)
    r.tally[:] = t
    r.n_total = n_total
    T, _ = r.temperatures()
    return g, T


def close_to(got, ref, rel_of_max):
    scale = np.abs(ref).max(axis=0, keepdims=True)
    return np.all(np.abs(got - ref) <= rel_of_max * scale + 1e-300)


@pytest.mark.parametrize("kind", ["gray", "nongray"])
def test_image_and_sed_match_oracle(M, oracle, RT, kind):
    d = disks.config_plain_gray(20, 16, 30.0) if kind == "gray" else disks.config_nongray(20, 16, 1e3)
    g, T = setup(M, oracle, d)
    rays = disks.polar_rays(d.r_faces_cm, n_sub=1, n_phi=12, n_inner=2)
    dist = 140 * PC
    for incl in (0.2, math.pi / 4, 1.45):
        g.set_rays(incl, dist, rays)
        I_or = RT.image(d, T, incl, rays.p, rays.q)
        F_or, _ = RT.sed(d, T, incl, dist, rays.p, rays.q, rays.w)
        Fs_or = RT.star_flux(d, incl, dist)
        assert I_or.max() > 0
        for prec, tol, tol_sed in ((64, 1e-9, 1e-10), (32, 3e-4, 5e-5)):
            out = g.raytrace(precision=prec, want_image=True)
            assert out["segments"] > rays.n
            assert close_to(out["I"], I_or, tol), (incl, prec, np.max(np.abs(out["I"] - I_or) / I_or.max(0)))
            assert np.allclose(out["F_star"], Fs_or, rtol=1e-12, atol=0)
            assert np.allclose(out["F"], F_or, rtol=tol_sed, atol=1e-300), (incl, prec)
    g.close()


def test_visibilities_match_oracle(M, oracle, RT):
    """N-band visibility amplitudes (bins between 8 and 13 micron, 10-130 m baselines at two position
    angles) of the traced image against the oracle's direct Fourier sum of its own image."""
    d = disks.config_nongray(20, 16, 1e3)
    g, T = setup(M, oracle, d)
    rays = disks.polar_rays(d.r_faces_cm, n_sub=2, n_phi=24, n_inner=4)
    dist = 150 * PC
    incl = math.pi / 4
    g.set_rays(incl, dist, rays)
    I_or = RT.image(d, T, incl, rays.p, rays.q)
    Fs = RT.star_flux(d, incl, dist)
    lc = np.sqrt(d.opacity.lam_edges_um[:-1] * d.opacity.lam_edges_um[1:])
    nband = np.nonzero((lc > 8) & (lc < 13))[0]
    assert nband.size >= 3
    bins, B, PA = [], [], []
    for b in nband:
        for base in (10e2, 50e2, 100e2, 130e2):
            for pa in (0.0, 1.1):
                bins.append(b), B.append(base), PA.append(pa)
    ref = np.array([RT.visibility(rays.p, rays.q, rays.w, I_or[:, b], dist, RT.bin_centre_cm(d, b), base, pa,
                                  F_star=Fs[b]) for b, base, pa in zip(bins, B, PA)])
    assert ref.min() < 0.95  # resolved at the long baselines
    for prec, tol in ((64, 1e-9), (32, 2e-5)):
        g.raytrace(precision=prec)
        got = g.visibilities(bins, B, PA, with_star=True)
        assert np.max(np.abs(got - ref)) < tol, (prec, np.max(np.abs(got - ref)))
    g.close()


def test_full_size_sampled_rays(M, oracle, RT):
    """The 200 x 120 rim-refined tau_mid = 1e6 disk with the benchmark's rays at 45 degrees (FP32, the
    benchmark's launch): 40 seeded rays against the oracle one by one; all other rays finite and >= 0;
    the SED equals the weighted sum of the returned image plus the star."""
    d = disks.config_thick_gray(200, 120, 1e6)
    g, T = setup(M, oracle, d)
    rays = disks.polar_rays(d.r_faces_cm, n_sub=4, n_phi=128, n_inner=16)
    dist = 140 * PC
    incl = math.pi / 4
    g.set_rays(incl, dist, rays)
    out = g.raytrace(precision=32, want_image=True)
    I = out["I"]
    assert np.all(np.isfinite(I)) and I.min() >= 0
    pick = np.random.default_rng(2).choice(rays.n, 40, replace=False)
    S_or = RT.source(d, T)
    ref = np.array([RT.intensity(d, T, incl, rays.p[k], rays.q[k], S_or) for k in pick])
    scale = I.max(axis=0, keepdims=True)
    assert np.all(np.abs(I[pick] - ref) <= 3e-4 * scale), np.max(np.abs(I[pick] - ref) / scale)
    Fd = (rays.w[:, None] * I).sum(axis=0) / dist ** 2
    assert np.allclose(out["F"], Fd + out["F_star"], rtol=1e-6, atol=1e-300)
    g.close()


def test_edge_cases(M, oracle, RT):
    d = disks.config_plain_gray(12, 10, 50.0)
    g, T = setup(M, oracle, d)
    with pytest.raises(M.McrtError) as e:
        g.raytrace()
    assert e.value.status == 7  # no rays yet
    rf = d.r_faces_cm
    # one ray outside the grid, one grazing the outer sphere, one through the cavity on the axis line
    rays = disks.Rays(np.array([1.01 * rf[-1], 0.0, 0.999999 * rf[-1], 0.3 * rf[0]]),
                      np.array([0.0, 1.02 * rf[-1], 0.0, 0.0]), np.ones(4))
    for incl in (0.0, math.pi / 2, math.pi):
        g.set_rays(incl, 100 * PC, rays)
        out = g.raytrace(precision=64, want_image=True)
        ref = RT.image(d, T, incl, rays.p, rays.q)
        assert np.all(out["I"][:2] == 0)
        assert close_to(out["I"], ref, 1e-9)
    with pytest.raises(M.McrtError) as e:
        g.raytrace(which=M.T_PDA)
    assert e.value.status == 7  # no PDA solution
    with pytest.raises(M.McrtError) as e:
        g.set_rays(-0.1, 100 * PC, rays)
    assert e.value.status == 1
    g.close()
    # no dust: the disk is transparent and the SED is the bare star
    empty = disks.Disk(rf, d.theta_faces, np.zeros(d.rho.shape), d.star, d.opacity, "empty")
    g = M.Disk.from_model(empty)
    g.set_rays(0.7, 100 * PC, disks.polar_rays(rf, 1, 8, 2))
    out = g.raytrace(precision=32)
    assert out["segments"] == 0 and np.all(out["F"] == out["F_star"])
    assert np.allclose(out["F_star"], RT.star_flux(empty, 0.7, 100 * PC), rtol=1e-12)
    g.close()
    # more than 256 wavelength bins are refused
    wide = disks.Disk(rf, d.theta_faces, d.rho, d.star, disks.gray_opacity(nlam=300), "wide")
    g = M.Disk.from_model(wide)
    with pytest.raises(M.McrtError) as e:
        g.set_rays(0.7, 100 * PC, rays)
    assert e.value.status == 1
    g.close()


def test_source_follows_new_temperatures(M, oracle, RT):
    """A new Monte Carlo state (restored tallies) changes the temperatures, and the next trace uses them."""
    d = disks.config_plain_gray(16, 12, 20.0)
    g, T = setup(M, oracle, d)
    rays = disks.polar_rays(d.r_faces_cm, 1, 8, 2)
    g.set_rays(0.5, 100 * PC, rays)
    a = g.raytrace(precision=64, want_image=True)["I"]
    t, v = S.state_for(d, 2.0 * S.wanted_T(d), np.zeros(d.rho.shape, bool), 10 ** 6, thick_only=False)
    g.restore(S.blob(d, t, v, 10 ** 6))
    b = g.raytrace(precision=64, want_image=True)["I"]
    r = oracle.Run(d)
    r.tally[:] = t
    r.n_total = 10 ** 6
    T2, _ = r.temperatures()
    assert not np.allclose(a, b)
    assert close_to(b, RT.image(d, T2, 0.5, rays.p, rays.q), 1e-9)
    g.close()
