"""GPU PDA solve and adjoint against the FP64 oracle (scipy sparse direct solve), through the C ABI.

The Monte Carlo state (tallies -> temperatures, visit counts -> PDA region) is set through
mcrt_restore, so the GPU and the oracle solve the same system."""
import math
import struct

import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

pytestmark = pytest.mark.gpu
EUNIT = 65536


@pytest.fixture(scope="module")
def M():
    from paper_0902_3092_gb300 import build, mcrt
    build.build()
    mcrt.lib()
    return mcrt


def blob(d, tally, visits, n_total):
    n = d.nr * d.ntheta
    hdr = struct.pack("<8Q", 0x4D43525443484B31, 1, d.nr, d.ntheta, d.opacity.nlam, int(n_total),
                      struct.unpack("<Q", struct.pack("<d", float(n_total)))[0], 0)
    z = np.zeros(n, np.uint64)
    return hdr + np.asarray(tally, np.uint64).tobytes() + np.asarray(visits, np.uint64).tobytes() + z.tobytes() + \
        np.zeros(d.opacity.nlam * 10, np.uint64).tobytes()


def state_for(d, T_wanted, pda_mask, n_total=10 ** 6):
    """Integer tallies whose temperatures approximate T_wanted (gray or not: via the oracle's inversion
    the exact T used by both sides is recomputed from the tallies), visits 0 in the PDA region."""
    rf, tf = d.r_faces_cm, d.theta_faces
    V = (2 * math.pi / 3) * (rf[1:] ** 3 - rf[:-1] ** 3)[:, None] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :]
    m = d.rho * V
    from oracle import oracle as O
    kP = d.opacity.kappa_abs[0]
    q = 4 * kP * O.SIGMA_SB * T_wanted ** 4  # gray estimate of L_abs / m; exact T is recomputed below
    op = d.opacity
    chi_max = float(np.max(op.kappa_abs + (1 - op.g) * op.kappa_sca))
    thick = d.rho * chi_max * O.cell_extent(d) >= 1.0
    # thick cells outside the PDA region get >= 1000 packet energies, so their error is below 5 %
    tally = np.where(thick, np.maximum(np.floor(q * m * n_total * EUNIT / d.star.L) + 1, 1000 * EUNIT), 0)
    tally = tally.astype(np.uint64)
    tally = np.where(pda_mask, 0, tally).astype(np.uint64)
    visits = np.where(pda_mask, 0, 1000).astype(np.uint64)
    return tally.ravel(), visits.ravel()


def problem(kind):
    if kind == "gray":
        d = disks.config_plain_gray(24, 20, 1e4)
    else:
        d = disks.config_nongray(24, 20, 1e4)
    rc, tc = disks.cell_centres(d.r_faces_cm, d.theta_faces)
    T = 400.0 * (rc[:, None] / disks.AU_CM) ** -0.5 * (1 + 0.3 * np.cos(tc)[None, :] ** 2)
    mask = (d.rho > 0) & (np.abs(tc - math.pi / 2)[None, :] < 0.15) & (np.arange(d.nr)[:, None] > 2)
    return d, T, mask


@pytest.mark.parametrize("kind", ["gray", "nongray"])
def test_pda_matches_oracle(M, oracle, kind):
    d, Tw, mask = problem(kind)
    tally, visits = state_for(d, Tw, mask)
    g = M.Disk.from_model(d)
    g.restore(blob(d, tally, visits, 10 ** 6))
    n_pda, iters = g.solve_pda()
    Tg, errg, _ = g.temperatures(M.T_PDA)
    r = oracle.Run(d)
    r.tally[:] = tally
    r.n_total = 10 ** 6
    To_mc, eo = r.temperatures()
    To, mo, uo, info = oracle.solve_pda(d, To_mc, tally, visits, eo)
    assert n_pda == int(mo.sum()) > 20 and iters > 0
    assert not np.any(mo & ~mask)
    mask = mo
    assert np.max(np.abs(Tg[mask] / To[mask] - 1)) < 1e-6
    fin = (~mask) & (To > 0)
    assert np.allclose(Tg[fin], To[fin], rtol=1e-12, atol=0)


@pytest.mark.parametrize("kind", ["gray", "nongray"])
def test_adjoint_matches_oracle(M, oracle, kind):
    d, Tw, mask = problem(kind)
    tally, visits = state_for(d, Tw, mask)
    g = M.Disk.from_model(d)
    g.restore(blob(d, tally, visits, 10 ** 6))
    g.solve_pda()
    rng = np.random.default_rng(1)
    r = oracle.Run(d)
    r.tally[:] = tally
    r.n_total = 10 ** 6
    To_mc, eo = r.temperatures()
    To, mo, uo, info = oracle.solve_pda(d, To_mc, tally, visits, eo)
    w = np.where(mo, rng.uniform(0.5, 1.5, mo.shape), 0.0)
    gl, gk = g.pda_adjoint(w)
    ol, ok_, _ = oracle.pda_adjoint(d, uo, mo, info, w)
    s1, s2 = np.abs(ol).max(), np.abs(ok_).max()
    assert np.max(np.abs(gl - ol)) < 1e-6 * s1
    assert np.max(np.abs(gk - ok_)) < 1e-6 * s2


def test_pda_after_monte_carlo(M, oracle):
    """Full path on a thick gray disk: FP32 transport, temperatures, PDA; the oracle solves the PDA
    from the GPU's own tallies and visit counts."""
    d = disks.config_thick_gray(60, 40, 1e5)
    g = M.Disk.from_model(d)
    g.run_photons(200_000, seed=4, mrw=True, gamma=2.0)
    n_pda, iters = g.solve_pda()
    assert n_pda > 0
    Tg, _, _ = g.temperatures(M.T_PDA)
    t, v, _ = g.tallies()
    r = oracle.Run(d)
    r.tally[:] = t
    r.n_total = 200_000
    To_mc, eo = r.temperatures()
    To, mo, uo, info = oracle.solve_pda(d, To_mc, t, v, eo)
    assert int(mo.sum()) == n_pda
    assert np.max(np.abs(Tg[mo] / To[mo] - 1)) < 1e-6


def test_singular_region_rejected(M):
    """Every cell thick and in the PDA region: no Monte Carlo boundary value anywhere."""
    rf = np.geomspace(1.0, 3.0, 7) * disks.AU_CM
    tf = np.linspace(0, math.pi, 7)
    d = disks.Disk(rf, tf, np.full((6, 6), 1e-10), disks.paper_star(), disks.gray_opacity(), "uniform")
    tally = np.full(36, 1000 * EUNIT, np.uint64)
    visits = np.zeros(36, np.uint64)
    g = M.Disk.from_model(d)
    g.restore(blob(d, tally, visits, 10 ** 6))
    with pytest.raises(M.McrtError) as e:
        g.solve_pda()
    assert e.value.status == 1


@pytest.mark.parametrize("ntheta", [20, 22])
@pytest.mark.parametrize("legacy_stream", [False, True])
def test_pda_launch_paths(M, oracle, ntheta, legacy_stream):
    """The 16-byte kernels (ntheta % 4 == 0) and the 4-byte ones, each with the CG iterations replayed as
    a CUDA graph (the disk's own stream) or launched one by one (the legacy default stream, which
    cannot be captured), solve the same system as the oracle."""
    d = disks.config_plain_gray(24, ntheta, 1e4)
    rc, tc = disks.cell_centres(d.r_faces_cm, d.theta_faces)
    Tw = 400.0 * (rc[:, None] / disks.AU_CM) ** -0.5 * (1 + 0.3 * np.cos(tc)[None, :] ** 2)
    mask = (d.rho > 0) & (np.abs(tc - math.pi / 2)[None, :] < 0.15) & (np.arange(d.nr)[:, None] > 2)
    tally, visits = state_for(d, Tw, mask)
    g = M.Disk.from_model(d, stream=1 if legacy_stream else None)  # 1: cudaStreamLegacy
    g.restore(blob(d, tally, visits, 10 ** 6))
    n_pda, iters = g.solve_pda()
    Tg, _, _ = g.temperatures(M.T_PDA)
    r = oracle.Run(d)
    r.tally[:] = tally
    r.n_total = 10 ** 6
    To_mc, eo = r.temperatures()
    To, mo, _, _ = oracle.solve_pda(d, To_mc, tally, visits, eo)
    assert n_pda == int(mo.sum()) > 20 and iters > 0
    assert np.max(np.abs(Tg[mo] / To[mo] - 1)) < 1e-6
