"""GPU PDA solve and adjoint against the FP64 oracle (scipy sparse direct solve), through the C ABI.

The Monte Carlo state (tallies -> temperatures, visit counts -> PDA region) is set through
mcrt_restore, so the GPU and the oracle solve the same system."""
import math

import numpy as np
import pytest

import mcstate as S
from paper_0902_3092_gb300 import disks

pytestmark = pytest.mark.gpu
EUNIT = S.EUNIT
blob = S.blob


@pytest.fixture(scope="module")
def M():
    from paper_0902_3092_gb300 import build, mcrt
    build.build()
    mcrt.lib()
    return mcrt


def problem(kind, ntheta=20):
    """tau_mid = 1e6: the midplane band is bounded above, below and at its inner edge by thick cells with
    Monte Carlo temperatures, so the PDA field varies by a factor of 2-3 across the band and depends on
    every conductance (at tau_mid = 1e4 only the inner edge bounds it and the solution is flat)."""
    if kind == "gray":
        d = disks.config_plain_gray(24, ntheta, 1e6)
    else:
        d = disks.config_nongray(24, ntheta, 1e6)
    return d, S.wanted_T(d), S.midplane_band(d)


def state_for(d, T_wanted, mask, n_total=10 ** 6):
    return S.state_for(d, T_wanted, mask, n_total)


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


def test_pda_after_monte_carlo(M):
    """Full path on a thick gray disk (FP32 transport, temperatures, PDA), checked through properties
    that hold for any Monte Carlo state, since the oracle takes no input from the GPU path:
    * the PDA region is the thick cells with fewer than 30 packet entries or a temperature error above
      5 % (Sect. 3.1, Sect. 2.2.1);
    * outside it the temperatures are the Monte Carlo ones, unchanged;
    * inside it T^4 solves a diffusion system whose off-diagonal couplings are negative and whose rows
      sum to zero once the Monte Carlo boundary cells are included, so every T^4 lies between the
      smallest and the largest T^4 of the Monte Carlo cells that border the region (discrete maximum
      principle);
    * a second solve of a fresh disk restored from the same state gives the same region and the same
      temperatures to 1e-6, the parity tolerance of the PDA tests (the CG dot products end in FP64
      atomics, whose order, and so the last bits of each iterate, may differ between runs)."""
    d = disks.config_thick_gray(60, 40, 1e5)
    g = M.Disk.from_model(d)
    g.run_photons(200_000, seed=4, mrw=True, gamma=2.0)
    T_mc, err, vis = g.temperatures()
    n_pda, iters = g.solve_pda()
    T, _, _ = g.temperatures(M.T_PDA)
    t, v, _ = g.tallies()
    t, v = t.reshape(d.rho.shape), v.reshape(d.rho.shape)
    region = (d.rho > 0) & S.thick(d) & ((v < 30) | (err > 0.05))
    assert n_pda == int(region.sum()) > 0 and iters > 0
    assert np.array_equal(T[~region], T_mc[~region])
    nb = np.zeros_like(region)
    nb[1:] |= region[:-1]
    nb[:-1] |= region[1:]
    nb[:, 1:] |= region[:, :-1]
    nb[:, :-1] |= region[:, 1:]
    bnd = nb & ~region & (d.rho > 0) & (t > 0)
    assert bnd.any()
    lo, hi = T_mc[bnd].min(), T_mc[bnd].max()
    assert np.all(T[region] >= lo * (1 - 1e-9)) and np.all(T[region] <= hi * (1 + 1e-9))
    ck = g.checkpoint()
    g2 = M.Disk.from_model(d)
    g2.restore(ck)
    assert g2.solve_pda()[0] == n_pda
    T2 = g2.temperatures(M.T_PDA)[0]
    assert np.max(np.abs(T2[region] / T[region] - 1)) < 1e-6 and np.array_equal(T2[~region], T[~region])


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
    d, Tw, mask = problem("gray", ntheta)
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
