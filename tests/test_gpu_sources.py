"""Internal sources (viscous heating, Sect. 5) on the GPU against the oracle: the same Philox draws
pick the same source cells and release points, so FP64 runs give the oracle's integer tallies; FP32
temperatures agree statistically; zero sources change nothing."""
import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_0902_3092_gb300 import build, mcrt
    build.build()
    mcrt.lib()
    return mcrt


def _sources(d, scale):
    L = disks.viscous_sources(d)
    return L * (scale * d.star.L / L.sum())


def test_fp64_tallies_and_launches_equal_oracle(M, oracle):
    """Sources carrying 3x the star's luminosity on a tau_mid = 100 gray disk with MRW: identical
    tallies, entry and absorption counts; the traced launches (cell, position) agree."""
    d = disks.config_plain_gray(30, 24, 100.0)
    L = _sources(d, 3.0)
    n = 20_000
    g = M.Disk.from_model(d)
    g.set_sources(L)
    st = g.run_photons(n, seed=3, precision=64, mrw=True, gamma=2.0, nmin=5, want_sed=True)
    ref = oracle.Run(d, sources=L).run(n, seed=3, mrw=True, gamma=2.0, nmin=5)
    t, v, a = g.tallies()
    assert np.array_equal(t, ref.tally) and np.array_equal(v, ref.visits) and np.array_equal(a, ref.nabs)
    for k in ("absorptions", "scatterings", "escaped", "capped", "mrw_jumps", "deposit_sum"):
        assert st[k] == ref.stats[k], k
    T, _, _ = g.temperatures()
    To, _ = ref.temperatures()
    m = To > 0
    assert np.max(np.abs(T[m] / To[m] - 1)) < 1e-12
    # launches of the first packets: source cell (or the star, -1) and position
    tg = g.trace(200, seed=3, precision=64, max_events=4)
    to = oracle.Run(d, sources=L).run(200, seed=3, trace_packets=200, trace_max=4).trace
    assert np.array_equal(tg["cell"][:, 0], to["cell"][:, 0]) and np.array_equal(tg["type"][:, :2], to["type"][:, :2])
    assert (tg["cell"][:, 0] >= 0).sum() > 100
    assert np.allclose(tg["pos"][:, 0], to["pos"][:, 0], rtol=1e-12, atol=1e-9 * d.r_faces_cm[0])
    g.close()


def test_fp64_nongray_launches_equal_oracle(M, oracle):
    """Non-gray dust: the same draws choose the same source cells and release points, and each release
    is the packet's first event, an absorption in that cell. (The release's wavelength comes from the
    kernel's tabulated T-grid rows, the oracle's from exact Planck integrals, as for any absorption of
    non-gray dust, so the runs are not compared bit for bit.)"""
    d = disks.config_nongray(12, 10, 100.0)
    L = _sources(d, 3.0)
    g = M.Disk.from_model(d)
    g.set_sources(L)
    tg = g.trace(300, seed=2, precision=64, max_events=2, mrw=True, gamma=2.0, nmin=5)
    to = oracle.Run(d, sources=L).run(300, seed=2, mrw=True, gamma=2.0, nmin=5, trace_packets=300, trace_max=2).trace
    src = to["cell"][:, 0] >= 0
    assert src.sum() > 150
    assert np.array_equal(tg["cell"][:, 0], to["cell"][:, 0])
    assert np.all(tg["type"][src, 1] == 3) and np.all(to["type"][src, 1] == 3)
    assert np.array_equal(tg["cell"][src, 1], to["cell"][src, 1])
    assert np.allclose(tg["pos"][:, 0], to["pos"][:, 0], rtol=1e-12, atol=1e-9 * d.r_faces_cm[0])
    g.close()


def test_fp32_temperatures_match_oracle(M, oracle):
    """A tau_mid = 100 gray disk whose viscous heating outshines the star (10x), FP32 without MRW (so
    every deposit is one packet energy and the counting error below is the whole scatter; MRW with
    sources is checked bit for bit in FP64 above): temperatures of the cells with >= 1e3 absorption
    events in both runs agree with the oracle's (independent seeds) within four counting errors of the
    difference, sqrt(1/(16 N_gpu) + 1/(16 N_or)), plus 0.5 % for the FP32 path."""
    d = disks.config_plain_gray(30, 24, 100.0)
    L = _sources(d, 10.0)
    n = 100_000
    g = M.Disk.from_model(d)
    g.set_sources(L)
    st = g.run_photons(n, seed=8)
    assert st["escaped"] + st["capped"] == n and st["error_flags"] == 0
    T, _, _ = g.temperatures()
    _, _, nabs = g.tallies()
    ref = oracle.Run(d, sources=L).run(n, seed=9)
    To, _ = ref.temperatures()
    ng, no = nabs.reshape(T.shape).astype(float), ref.nabs.reshape(T.shape).astype(float)
    sel = (ng >= 1000) & (no >= 1000)
    assert sel.sum() >= 20
    sig = np.sqrt(1 / (16 * ng[sel]) + 1 / (16 * no[sel]))
    assert np.all(np.abs(T[sel] / To[sel] - 1) < 4 * sig + 0.005), np.max(np.abs(T[sel] / To[sel] - 1) / sig)
    g.close()


def test_zero_sources_and_validation(M):
    d = disks.config_plain_gray(12, 12, 50.0)
    a = M.Disk.from_model(d)
    a.run_photons(5000, seed=4, precision=64)
    b = M.Disk.from_model(d)
    b.set_sources(np.zeros(d.rho.shape))
    b.run_photons(5000, seed=4, precision=64)
    assert all(np.array_equal(x, y) for x, y in zip(a.tallies(), b.tallies()))
    bad = np.zeros(d.rho.shape)
    bad[3, 3] = -1.0
    with pytest.raises(M.McrtError) as e:
        b.set_sources(bad)
    assert e.value.status == 1
    empty = np.argwhere(d.rho == 0)
    if len(empty):
        bad = np.zeros(d.rho.shape)
        bad[tuple(empty[0])] = 1.0
        with pytest.raises(M.McrtError) as e:
            b.set_sources(bad)
        assert e.value.status == 1
    a.close()
    b.close()
