"""GPU transport against the FP64 CPU oracle, through the C ABI."""
import math

import numpy as np
import pytest

import mcstate as S
from paper_0902_3092_gb300 import disks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_0902_3092_gb300 import build, mcrt
    build.build()
    mcrt.lib()
    return mcrt


def test_philox_stream_matches_oracle(M, oracle):
    for seed, model, packet in ((1, 0, 0), (0xDEADBEEF12345678, 0, 123456789), (7, 3, (1 << 40) + 5)):
        g = M.debug_uniforms(seed, model, packet, 257)
        o = oracle.uniforms(seed, model, packet, 257)
        assert np.array_equal(g, o)


def test_mrw_table_against_bisection(M, oracle):
    rng = np.random.default_rng(3)
    P = np.concatenate([rng.uniform(0, 1, 2000), [2 ** -24, 0.5 - 2 ** -24, 0.5, 0.5 + 2 ** -24, 1 - 2 ** -24]])
    P = np.clip(P, 2 ** -24, 1 - 2 ** -24)
    x = M.debug_mrw_x(P)
    ref = np.array([oracle.mrw_x(p) for p in P])
    assert np.max(np.abs(x / ref - 1)) < 2e-5


def _compare_traces(tg, to, nt, tol=1e-9):
    n_pk = tg["n"].shape[0]
    for k in range(n_pk):
        n = int(to["n"][k])
        assert int(tg["n"][k]) == n, (k, tg["n"][k], n)
        assert np.array_equal(tg["type"][k, :n], to["type"][k, :n]), k
        assert np.array_equal(tg["cell"][k, :n], to["cell"][k, :n]), k
        pg, po = tg["pos"][k, :n], to["pos"][k, :n]
        scale = np.maximum(np.linalg.norm(po, axis=1), 1.0)
        assert np.max(np.linalg.norm(pg - po, axis=1) / scale) < tol, k


@pytest.mark.parametrize("nr,nt,tau", [(8, 8, 30.0), (40, 40, 100.0)])
def test_fp64_trace_matches_oracle_event_by_event(M, oracle, nr, nt, tau):
    d = disks.config_plain_gray(nr=nr, ntheta=nt, tau_mid=tau)
    N, E = 400, 3000
    g = M.Disk.from_model(d)
    tg = g.trace(N, seed=1, max_events=E, want_sed=False)
    to = oracle.Run(d).run(N, seed=1, want_sed=False, trace_packets=N, trace_max=E).trace
    _compare_traces(tg, to, nt)
    # launch wavelength bin (stellar spectrum) agrees too
    assert np.array_equal(tg["lam"][:, 0], to["lam"][:, 0])


def test_fp64_tallies_bit_exact_c1(M, oracle):
    """The 40x40, tau_mid = 100 gray disk, 1e5 packets, seed 1: identical integer tallies."""
    d = disks.config_plain_gray()
    g = M.Disk.from_model(d)
    st = g.run_photons(100_000, seed=1, precision=64, want_sed=False)
    ref = oracle.Run(d).run(100_000, seed=1, want_sed=False)
    t, v, a = g.tallies()
    assert np.array_equal(t, ref.tally)
    assert np.array_equal(v, ref.visits)
    assert np.array_equal(a, ref.nabs)
    rs = ref.stats
    for k in ("absorptions", "scatterings", "crossings", "escaped", "capped", "deposit_sum"):
        assert st[k] == rs[k], k


@pytest.mark.parametrize("N,min_cells", [(100_000, 3), (1_000_000, 15)])
def test_fp32_temperatures_within_2_percent(M, oracle, N, min_cells):
    """FP32 production transport vs the oracle on the same Philox streams: per-cell T within 2 % in
    cells with >= 1e3 absorption events; total energy identities exact."""
    d = disks.config_plain_gray()
    g = M.Disk.from_model(d)
    st = g.run_photons(N, seed=1, precision=32, want_sed=True)
    T, err, vis = g.temperatures()
    ref = oracle.Run(d).run(N, seed=1, want_sed=False)
    To, eo = ref.temperatures()
    _, _, nabs = g.tallies()
    sel = nabs.reshape(T.shape) >= 1000
    assert sel.sum() >= min_cells
    rel = np.abs(T[sel] / To[sel] - 1)
    assert rel.max() <= 0.02, rel.max()
    assert st["escaped"] + st["capped"] == N
    t, _, _ = g.tallies()
    assert int(t.sum()) == st["deposit_sum"]
    assert st["error_flags"] == 0


def test_temperature_inversion_matches_oracle(M, oracle):
    """Same tallies -> same temperatures (FP64, gray closed form and non-gray bracketed Newton): seeded
    tallies for cell temperatures from 3 K to 3000 K, restored into the disk, so the oracle takes
    nothing from the GPU path."""
    for d in (disks.config_plain_gray(12, 12, 50.0), disks.config_nongray(12, 12, 1e3),
              disks.config_nongray(30, 24, 1e5)):
        t, v = S.random_tallies(d, seed=d.nr, n_total=20000)
        g = M.Disk.from_model(d)
        g.restore(S.blob(d, t, v, 20000))
        T, err, vis = g.temperatures()
        assert np.array_equal(vis, v.reshape(vis.shape))
        r = oracle.Run(d)
        r.tally[:] = t
        r.n_total = 20000
        To, eo = r.temperatures()
        assert (To > 0).sum() >= 40 and To[To > 0].max() / To[To > 0].min() > 100
        m = To > 0
        assert np.all((T > 0) == m)
        assert np.max(np.abs(T[m] / To[m] - 1)) < 1e-12
        assert np.allclose(err[np.isfinite(eo)], eo[np.isfinite(eo)], rtol=1e-14)


def test_energy_identities_and_sed(M, oracle):
    d = disks.config_plain_gray(20, 20, 300.0)
    N = 200_000
    g = M.Disk.from_model(d)
    st = g.run_photons(N, seed=11)
    L = g.sed(10)
    assert st["escaped"] + st["capped"] == N
    assert math.isclose(L.sum(), st["escaped"] * d.star.L / N, rel_tol=1e-12)
    # radiative equilibrium of the FP64 temperatures: sum 4 m kappa sigma T^4 = absorbed luminosity
    T, _, _ = g.temperatures()
    t, _, _ = g.tallies()
    rf, tf = d.r_faces_cm, d.theta_faces
    V = (2 * math.pi / 3) * (rf[1:] ** 3 - rf[:-1] ** 3)[:, None] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :]
    em = np.sum(4 * d.rho * V * d.opacity.kappa_abs[0] * oracle.SIGMA_SB * T ** 4)
    assert math.isclose(em, t.sum() / 65536 * d.star.L / N, rel_tol=1e-12)
    # spectrum against the oracle's (statistical: total escaped luminosity per wavelength bin)
    ref = oracle.Run(d).run(N, seed=11, want_sed=True)
    no = ref.sed.reshape(-1, 10).sum(1).astype(float)
    ng = np.rint(L.sum(1) * N / d.star.L)
    assert ng.sum() == no.sum() == st["escaped"]
    # per wavelength bin, Poisson-scale agreement (BW bins depend on the order of absorptions)
    assert np.all(np.abs(ng - no) <= 5 * np.sqrt(ng + no + 1) + 0.005 * no.max())


def test_resume_is_bitwise(M):
    """Gray FP32 runs without the tail kernel (whose batched interactions make a packet's floating-point
    order depend on whether it was in flight when the queue drained) resume bit for bit."""
    d = disks.config_plain_gray(16, 16, 100.0)
    a = M.Disk.from_model(d)
    a.run_photons(50_000, seed=3, n_total=50_000, tail_warps=-1)
    b = M.Disk.from_model(d)
    b.run_photons(20_000, seed=3, first_id=0, n_total=50_000, tail_warps=-1)
    blob = b.checkpoint()
    c = M.Disk.from_model(d)
    c.restore(blob)
    c.run_photons(30_000, seed=3, first_id=20_000, n_total=50_000, tail_warps=-1)
    for x, y in zip(a.tallies(), c.tallies()):
        assert np.array_equal(x, y)
    # escape directions are order independent for gray dust; the BW wavelength is not (it depends on
    # the tally seen at absorption time), so the spectrum is compared summed over wavelength
    assert np.allclose(a.sed().sum(0), c.sed().sum(0), rtol=1e-12, atol=0)


def test_tail_kernel_statistically_equal(M):
    """The tail kernel (batched interactions of the packets in flight at the drain) changes no physics:
    four seeds without it and four with it give per-run mean cell temperatures that agree within the
    run-to-run scatter (cells share packets, so runs, not cells, are the independent samples), and
    per-cell differences of the two groups' means as large as the within-group scatter predicts."""
    d = disks.config_thick_gray(60, 40, 1e5)
    g = M.Disk.from_model(d)
    T, V = {}, {}
    runs = [(-1, 11), (-1, 12), (-1, 13), (-1, 14), (0, 21), (0, 22), (0, 23), (0, 24)]
    for tw, seed in runs:
        g.reset()
        st = g.run_photons(1_000_000, seed=seed, mrw=True, gamma=2.0, max_events=10 ** 5, tail_warps=tw)
        assert st["escaped"] + st["capped"] == 1_000_000 and st["error_flags"] == 0
        T[seed], _, V[seed] = g.temperatures()
    ok = (np.minimum.reduce([V[s] for s in T]) > 3000) & (np.minimum.reduce([T[s] for s in T]) > 0)  # dusty cells
    assert ok.sum() > 200
    lg = {s: np.log(T[s][ok]) for s in T}
    a = np.array([lg[s] for tw, s in runs if tw < 0])
    b = np.array([lg[s] for tw, s in runs if tw >= 0])
    ma, mb = a.mean(axis=1), b.mean(axis=1)  # one mean log T per run
    se = np.sqrt(ma.var(ddof=1) / len(ma) + mb.var(ddof=1) / len(mb))
    assert abs(ma.mean() - mb.mean()) < 5 * se + 1e-4
    diff = a.mean(axis=0) - b.mean(axis=0)
    expected = np.sqrt(a.var(axis=0, ddof=1).mean() / len(a) + b.var(axis=0, ddof=1).mean() / len(b))
    assert np.sqrt(np.mean(diff ** 2)) < 1.5 * expected
