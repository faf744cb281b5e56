"""The transport kernels' per-packet code (transport.cuh: launch_packet, step, advance, interact, the MRW
chain, the mean-intensity tally and the polarization) compiled for the host, FP64 and FP32, over a model
built by the library's own host builders (tables.h), packets run one after another as one lane of a
single-disk kernel runs them, and compared with the oracle on the CPU.

Gray dust with MRW: the same events as the oracle (every counter, entry and absorption count equal);
energy tallies within 1e-5 (the tabulated MRW escape time, within 6e-6 of the exact inverse); the
mean intensity per cell within 1e-5, per bin within 5e-3 of itself plus 1e-5 of the cell's (the walks'
spectrum from the FP32 weight table). The J tally changes nothing else (the same run without
it: identical tallies and counters). Non-gray dust, where the tabulated re-emission sampling lets the
packets' histories part from the oracle's: radiative equilibrium on the run's own J and temperatures,
sum_b kappa_b J_b = sum_b kappa_b Bbar_b(T), in every cell with 100 packet energies, within four counting
errors plus 2e-3. Polarized transport: FP64 equal to the oracle's events, tallies and (within three
fixed-point units) Stokes sums; FP32 Q/I of a thin scattering disk within Monte Carlo errors."""
import ctypes as C
import dataclasses
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if not shutil.which("g++") or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers not found")
    out = tmp_path_factory.mktemp("transport") / "libhosttransport.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I", CUDA_INC,
                           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_0902_3092_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "hostshim", "transport_shim.cpp"), "-o", str(out)])
    return C.CDLL(str(out))


def run(lib, d, n, seed, mrw, gamma, nmin, want_sed, keep_j, prec=64, mueller=None, sources=None):
    op = d.opacity
    nc = d.nr * d.ntheta
    t, v, a = (np.zeros(nc, np.uint64) for _ in range(3))
    sed, q, u = (np.zeros(op.nlam * 10, np.uint64) for _ in range(3))
    j = np.zeros(nc * op.nlam) if keep_j else None
    cnt = np.zeros(8, np.uint64)
    arrs = [np.ascontiguousarray(x, np.float64) for x in
            (d.r_faces_cm, d.theta_faces, d.rho.ravel(), op.lam_edges_um, op.kappa_abs, op.kappa_sca, op.g)]
    mu = None if mueller is None else np.ascontiguousarray(mueller, np.float64)
    src = None if sources is None else np.ascontiguousarray(sources, np.float64).ravel()
    P = lambda x: None if x is None else x.ctypes.data_as(C.c_void_p)
    lib.host_transport(C.c_int(d.nr), C.c_int(d.ntheta), P(arrs[0]), P(arrs[1]), P(arrs[2]), C.c_int(op.nlam),
                       P(arrs[3]), P(arrs[4]), P(arrs[5]), P(arrs[6]), C.c_double(d.star.T_K), C.c_double(d.star.R_cm),
                       C.c_uint64(n), C.c_uint64(seed), C.c_int(mrw), C.c_double(gamma), C.c_int(nmin),
                       C.c_int(want_sed), C.c_int(prec), C.c_int(0 if mu is None else mu.shape[-1]), P(mu), P(src),
                       P(t), P(v), P(a), P(sed), P(q), P(u), P(j), P(cnt))
    out = dict(tally=t, visits=v, nabs=a, sed=sed, counters=cnt, sed_q=q.view(np.int64), sed_u=u.view(np.int64))
    if keep_j:  # path lengths (internal units, l = r_in) -> J = E_pkt * length / (4 pi V)
        rf, tf = d.r_faces_cm, d.theta_faces
        V = (2 * np.pi / 3) * np.diff(rf ** 3)[:, None] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :]
        Lpkt = d.star.L + (0.0 if src is None else src.sum())
        out["J"] = (Lpkt / n) * j.reshape(d.nr, d.ntheta, op.nlam) * rf[0] / (4 * np.pi * V[:, :, None])
    return out


def counters_of(stats):
    return [stats[k] for k in ("packets", "absorptions", "scatterings", "crossings", "mrw_jumps", "capped", "escaped",
                               "error_flags")]


def _scatter_disk(tau, albedo, nlam=4):
    op = disks.gray_opacity(nlam=nlam, albedo=albedo)
    return disks.make_disk(disks.log_r_faces(0.1, 100.0, 16), disks.midplane_refined_theta_faces(16),
                           disks.paper_star(), op, tau, h1_au=0.2, p=1.0, name="scatter")


def test_gray_mrw_transport_and_mean_intensity_match_oracle(lib, oracle):
    d = disks.config_thick_gray(30, 20, 1e4)
    n = 2000
    h = run(lib, d, n, seed=3, mrw=1, gamma=2.0, nmin=20, want_sed=0, keep_j=1)
    ref = oracle.Run(d).run(n, seed=3, mrw=True, gamma=2.0, want_sed=False, want_j=True)
    assert [int(x) for x in h["counters"]] == counters_of(ref.stats) and ref.stats["mrw_jumps"] > 1000
    assert np.array_equal(h["visits"], ref.visits) and np.array_equal(h["nabs"], ref.nabs)
    m = ref.tally > 0
    assert np.array_equal(h["tally"] > 0, m)
    assert np.max(np.abs(h["tally"][m].astype(float) / ref.tally[m].astype(float) - 1)) < 1e-5
    J, Jo = h["J"], ref.mean_intensity()
    tot, toto = J.sum(axis=2), Jo.sum(axis=2)
    assert np.array_equal(tot > 0, toto > 0)
    pos = toto > 0
    assert np.max(np.abs(tot[pos] / toto[pos] - 1)) < 1e-5
    # per bin: the walks' spectrum comes from the FP32 weight table (within 3.4e-3 of the exact weights
    # where they exceed 1e-6 of the total, zero where the exact ones fall below ~1e-45)
    assert np.all(np.abs(J - Jo) <= 5e-3 * Jo + 1e-5 * toto[:, :, None])
    # without the tally: the same transport
    h2 = run(lib, d, n, seed=3, mrw=1, gamma=2.0, nmin=20, want_sed=0, keep_j=0)
    for k in ("tally", "visits", "nabs", "sed", "counters"):
        assert np.array_equal(h[k], h2[k]), k


@pytest.mark.parametrize("prec", [64, 32])
def test_nongray_mean_intensity_balances_absorption(lib, oracle, prec):
    d = disks.config_nongray(16, 16, 1e4)
    n = 300_000
    h = run(lib, d, n, seed=8, mrw=1, gamma=2.0, nmin=5, want_sed=1, keep_j=1, prec=prec)
    assert int(h["counters"][4]) > 10_000 and int(h["counters"][7]) == 0
    r = oracle.Run(d)
    r.tally[:] = h["tally"]
    r.n_total = n
    T, _ = r.temperatures()
    op = d.opacity
    units = h["tally"].reshape(d.nr, d.ntheta) / 65536.0
    nabs = h["nabs"].reshape(d.nr, d.ntheta).astype(float)
    n_mrw_cells = 0
    for i, j in zip(*np.nonzero(units >= 100)):
        absorbed = (op.kappa_abs * h["J"][i, j]).sum()
        emitted = (op.kappa_abs * oracle.planck_bins(op.lam_edges_um, T[i, j])).sum()
        assert abs(absorbed / emitted - 1) < 4 * math.sqrt(nabs[i, j]) / units[i, j] + 2e-3, (i, j)
        n_mrw_cells += nabs[i, j] < 0.6 * units[i, j]
    assert n_mrw_cells >= 2


def test_fp64_polarized_transport_matches_oracle(lib, oracle):
    """tau_mid = 3 gray disk, albedo 0.7, Rayleigh matrix, MRW: the oracle's events and integer tallies
    exactly; Stokes Q and U per inclination bin (summed over wavelength) within three fixed-point units."""
    d = _scatter_disk(3.0, 0.7)
    mu = disks.rayleigh_mueller(4, 181)
    n = 20_000
    h = run(lib, d, n, seed=3, mrw=1, gamma=2.0, nmin=5, want_sed=1, keep_j=0, mueller=mu)
    ref = oracle.Run(d, mueller=mu).run(n, seed=3, mrw=True, gamma=2.0, nmin=5)
    assert [int(x) for x in h["counters"]] == counters_of(ref.stats) and ref.stats["scatterings"] > 2000
    for k in ("tally", "visits", "nabs"):
        assert np.array_equal(h[k], getattr(ref, k)), k
    Q, U = (h[k].reshape(4, 10).sum(axis=0) for k in ("sed_q", "sed_u"))
    Qo, Uo = (getattr(ref, k).reshape(4, 10).sum(axis=0) for k in ("sed_q", "sed_u"))
    assert np.all(np.abs(Q - Qo) <= 3) and np.all(np.abs(U - Uo) <= 3) and np.abs(Qo).max() > 1000


def test_fp32_thin_disk_polarization_matches_oracle(lib, oracle):
    """FP32 polarized transport of the optically thin Rayleigh-scattering disk (albedo 0.9999, h/r = 0.2,
    midplane optical depth 0.05): Q/I per inclination bin within four Monte Carlo errors of the oracle's
    (independent seeds), U/I consistent with zero, Q/I positive and largest edge-on."""
    d = _scatter_disk(0.05, 0.9999)
    mu = disks.rayleigh_mueller(4, 181)
    n = 1_000_000
    h = run(lib, d, n, seed=12, mrw=0, gamma=2.0, nmin=20, want_sed=1, keep_j=0, prec=32, mueller=mu)
    assert int(h["counters"][6]) == n and int(h["counters"][7]) == 0
    ref = oracle.Run(d, mueller=mu).run(n, seed=11)
    I, Q, U = (h[k].reshape(4, 10).sum(axis=0).astype(float) for k in ("sed", "sed_q", "sed_u"))
    Q, U = Q / 2 ** 20, U / 2 ** 20
    Io, Qo = ref.sed.reshape(4, 10).sum(axis=0).astype(float), ref.sed_q.reshape(4, 10).sum(axis=0) / 2 ** 20
    sig = math.sqrt(2 * 0.5 * ref.stats["scatterings"] / 10) / (n / 10)  # two runs, per bin
    assert np.all(np.abs(Q / I - Qo / Io) < 4 * sig), (Q / I, Qo / Io, sig)
    assert np.all(np.abs(U / I) < 4 * sig)
    assert Q[0] > 0 and Q[0] / I[0] > Q[9] / I[9]


def test_internal_sources_with_mean_intensity_match_oracle(lib, oracle):
    """Viscous-heating sources carrying 3x the star's luminosity on a tau_mid = 1e4 gray disk with MRW and
    the J tally (sources and the J tally together run on no GPU test): the oracle's absorptions,
    scatterings, MRW jumps and escapes exactly, and its absorption counts per cell; tallies and J per
    cell within 1e-5. Face crossings and cell entries may differ by a few: over hundreds of walks per
    packet the positions drift apart by rounding, and a packet grazing a cell's corner can cross a pair
    of faces on one side only (as in the MRW trace tests)."""
    d = disks.config_plain_gray(30, 24, 1e4)
    L = disks.viscous_sources(d)
    L *= 3.0 * d.star.L / L.sum()
    n = 500
    h = run(lib, d, n, seed=3, mrw=1, gamma=2.0, nmin=5, want_sed=1, keep_j=1, sources=L)
    ref = oracle.Run(d, sources=L).run(n, seed=3, mrw=True, gamma=2.0, nmin=5, want_j=True)
    got, want = [int(x) for x in h["counters"]], counters_of(ref.stats)
    for i in (0, 1, 2, 4, 5, 6, 7):  # all but the crossings
        assert got[i] == want[i], i
    assert abs(got[3] - want[3]) <= 4 + 1e-4 * want[3] and want[4] > 10_000
    assert np.array_equal(h["nabs"], ref.nabs)
    assert np.abs(h["visits"].astype(np.int64) - ref.visits.astype(np.int64)).sum() <= 8
    m = ref.tally > 0
    assert np.max(np.abs(h["tally"][m].astype(float) / ref.tally[m].astype(float) - 1)) < 1e-5
    tot, toto = h["J"].sum(axis=2), ref.mean_intensity().sum(axis=2)
    assert np.array_equal(tot > 0, toto > 0)
    assert np.max(np.abs(tot[toto > 0] / toto[toto > 0] - 1)) < 1e-5


@pytest.mark.parametrize("prec", [64, 32])
def test_j_tally_leaves_transport_unchanged_with_sed(lib, prec):
    """With the escape spectrum wanted, the J tally makes gray packets draw their bin at every event
    instead of once at escape; the transport itself (tallies, entries, absorptions, counters) is the same."""
    d = disks.config_thick_gray(30, 20, 1e4)
    a = run(lib, d, 1000, seed=4, mrw=1, gamma=2.0, nmin=20, want_sed=1, keep_j=0, prec=prec)
    b = run(lib, d, 1000, seed=4, mrw=1, gamma=2.0, nmin=20, want_sed=1, keep_j=1, prec=prec)
    assert int(a["counters"][4]) > 500
    for k in ("tally", "visits", "nabs", "counters"):
        assert np.array_equal(a[k], b[k]), k


# A packet of the 200x120 tau_mid = 1e6 benchmark disk (packet 1306294732 of the FP32 MRW run, seed 1) that
# the GPU's step guard dropped after 1e5 face crossings without an interaction: recorded position (units of
# the inner radius) and direction, FP32 values, in cell (0, 54). It lies on the inner sphere and moves along
# it (p.u / r = +6e-9 exactly), but in FP32 p.u rounds to -2.4e-9 and |p|^2 to 1.
TANGENT_STATE = dict(ir=0, it=54, p=(-0.874395668506622314453125, -0.4849975109100341796875, 0.01447851955890655517578125),
                     u=(0.48418593406677246, -0.8740962147712708, -0.03898179531097412))


def replay(lib, d, prec, state, tau=1.0, xcross=0, max_calls=300000):
    op = d.opacity
    arrs = [np.ascontiguousarray(x, np.float64) for x in
            (d.r_faces_cm, d.theta_faces, d.rho.ravel(), op.lam_edges_um, op.kappa_abs, op.kappa_sca, op.g)]
    st = np.array([state["ir"], state["it"], *state["p"], *state["u"], tau, xcross, max_calls], np.float64)
    out = np.zeros(6, np.int64)
    P = lambda x: x.ctypes.data_as(C.c_void_p)
    lib.host_replay(C.c_int(d.nr), C.c_int(d.ntheta), P(arrs[0]), P(arrs[1]), P(arrs[2]), C.c_int(op.nlam),
                    P(arrs[3]), P(arrs[4]), P(arrs[5]), P(arrs[6]), C.c_double(d.star.T_K), C.c_double(d.star.R_cm),
                    C.c_int(prec), P(st), P(out))
    return dict(calls=int(out[0]), crossings=int(out[1]), result=int(out[2]), err=int(out[3]), ir=int(out[4]),
                it=int(out[5]))


def test_tangent_packet_at_the_inner_radius_moves_on(lib):
    """The recorded state of the dropped packet, replayed by the FP32 per-packet code: the rounded p.u and
    |p| put the inner sphere at distance 0 and the chord through the cavity (2|p.u|) below the position's
    resolution, so without a minimum move after a crossing the packet steps between cell 0 and the cavity
    until the guard drops it. It must instead leave the face within a few crossings and reach its
    interaction point in the dense rim cell, without a guard flag."""
    f32 = lambda v: tuple(float(np.float32(x)) for x in v)
    st = dict(TANGENT_STATE, p=f32(TANGENT_STATE["p"]), u=f32(TANGENT_STATE["u"]))
    p, u = np.array(st["p"], np.float32), np.array(st["u"], np.float32)
    b = np.float32(np.float32(p[0] * u[0] + p[1] * u[1]) + p[2] * u[2])
    r2 = np.float32(np.float32(p[0] * p[0] + p[1] * p[1]) + p[2] * p[2])
    assert b < 0 and r2 == np.float32(1.0)  # the rounding that the state was recorded with
    d = disks.config_thick_gray(200, 120, 1e6)
    r = replay(lib, d, 32, st)
    assert r["err"] == 0 and r["crossings"] < 10 and r["result"] == 2, r
    # the same ray with a little optical depth left: it ends in cell 0 or 1 next to the face, not in the cavity
    assert r["ir"] in (0, 1), r


def test_grazing_rays_at_spheres_and_cones_make_progress(lib):
    """Rays started exactly on a face of the 200x120 disk and tangent to it (spheres at the rim, cones near the
    midplane), FP32 per-packet code with no optical depth used up (tau = 1e30 in a dust-free disk): each must
    leave the grid (a straight line meets each face at most twice), never stepping back and forth across the
    face it grazes. (The FP64 debug path keeps the oracle's geometry operation by operation, and both accept
    a root up to 1e-9 of the radius behind the packet as on the face, so an exactly tangent ray steps back
    and forth there until the crossing guard drops it.)"""
    prec = 32
    d = disks.config_thick_gray(200, 120, 1e6)
    d = dataclasses.replace(d, rho=np.zeros_like(d.rho))
    rng = np.random.default_rng(5)
    rf = d.r_faces_cm / d.r_faces_cm[0]
    tf = d.theta_faces
    bad = []
    for k in range(400):
        kind = k % 2
        if kind == 0:  # on sphere ir (the inner face of cell ir), tangent
            ir = int(rng.integers(0, 25))
            it = int(rng.integers(40, 80))
            th = tf[it] + rng.random() * (tf[it + 1] - tf[it])
            ph = rng.random() * 2 * np.pi
            n = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
            p = rf[ir] * n
            t = np.cross(n, rng.normal(size=3))
        else:  # on cone it (the lower face of cell it), tangent to the cone along its generator's normal
            ir = int(rng.integers(0, 40))
            it = int(rng.integers(50, 70))
            r = rf[ir] + rng.random() * (rf[ir + 1] - rf[ir])
            th, ph = tf[it], rng.random() * 2 * np.pi
            p = r * np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
            t = np.array([-np.sin(ph), np.cos(ph), 0.0])  # azimuthal: tangent to the cone
            t = t + 0.01 * rng.normal() * p / np.linalg.norm(p)
        t /= np.linalg.norm(t)
        st = dict(ir=ir, it=it, p=tuple(p), u=tuple(t))
        res = replay(lib, d, prec, st, tau=1e30, xcross=1, max_calls=5000)
        if res["err"] or res["calls"] >= 5000 or res["result"] != 0:
            bad.append((k, res))
    assert not bad, bad[:5]


def _run_interleaved(lib, d, n, lanes, seed):
    op = d.opacity
    arrs = [np.ascontiguousarray(x, np.float64) for x in
            (d.r_faces_cm, d.theta_faces, d.rho.ravel(), op.lam_edges_um, op.kappa_abs, op.kappa_sca, op.g)]
    t, v, a = (np.zeros(d.nr * d.ntheta, np.uint64) for _ in range(3))
    sed = np.zeros(op.nlam * 10, np.uint64)
    cnt = np.zeros(8, np.uint64)
    P = lambda x: x.ctypes.data_as(C.c_void_p)
    lib.host_transport_interleaved(C.c_int(d.nr), C.c_int(d.ntheta), P(arrs[0]), P(arrs[1]), P(arrs[2]),
                                   C.c_int(op.nlam), P(arrs[3]), P(arrs[4]), P(arrs[5]), P(arrs[6]),
                                   C.c_double(d.star.T_K), C.c_double(d.star.R_cm), C.c_uint64(n), C.c_uint64(seed),
                                   C.c_int(0), C.c_double(2.0), C.c_int(20), C.c_int(1), C.c_int(32),
                                   C.c_uint64(lanes), P(t), P(v), P(a), P(sed), P(cnt))
    assert int(cnt[5] + cnt[6]) == n  # capped + escaped
    return t.reshape(d.nr, d.ntheta)


def test_bjorkman_wood_depends_on_how_many_packets_are_in_flight(lib):
    """Why non-gray runs cap the packets in flight (MCRT_NONGRAY_IN_FLIGHT): the FP32 per-packet code on a
    12x10 non-gray disk of midplane optical depth 1e5 (5e4 packets, 16 seeds each), run one packet after
    another as Sect. 2.1's Bjorkman-Wood transport is, and with many packets in flight at once, each
    taking one step per round as a persistent kernel's lanes do. With a tenth of the packets in flight the
    inner-rim midplane absorbs far more energy (each re-emission's wavelength comes from temperatures the
    other packets move, and in these thick cells the wavelength decides how long a packet stays); with
    n / 3000 in flight, the library's default, it agrees with the one-at-a-time run."""
    d = disks.make_disk(disks.log_r_faces(0.1, 100.0, 12), disks.midplane_refined_theta_faces(10),
                        disks.paper_star(), disks.powerlaw_opacity(nlam=12, g=0.6), 1e5)
    n, j = 50_000, d.ntheta // 2

    def rim(lanes):
        x = np.array([float(_run_interleaved(lib, d, n, lanes, 100 + s)[0, j - 1:j + 1].sum()) for s in range(16)])
        return x.mean(), x.std(ddof=1) / np.sqrt(len(x))

    one, e1 = rim(1)
    many, em = rim(n // 10)
    few, ef = rim(max(1, n // 3000))
    assert (many - one) / np.hypot(e1, em) > 4.0, (one, many)
    assert abs(few - one) / np.hypot(e1, ef) < 3.0, (one, few)
