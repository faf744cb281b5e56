"""The mean-intensity tally and the scattered light of the ray tracer on the GPU (Sect. 2.3: the
observables integrate the computed source function, scattering included), through the C ABI.

Tolerances. FP64 gray runs with want_sed = 0 keep every packet in its launch bin on both sides, and the
two sides follow the same events (the MRW trace tests), so every flight has the same length: the flight
part of J differs only by the order of the sums. An MRW walk adds c t = x R0^2 / D, with x from the
library's escape-time table (the tallies agree to 1e-4 for that reason), spread with Eq. 10's weights,
interpolated in the library's FP32 table of dBbar/dT on its temperature grid: within 3.4e-3 of the exact
weights where they exceed 1e-6, and 8.8e-6 of the cell's walk length everywhere (measured against the
oracle's fixed point of Eq. 13 over 5 K - 2000 K)."""
import math

import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

pytestmark = pytest.mark.gpu
PC = 3.0856775814913673e18


@pytest.fixture(scope="module")
def M():
    from paper_0902_3092_gb300 import build, mcrt
    build.build()
    mcrt.lib()
    return mcrt


def test_fp64_mean_intensity_matches_oracle(M, oracle):
    """Gray disk of tau_mid = 1e4 with MRW walks. The path length per bin over the whole disk
    (sum_c V_c J_cb) within 5e-3 of the oracle's plus 1e-4 of the total; J per cell (summed over bins)
    the same cells nonzero, within 1e-4 of the oracle's in 99 % of them and 2e-2 in all (a packet whose
    position drifts by up to 1e-4 over thousands of events, as in the MRW trace test, changes the flights
    it makes in a thin rim cell)."""
    d = disks.config_thick_gray(30, 20, 1e4)
    n = 2000
    g = M.Disk.from_model(d)
    g.keep_mean_intensity()
    assert not g.mean_intensity().any()  # before any run
    st = g.run_photons(n, seed=3, precision=64, mrw=True, gamma=2.0, want_sed=False)
    ref = oracle.Run(d).run(n, seed=3, mrw=True, gamma=2.0, want_sed=False, want_j=True)
    assert st["mrw_jumps"] == ref.stats["mrw_jumps"] > 0
    J, Jo = g.mean_intensity(), ref.mean_intensity()
    rf, tf = d.r_faces_cm, d.theta_faces
    V = (2 * np.pi / 3) * np.diff(rf ** 3)[:, None] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :]
    L, Lo = (np.einsum("ij,ijb->b", V, x) for x in (J, Jo))
    assert np.all(np.abs(L - Lo) <= 5e-3 * Lo + 1e-4 * Lo.sum())
    tot, toto = J.sum(axis=2), Jo.sum(axis=2)
    assert np.array_equal(tot > 0, toto > 0)
    m = toto > 0
    dev = np.abs(tot[m] / toto[m] - 1)
    assert np.mean(dev < 1e-4) >= 0.99 and dev.max() < 2e-2
    g.close()


def test_fp32_mean_intensity_balances_absorption(M, oracle):
    """Radiative equilibrium on the library's own outputs, non-gray dust with MRW: in every cell with
    100 or more packet energies, 4 pi m sum_b kappa_b J_b equals the absorbed energy that set the
    temperature, sum_b kappa_b Bbar_b(T) = sum_b kappa_b J_b, within five counting errors
    sqrt(n_abs) / (absorbed packet energies) plus 2e-3; cells where the walks deposit over 40 % take
    part."""
    d = disks.config_nongray(16, 16, 1e4)
    n = 200_000
    g = M.Disk.from_model(d)
    g.keep_mean_intensity()
    st = g.run_photons(n, seed=8, mrw=True, gamma=2.0, nmin=5)
    assert st["error_flags"] == 0 and st["mrw_jumps"] > 1000
    J = g.mean_intensity()
    T = g.temperatures()[0]
    t, _, a = g.tallies()
    units = t.reshape(d.nr, d.ntheta) / 65536.0
    nabs = a.reshape(d.nr, d.ntheta).astype(float)
    op = d.opacity
    n_mrw_cells = 0
    for i, j in zip(*np.nonzero(units >= 100)):
        absorbed = (op.kappa_abs * J[i, j]).sum()
        emitted = (op.kappa_abs * oracle.planck_bins(op.lam_edges_um, T[i, j])).sum()
        assert abs(absorbed / emitted - 1) < 5 * math.sqrt(nabs[i, j]) / units[i, j] + 2e-3, (i, j)
        n_mrw_cells += nabs[i, j] < 0.6 * units[i, j]
    assert n_mrw_cells >= 2
    g.close()


def test_fp64_scattered_light_sed_matches_oracle(M, oracle):
    """Scattering-dominated thin gray disk (albedo 0.9999, tau_mid = 0.05), no MRW, bins kept: the
    same flights on both sides, so J agrees to 1e-10 in 99.9 % of the cells and bins (FP64 face
    distances differ from the oracle's by ~1e-15, which could turn a rare near-tie into another event),
    and the ray-traced SED with the scattered light equals the oracle's ray tracer on the oracle's J to
    1e-6 of each bin; in the bins the packets reach, the scattered light is most of the disk's flux."""
    from oracle import raytrace as R
    op = disks.gray_opacity(nlam=4, albedo=0.9999)
    d = disks.make_disk(disks.log_r_faces(0.1, 100.0, 16), disks.midplane_refined_theta_faces(16),
                        disks.paper_star(), op, 0.05, h1_au=0.2, p=1.0, name="thin_scatter")
    n = 200_000
    g = M.Disk.from_model(d)
    g.keep_mean_intensity()
    g.run_photons(n, seed=7, precision=64, want_sed=False)
    ref = oracle.Run(d).run(n, seed=7, want_sed=False, want_j=True)
    J, Jo = g.mean_intensity(), ref.mean_intensity()
    assert np.array_equal(J > 0, Jo > 0)
    dev = np.abs(J[Jo > 0] / Jo[Jo > 0] - 1)
    assert np.mean(dev < 1e-10) > 0.999 and dev.max() < 1e-2
    T, _ = ref.temperatures()
    rays = disks.polar_rays(d.r_faces_cm, n_sub=1, n_phi=8, n_inner=2)
    incl, dist = math.radians(60.0), 100 * PC
    g.set_rays(incl, dist, rays)
    plain = g.raytrace(precision=64)["F"]
    F = g.raytrace(precision=64, scattering=True)["F"]
    Fo, Fdo = R.sed(d, T, incl, dist, rays.p, rays.q, rays.w, J=Jo)
    assert np.all(np.abs(F - Fo) <= 1e-6 * np.abs(Fo))
    Fd0 = R.sed(d, T, incl, dist, rays.p, rays.q, rays.w)[1]
    lit = Jo.sum(axis=(0, 1)) > 0
    assert lit.sum() >= 3
    assert np.all(Fdo[lit] > 2 * Fd0[lit]) and np.all(F[lit] > plain[lit]) and np.all(F[~lit] == plain[~lit])
    g.close()


def test_tally_leaves_transport_unchanged_and_refusals(M):
    """The same FP64 run with and without the tally: identical tallies and counters. Polarized disks,
    event traces and batches refuse it; the scattered light and J need it."""
    d = disks.config_thick_gray(30, 20, 1e4)
    a = M.Disk.from_model(d)
    sa = a.run_photons(1000, seed=4, precision=64, mrw=True)
    b = M.Disk.from_model(d)
    b.keep_mean_intensity()
    sb = b.run_photons(1000, seed=4, precision=64, mrw=True)
    assert all(np.array_equal(x, y) for x, y in zip(a.tallies(), b.tallies()))
    for k in ("events", "absorptions", "scatterings", "crossings", "mrw_jumps", "escaped"):
        assert sa[k] == sb[k], k
    with pytest.raises(M.McrtError) as e:
        b.trace(10, seed=1)
    assert e.value.status == 1
    with pytest.raises(M.McrtError) as e:
        M.Batch([b], [100])
    assert e.value.status == 1
    b.set_mueller(disks.rayleigh_mueller(d.opacity.nlam, 91))
    with pytest.raises(M.McrtError) as e:
        b.run_photons(100, seed=1)
    assert e.value.status == 1
    b.set_mueller(None)
    b.keep_mean_intensity(False)
    with pytest.raises(M.McrtError) as e:
        b.mean_intensity()
    assert e.value.status == 7
    b.set_rays(0.5, 100 * PC, disks.polar_rays(d.r_faces_cm, n_sub=1, n_phi=4, n_inner=1))
    with pytest.raises(M.McrtError) as e:
        b.raytrace(scattering=True)
    assert e.value.status == 7
    a.close()
    b.close()


def test_restore_zeroes_the_tallies_a_checkpoint_does_not_hold(M):
    """A checkpoint holds the integer tallies, not the path lengths: restoring one zeroes J (and the
    restored tallies are the checkpoint's)."""
    d = disks.config_plain_gray(10, 10, 30.0)
    g = M.Disk.from_model(d)
    g.keep_mean_intensity()
    g.run_photons(2000, seed=1, precision=64)
    blob = g.checkpoint()
    saved = g.tallies()
    g.run_photons(2000, seed=1, first_id=2000, precision=64)
    assert g.mean_intensity().any()
    g.restore(blob)
    assert not g.mean_intensity().any()
    assert all(np.array_equal(x, y) for x, y in zip(g.tallies(), saved))
    g.close()
