"""Polarized transport (Mueller matrix per scattering, Sect. 2.3) on the GPU against the oracle: the same
Philox draws give the same scattering angles, planes and Stokes updates, so an FP64 run equals the
oracle's integer tallies and its Stokes sums up to the rounding of the fixed-point tallies; FP32 Q/I of
an optically thin scattering disk agrees within Monte Carlo errors."""
import math

import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

pytestmark = pytest.mark.gpu
QUNIT = 1048576.0


@pytest.fixture(scope="module")
def M():
    from paper_0902_3092_gb300 import build, mcrt
    build.build()
    mcrt.lib()
    return mcrt


def _scatter_disk(tau, albedo, nlam=4):
    op = disks.gray_opacity(nlam=nlam, albedo=albedo)
    return disks.make_disk(disks.log_r_faces(0.1, 100.0, 16), disks.midplane_refined_theta_faces(16),
                           disks.paper_star(), op, tau, h1_au=0.2, p=1.0, name="scatter")


def test_fp64_equals_oracle(M, oracle):
    """tau_mid = 3 gray disk, albedo 0.7, Rayleigh matrix, MRW: multiple scatterings, absorptions and
    jumps. Integer tallies equal; Q and U per inclination bin (summed over wavelength) within three
    fixed-point units (2^-20 of a packet each) of the oracle's."""
    d = _scatter_disk(3.0, 0.7)
    mu = disks.rayleigh_mueller(4, 181)
    n = 20_000
    g = M.Disk.from_model(d)
    g.set_mueller(mu)
    st = g.run_photons(n, seed=3, precision=64, mrw=True, gamma=2.0, nmin=5)
    ref = oracle.Run(d, mueller=mu).run(n, seed=3, mrw=True, gamma=2.0, nmin=5)
    t, v, a = g.tallies()
    assert np.array_equal(t, ref.tally) and np.array_equal(v, ref.visits) and np.array_equal(a, ref.nabs)
    for k in ("scatterings", "absorptions", "escaped", "mrw_jumps"):
        assert st[k] == ref.stats[k], k
    assert st["scatterings"] > 2000
    I, Q, U = (x.sum(axis=0) for x in g.sed_stokes())
    Io, Qo, Uo = (x.sum(axis=0) for x in ref.sed_stokes())
    e = d.star.L / n / QUNIT  # one fixed-point unit of one packet
    assert np.allclose(I, Io, rtol=1e-12, atol=0)
    assert np.all(np.abs(Q - Qo) <= 3 * e) and np.all(np.abs(U - Uo) <= 3 * e)
    assert np.abs(Qo).max() > 1000 * e
    g.close()


def test_fp32_thin_disk_polarization(M, oracle):
    """Rayleigh scattering (albedo 0.9999: the library takes no dust without absorption) in the optically
    thin disk of the oracle's single-scattering pin (h/r = 0.2, midplane optical depth 0.05): FP32 Q/I
    per inclination bin within four Monte Carlo errors of the oracle's (independent seeds; two oracle
    runs differ by at most 1.75 of these errors), positive and largest edge-on."""
    d = _scatter_disk(0.05, 0.9999)
    mu = disks.rayleigh_mueller(4, 181)
    n = 4_000_000
    g = M.Disk.from_model(d)
    g.set_mueller(mu)
    st = g.run_photons(n, seed=12)
    assert st["escaped"] == n and st["error_flags"] == 0
    I, Q, U = (x.sum(axis=0) for x in g.sed_stokes())
    ref = oracle.Run(d, mueller=mu).run(n, seed=11)
    Io, Qo, Uo = (x.sum(axis=0) for x in ref.sed_stokes())
    sig = math.sqrt(2 * 0.5 * ref.stats["scatterings"] / 10) / (n / 10)  # two runs, per bin
    assert np.all(np.abs(Q / I - Qo / Io) < 4 * sig), (Q / I, Qo / Io, sig)
    assert np.all(np.abs(U / I) < 4 * sig)
    assert Q[0] > 0 and Q[0] / I[0] > Q[9] / I[9]
    g.close()


def test_unpolarized_again_and_refusals(M):
    d = disks.config_plain_gray(10, 10, 30.0)
    a = M.Disk.from_model(d)
    a.run_photons(3000, seed=2, precision=64)
    b = M.Disk.from_model(d)
    b.set_mueller(disks.rayleigh_mueller(d.opacity.nlam, 91))
    with pytest.raises(M.McrtError) as e:
        b.trace(10, seed=1)
    assert e.value.status == 1
    with pytest.raises(M.McrtError) as e:
        M.Batch([b], [100])
    assert e.value.status == 1
    b.set_mueller(None)
    b.run_photons(3000, seed=2, precision=64)
    assert all(np.array_equal(x, y) for x, y in zip(a.tallies(), b.tallies()))
    with pytest.raises(M.McrtError) as e:
        b.sed_stokes()
    assert e.value.status == 7
    a.close()
    b.close()
