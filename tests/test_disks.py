"""Synthetic disk inputs: Eq. 17-19 of Sect. 2.4."""
import math

import numpy as np
from scipy import integrate

from paper_0902_3092_gb300 import disks


def test_midplane_tau_matches_eq19():
    for p, tau in ((9 / 7, 100.0), (1.3, 1e6), (1.2, 3.0)):
        d = disks.make_disk(disks.log_r_faces(0.1, 100, 8), disks.midplane_refined_theta_faces(8),
                            disks.paper_star(), disks.gray_opacity(), tau, p=p)
        P = d.params
        f = lambda lnR: disks.density(math.exp(lnR) * disks.AU_CM, 0.0, P["rho0"], P["h1_au"], p, P["R_in_au"],
                                      P["R_out_au"]) * math.exp(lnR) * disks.AU_CM * P["chi_ref"]
        val = integrate.quad(f, math.log(P["R_in_au"]) + 1e-15, math.log(P["R_out_au"]) - 1e-15,
                             epsrel=1e-13, limit=200)[0]
        assert math.isclose(val, tau, rel_tol=1e-10)


def test_mass_matches_eq17_prefactor():
    rho0, h1, p, Ri, Ro = 2e-12, 0.03, 1.3, 0.75, 200.0
    def inner(R_au):
        h = h1 * R_au ** p
        zmax = 12 * h
        g = lambda z: disks.density(R_au * disks.AU_CM, z * disks.AU_CM, rho0, h1, p, Ri, Ro)
        return 2 * integrate.quad(g, 0, zmax, epsrel=1e-12)[0] * disks.AU_CM
    M = integrate.quad(lambda lnR: 2 * math.pi * math.exp(2 * lnR) * disks.AU_CM ** 2 * inner(math.exp(lnR)),
                       math.log(Ri) + 1e-12, math.log(Ro) - 1e-12, epsrel=1e-10, limit=200)[0]
    assert math.isclose(M, disks.disk_mass_eq17(rho0, h1, Ri, Ro), rel_tol=1e-6)


def test_theta_faces():
    t = disks.midplane_refined_theta_faces(40)
    assert t[0] == 0 and t[-1] == math.pi and t[20] == math.pi / 2
    assert np.all(np.diff(t) > 0)
    assert np.allclose(t + t[::-1], math.pi, atol=1e-15)


def test_rim_refined_grid():
    f = disks.rim_refined_r_faces(0.1, 100, 200) / disks.AU_CM
    assert len(f) == 201 and math.isclose(f[0], 0.1) and math.isclose(f[-1], 100)
    dr = np.diff(f)
    assert math.isclose(dr[0], 1e-4, rel_tol=1e-12)
    assert np.allclose(dr[1:20] / dr[:19], 1.3)
    assert 0.16 < f[20] < 0.17


def test_batch_sweep_ranges():
    ds, npk = disks.batch_sweep(64, seed=1)
    assert len(ds) == 64
    for d, n in zip(ds, npk):
        assert 50 <= d.nr <= 300 and 30 <= d.ntheta <= 180 and d.ntheta % 2 == 0
        assert 1e2 <= d.params["tau_mid"] <= 1e6 and 1e5 <= n <= 1e7
        assert 1 + 1 / 7 <= d.params["p"] <= 1 + 3 / 7
