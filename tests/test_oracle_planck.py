"""Bin-integrated Planck function and its temperature derivative (used by Eq. 3, 10, 13)."""
import math

import numpy as np
from scipy import integrate

H, CL, KB = 6.62607015e-27, 2.99792458e10, 1.380649e-16
SIG = 2 * math.pi ** 5 * KB ** 4 / (15 * H ** 3 * CL ** 2)


def _g3_quad(x):
    f = lambda t: t ** 3 * math.exp(-t) / (-math.expm1(-t))
    return integrate.quad(f, x, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]


def _g4_quad(x):
    f = lambda t: t ** 4 * math.exp(-t) / (-math.expm1(-t)) ** 2
    return integrate.quad(f, x, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]


def test_G3_G4_against_quadrature(oracle):
    L = oracle.lib()
    for x in [1e-3, 0.05, 0.3, 0.999, 1.0, 1.5, 3.0, 10.0, 40.0]:
        assert math.isclose(L.oracle_G3(x), _g3_quad(x), rel_tol=1e-11), x
        assert math.isclose(L.oracle_G4(x), _g4_quad(x), rel_tol=1e-11), x
    assert math.isclose(L.oracle_G3(0.0), math.pi ** 4 / 15, rel_tol=1e-15)
    assert math.isclose(L.oracle_G4(0.0), 4 * math.pi ** 4 / 15, rel_tol=1e-15)


def test_bins_sum_to_stefan_boltzmann(oracle):
    e = np.geomspace(0.1, 1000, 101)
    for T in [3.0, 50.0, 700.0, 4000.0]:
        B = oracle.planck_bins(e, T)
        assert np.all(B >= 0)
        assert math.isclose(B.sum(), SIG * T ** 4 / math.pi, rel_tol=1e-12)
        dB = oracle.dplanck_bins(e, T)
        assert math.isclose(dB.sum(), 4 * SIG * T ** 3 / math.pi, rel_tol=1e-12)


def test_single_bin_against_direct_quadrature(oracle):
    e = np.geomspace(0.1, 1000, 101)
    T = 300.0
    B = oracle.planck_bins(e, T)
    for b in [5, 40, 63, 90]:
        nu1, nu2 = CL / (e[b + 1] * 1e-4), CL / (e[b] * 1e-4)
        Bnu = lambda nu: 2 * H * nu ** 3 / CL ** 2 / math.expm1(H * nu / (KB * T))
        ref = integrate.quad(Bnu, nu1, nu2, epsrel=1e-12)[0]
        assert math.isclose(B[b], ref, rel_tol=1e-9), b


def test_derivative_against_finite_difference(oracle):
    e = np.geomspace(0.1, 1000, 101)
    T, h = 150.0, 1e-3
    fd = (oracle.planck_bins(e, T + h) - oracle.planck_bins(e, T - h)) / (2 * h)
    dB = oracle.dplanck_bins(e, T)
    m = dB > 1e-12 * dB.max()
    assert np.allclose(dB[m], fd[m], rtol=1e-6)
