"""MRW escape-time law, Eq. 7-8, and its inverse used to sample the time spent in the sphere."""
import math

import numpy as np
from scipy import integrate


def _P_theta(x, n=60):
    # Jacobi theta transform of Eq. 7: 1 - P(x) = 2/sqrt(pi x) sum_{n>=0} exp(-(n+1/2)^2/x)
    k = np.arange(n)
    return 1.0 - 2.0 / math.sqrt(math.pi * x) * np.exp(-((k + 0.5) ** 2) / x).sum()


def test_series_matches_theta_transform(oracle):
    for x in [0.005, 0.01, 0.03, 0.1, 0.2, 0.5, 1.0, 2.0]:
        assert abs(oracle.mrw_P(x) - _P_theta(x)) < 2e-15, x


def test_limits(oracle):
    assert oracle.mrw_P(0.0) == 1.0
    # long-time asymptote P -> 2 exp(-pi^2 x)
    x = 3.0
    assert math.isclose(oracle.mrw_P(x), 2 * math.exp(-math.pi ** 2 * x), rel_tol=1e-12)


def test_inverse_solves_equation(oracle):
    for P0 in [1e-7, 1e-3, 0.1, 0.5, 0.9, 0.999, 1 - 2 ** -23]:
        x = oracle.mrw_x(P0)
        assert math.isclose(oracle.mrw_P(x), P0, rel_tol=1e-12, abs_tol=1e-15)


def test_moments_and_median(oracle):
    """E[x] = 1/6 (mean square displacement R0^2 = 6 D c t), E[x^2] = 7/180, median 0.1387853."""
    f = lambda P: oracle.mrw_x(P)
    m1 = integrate.quad(f, 0, 1, limit=200, epsabs=1e-12)[0]
    m2 = integrate.quad(lambda P: f(P) ** 2, 0, 1, limit=200, epsabs=1e-12)[0]
    assert abs(m1 - 1 / 6) < 1e-8
    assert abs(m2 - 7 / 180) < 1e-8
    assert abs(oracle.mrw_x(0.5) - 0.13878529704) < 1e-9


def _walk(R0, n, rng):
    p = np.zeros((n, 3))
    s = np.zeros(n)
    alive = np.ones(n, bool)
    while alive.any():
        k = np.flatnonzero(alive)
        mu = rng.uniform(-1, 1, k.size)
        ph = rng.uniform(0, 2 * np.pi, k.size)
        st = np.sqrt(1 - mu ** 2)
        d = np.stack([st * np.cos(ph), st * np.sin(ph), mu], 1)
        l = rng.exponential(1.0, k.size)
        b = (p[k] * d).sum(1)
        c = (p[k] ** 2).sum(1) - R0 ** 2
        t_exit = -b + np.sqrt(b * b - c)
        out = l >= t_exit
        step = np.where(out, t_exit, l)
        p[k] += step[:, None] * d
        s[k] += step
        alive[k[out]] = False
    return s * (1.0 / 3.0) / R0 ** 2  # x = s D / R0^2 with D = mfp/3


def test_brute_force_random_walk(oracle):
    """Plain isotropic random walk (unit mean free path) started at the centre of a sphere of
    radius R0: x = s D / R0^2 approaches the Eq. 7 law as R0 grows. For finite R0 the walk
    takes longer than the diffusion law (Sect. 3.2: the diffusion solution underestimates the
    time to leave a small sphere), with an excess that falls off like 1/R0."""
    rng = np.random.default_rng(5)
    x12 = _walk(12.0, 20000, rng)
    x24 = _walk(24.0, 20000, rng)
    e12, e24 = x12.mean() - 1 / 6, x24.mean() - 1 / 6
    assert 0.010 < e12 < 0.032
    assert 0.3 < e24 / e12 < 0.75
    # quantiles of the walk against the inverse of Eq. 7 at the larger sphere
    for q in (0.25, 0.5, 0.75):
        assert abs(np.quantile(x24, q) - oracle.mrw_x(1 - q)) < 0.02


def test_mrw_deposit_against_brute_force(oracle):
    """Eq. 9: the energy absorbed while crossing the sphere is E_gamma c t rho kappa_bar, i.e. on average
    kappa/chi times the path length in mean free paths: 3 E[x] tau0^2 (kappa/chi) = tau0^2 / 2 (kappa/chi)
    for the escape-time law. A brute-force walk of tau0 = 20 mean free paths counts its absorptions
    (albedo 1/2) and agrees once the 1/tau0 excess of small spheres is allowed for."""
    rng = np.random.default_rng(9)
    tau0, n = 20.0, 4000
    x = _walk(tau0, n, rng)  # x = s/(3 tau0^2), s the path length in mean free paths
    steps = 3 * x * tau0 ** 2
    absorbed = rng.binomial(np.maximum(1, np.rint(steps)).astype(np.int64), 0.5)
    law = 3 * (1 / 6) * tau0 ** 2 * 0.5  # Eq. 9 averaged over Eq. 7
    ratio = absorbed.mean() / law
    assert 1.0 < ratio < 1.0 + 3.0 / tau0
