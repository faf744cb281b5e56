"""The hydrostatic kernel's column sweep (hydro.cuh: hydro_shell, Sect. 2.5, Eq. 20; host and device code)
compiled for the host and compared with the oracle's hydrostatic density on a seeded temperature field
with cells below the floor and dust-free cells: the same density to 1e-12 (relative, where it is above
1e-200 of the maximum), dust-free cells empty, every shell's mass kept."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
G_CGS = 6.67430e-8


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = tmp_path_factory.mktemp("hydro") / "libhydro.so"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_0902_3092_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "hostshim", "hydro_shim.cu"), "-o", str(out)])
    return C.CDLL(str(out))


def test_hydro_shell_matches_oracle(lib):
    from oracle import hydro as H
    d = disks.config_thick_gray(40, 30, 1e4)
    rho = d.rho.copy()
    rho[5, :4] = 0.0  # dust-free cells inside a shell
    rng = np.random.default_rng(3)
    rc = 0.5 * (d.r_faces_cm[1:] + d.r_faces_cm[:-1])
    T = 300.0 * (rc[:, None] / disks.AU_CM) ** -0.5 * np.exp(0.3 * rng.standard_normal(rho.shape))
    T[rng.random(rho.shape) < 0.1] = 0.0  # no packet: raised to the floor
    shell = H.shell_masses(d.r_faces_cm, d.theta_faces, rho)
    Ms = 2.5 * H.M_SUN
    want = H.hydrostatic_density(d.r_faces_cm, d.theta_faces, rho > 0, T, shell, M_star=Ms, mu=2.3, T_floor=10.0)
    P = lambda a: np.ascontiguousarray(a, np.float64).ctypes.data_as(C.c_void_p)
    got = np.zeros(rho.size)
    lib.host_hydro(d.nr, d.ntheta, P(d.r_faces_cm), P(d.theta_faces), P(T.ravel()), P(rho.ravel()), P(shell),
                   C.c_double(G_CGS * Ms), C.c_double(2.3), C.c_double(10.0), P(got))
    got = got.reshape(rho.shape)
    assert np.all(got[rho == 0] == 0)
    big = want > 1e-200 * want.max()
    assert big.sum() > 500
    assert np.max(np.abs(got[big] / want[big] - 1)) < 1e-12
    assert np.allclose(H.shell_masses(d.r_faces_cm, d.theta_faces, got), shell, rtol=1e-12, atol=0)


def test_hydro_relax_matches_oracle(lib):
    """The damped step of the structure iteration (hydro.cuh: hydro_relax) against the oracle's
    relaxed_density: the same density to 1e-12 for factors 0.3, 1 and 1.7 across the shells, the shells'
    masses kept, dust-free cells empty."""
    from oracle import hydro as H
    d = disks.config_thick_gray(40, 30, 1e4)
    rho = d.rho.copy()
    rho[5, :4] = 0.0
    rng = np.random.default_rng(4)
    rc = 0.5 * (d.r_faces_cm[1:] + d.r_faces_cm[:-1])
    T = 300.0 * (rc[:, None] / disks.AU_CM) ** -0.5 * np.exp(0.2 * rng.standard_normal(rho.shape))
    shell = H.shell_masses(d.r_faces_cm, d.theta_faces, rho)
    Ms = 2.5 * H.M_SUN
    rho_h = H.hydrostatic_density(d.r_faces_cm, d.theta_faces, rho > 0, T, shell, M_star=Ms, mu=2.3, T_floor=10.0)
    a = np.array([(0.3, 1.0, 1.7)[i % 3] for i in range(d.nr)])
    want = H.relaxed_density(d.r_faces_cm, d.theta_faces, rho, rho_h, a, shell)
    P = lambda x: np.ascontiguousarray(x, np.float64).ctypes.data_as(C.c_void_p)
    got = np.ascontiguousarray(rho_h, np.float64).ravel().copy()
    lib.host_hydro_relax(d.nr, d.ntheta, P(d.r_faces_cm), P(d.theta_faces), P(rho.ravel()), P(a), P(shell),
                         got.ctypes.data_as(C.c_void_p))
    got = got.reshape(rho.shape)
    assert np.all(got[rho == 0] == 0)
    big = want > 1e-200 * want.max()
    assert big.sum() > 500
    assert np.max(np.abs(got[big] / want[big] - 1)) < 1e-12
    assert np.allclose(H.shell_masses(d.r_faces_cm, d.theta_faces, got), shell, rtol=1e-12, atol=0)


def test_halves_statistic_is_0_9_for_noise_and_grows_with_a_change():
    """temperature_change_halves on synthetic Monte Carlo noise: each iteration's T is the mean of two
    halves with N(0, 2 s^2) errors, so T has error s and sigma = |T_a - T_b| / 2 is half-normal with
    scale s. Then E|T_new - T_old| = 2 s / sqrt(pi) and E sqrt(sigma_old^2 + sigma_new^2) = s sqrt(pi / 2)
    (Rayleigh): a ratio of 2 sqrt(2) / pi = 0.900 for noise alone, whatever s is per cell. A systematic
    change of 3 s in every cell raises it (to ~2.4)."""
    from paper_0902_3092_gb300.hydro import temperature_change_halves
    rng = np.random.default_rng(21)
    n = 200_000
    mu = rng.uniform(20.0, 800.0, n)
    s = mu * rng.uniform(0.002, 0.05, n)  # per-cell error of the mean of the two halves

    def iteration(shift=0.0):
        a = mu + shift + rng.normal(0.0, np.sqrt(2.0) * s)
        b = mu + shift + rng.normal(0.0, np.sqrt(2.0) * s)
        return 0.5 * (a + b), np.abs(a - b) / 2.0

    T0, s0 = iteration()
    T1, s1 = iteration()
    x = temperature_change_halves(T0, s0, T1, s1)
    assert abs(x - 2.0 * np.sqrt(2.0) / np.pi) < 0.01, x
    T2, s2 = iteration(shift=3.0 * s)
    y = temperature_change_halves(T1, s1, T2, s2)
    assert y > 2.0, y
    # cells without a temperature or a sigma in either iteration are left out
    s1_nan = s1.copy()
    s1_nan[: n // 2] = np.nan
    z = temperature_change_halves(T0, s0, T1, s1_nan)
    assert abs(z - 2.0 * np.sqrt(2.0) / np.pi) < 0.015, z
