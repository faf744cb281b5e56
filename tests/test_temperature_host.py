"""The temperature kernel's per-cell solve (temperature.cuh: cell_temperature over q_sum, the exact bin
integrals, from a Hermite guess on the library's grid tables; host and device code) compiled for the host:
for temperatures from 0.3 K to 3e4 K (below the grid's first point, on it, and beyond its end), q = Q(T)
from the oracle's Planck integrals is inverted back to T within 1e-10, and agrees with the oracle's own
inversion; non-gray dust and gray dust (closed form)."""
import ctypes as C
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = tmp_path_factory.mktemp("temperature") / "libtemperature.so"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_0902_3092_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "hostshim", "temperature_shim.cu"), "-o", str(out)])
    return C.CDLL(str(out))


@pytest.mark.parametrize("kind", ["nongray", "gray"])
def test_cell_temperature_inverts_Q(lib, oracle, kind):
    d = disks.config_nongray(8, 8, 100.0) if kind == "nongray" else disks.config_plain_gray(8, 8, 100.0)
    op = d.opacity
    rng = np.random.default_rng(5)
    T_true = np.concatenate([np.exp(rng.uniform(math.log(0.3), math.log(3e4), 150)), [0.5, 1.0, 1.0 + 1e-9, 9999.0, 2e4]])
    q = np.array([4 * math.pi * (op.kappa_abs * oracle.planck_bins(op.lam_edges_um, t)).sum() for t in T_true])
    P = lambda a: np.ascontiguousarray(a, np.float64).ctypes.data_as(C.c_void_p)
    T = np.zeros(len(q))
    lib.host_temperatures(op.nlam, P(op.lam_edges_um), P(op.kappa_abs), P(op.kappa_sca), P(op.g),
                          C.c_double(d.star.T_K), len(q), P(q), P(T))
    assert np.max(np.abs(T / T_true - 1)) < 1e-10
    To = np.array([oracle.T_of_q(d, x) for x in q[::10]])
    assert np.max(np.abs(T[::10] / To - 1)) < 1e-10


def test_rosseland_mean_matches_oracle(lib, oracle):
    """The Rosseland mean of chi' that the PDA kernels compute per cell (planck.cuh: rosseland, Eq. 3 with
    Eq. 16) against the oracle's, non-gray dust with anisotropic scattering, 1 K - 3e4 K: 1e-12."""
    d = disks.config_nongray(8, 8, 100.0)
    op = d.opacity
    chip = np.ascontiguousarray(op.kappa_abs + (1.0 - op.g) * op.kappa_sca)
    T = np.exp(np.linspace(0.0, math.log(3e4), 60))
    P = lambda a: np.ascontiguousarray(a, np.float64).ctypes.data_as(C.c_void_p)
    out = np.zeros(len(T))
    lib.host_rosseland(op.nlam, P(op.lam_edges_um), P(chip), len(T), P(T), P(out))
    ref = np.array([oracle.rosseland_chi(d, t) for t in T])
    assert np.max(np.abs(out / ref - 1)) < 1e-12
    assert not np.allclose(ref, ref[0])  # the mean does depend on T for this dust
