"""The wavelength sampling of the transport kernels (transport.cuh: qpos, sample_bw, sample_exit,
sample_star; host and device code) compiled for the host over the library's own temperature-grid
tables, and its distributions compared with the exact spectra of the oracle (non-gray dust): the
launch bin against the stellar spectrum, the MRW exit bin against dBbar_b/dT / chi'_b (Sect. 2.2.2), and
the re-emission bin after an absorption against kappa_b [Bbar_b(T_new) - Bbar_b(T_old)] (Bjorkman &
Wood, Sect. 2.1). Each distribution is read off 20000 evenly spaced uniforms (resolution 5e-5).
Bounds: launch and exit CDFs 1.5e-4 (tables interpolated in log T); re-emission 3e-4 when the two
temperatures lie in different grid intervals, and 1.5e-3 when both lie in one interval (1 % apart at
most: the library interpolates the derivative spectrum at the pair's position between the difference
spectra C(T_k+1) - C(T_k) of that interval and its neighbour, second order in the grid spacing
dlnT = 0.009; measured 1e-4 for steps of 1e-5-1e-3 in T, 1.3e-3 for a step of a third of an interval;
the interval's own difference spectrum alone, first order, is 3.4e-3 off)."""
import ctypes as C
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
US = (np.arange(20000) + 0.5) / 20000


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = tmp_path_factory.mktemp("sampling") / "libsampling.so"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_0902_3092_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "hostshim", "sampling_shim.cu"), "-o", str(out)])
    L = C.CDLL(str(out))
    L.star_bin_host.argtypes = [C.c_double]
    L.bw_bin_host.argtypes = [C.c_ulonglong, C.c_ulonglong, C.c_float]
    L.exit_bin_host.argtypes = [C.c_ulonglong, C.c_float]
    return L


def _cdf(nl, draw):
    b = np.sort([draw(u) for u in US])
    return np.searchsorted(b, np.arange(nl), side="right") / len(US)


def test_sampled_bins_follow_exact_spectra(lib, oracle):
    d = disks.config_nongray(8, 8, 100.0)
    op = d.opacity
    nl = op.nlam
    P = lambda a: np.ascontiguousarray(a, np.float64).ctypes.data_as(C.c_void_p)
    chip = op.kappa_abs + (1 - op.g) * op.kappa_sca
    Q = lambda T: 4 * math.pi * (op.kappa_abs * oracle.planck_bins(op.lam_edges_um, T)).sum()
    lq_run = math.log(Q(2000.0)) - 62 * math.log(2)  # tallies up to 2^62 at 2000 K
    star = np.cumsum(oracle.planck_bins(op.lam_edges_um, d.star.T_K))
    lib.sampling_setup(nl, P(op.lam_edges_um), P(op.kappa_abs), P(chip), 1024, C.c_double(1.0),
                       C.c_double(max(1e4, 2 * d.star.T_K)), P(star), C.c_float(lq_run))
    tally = lambda T: int(round(math.exp(math.log(Q(T)) - lq_run)))
    assert np.max(np.abs(_cdf(nl, lib.star_bin_host) - star / star[-1])) < 1.5e-4
    for T in (30.0, 150.0, 600.0, 1500.0):
        p = oracle.dplanck_bins(op.lam_edges_um, T) / chip
        F = np.cumsum(p) / p.sum()
        assert np.max(np.abs(_cdf(nl, lambda u: lib.exit_bin_host(tally(T), u)) - F)) < 1.5e-4, T
    for T_old, ratio, tol in ((50.0, 1.001, 1.5e-3), (50.0, 1.0001, 1.5e-3), (300.0, 1.00001, 1.5e-3),
                              (300.0, 1.003, 1.5e-3), (123.4, 1.0002, 1.5e-3), (777.7, 1.0005, 1.5e-3),
                              (300.0, 1.02, 3e-4), (800.0, 1.1, 3e-4), (1200.0, 2.0, 3e-4), (100.0, 5.0, 3e-4)):
        T_new = T_old * ratio
        p = op.kappa_abs * (oracle.planck_bins(op.lam_edges_um, T_new) - oracle.planck_bins(op.lam_edges_um, T_old))
        F = np.cumsum(p) / p.sum()
        dev = np.max(np.abs(_cdf(nl, lambda u: lib.bw_bin_host(tally(T_old), tally(T_new), u)) - F))
        assert dev < tol, (T_old, ratio, dev)


def test_kernel_mrw_escape_time_matches_oracle(lib, oracle):
    """The kernels' MRW escape-time lookup (mrw_x over the library's table, Eq. 7-8), FP32 and FP64, at
    uniforms on the kernels' 2^-23 grid (where 1 - u is exact): within 1e-5 of the oracle's inverse of
    P(x), including both tails, the switch of tables at u = 1/2 and the grid's end points (measured
    5.9e-6, at u = 1/2, where the index clamp keeps 1e-3 of an interval)."""
    lib.mrw_x_host.restype = C.c_double
    lib.mrw_x_host.argtypes = [C.c_double, C.c_int]
    rng = np.random.default_rng(2)
    k = np.concatenate([rng.integers(0, 2 ** 23, 400), np.arange(0, 30), 2 ** 23 - 1 - np.arange(0, 30),
                        [2 ** 22 - 1, 2 ** 22]])
    u = (k + 0.5) / 2 ** 23
    ref = np.array([oracle.mrw_x(x) for x in u])
    for prec in (32, 64):
        x = np.array([lib.mrw_x_host(float(v), prec) for v in u])
        assert np.max(np.abs(x / ref - 1)) < 1e-5, prec
