"""The Planck bin integrals of the library (planck.cuh, host and device code; the temperature, source-
function and Rosseland kernels use them) compiled for the host and compared with the oracle's own
series: every bin holding more than 1e-10 of the total to 2e-12 relative, and the sums over the bins
to 1e-14, from 2 K to 3e4 K on the benchmark's 100 bins."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = tmp_path_factory.mktemp("planck") / "libplanck.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I",
                           os.path.join(ROOT, "paper_0902_3092_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "hostshim", "planck_shim.cpp"), "-o", str(out)])
    return C.CDLL(str(out))


def test_planck_bins_match_oracle(shim, oracle):
    lam = disks.lam_edges(100)
    n = len(lam) - 1
    P = lambda a: a.ctypes.data_as(C.c_void_p)
    for T in np.geomspace(2.0, 3e4, 120):
        B, dB = np.zeros(n), np.zeros(n)
        shim.planck_bins_host(P(lam), C.c_int(n), C.c_double(T), P(B), P(dB))
        Bo, dBo = oracle.planck_bins(lam, T), oracle.dplanck_bins(lam, T)
        for x, y in ((B, Bo), (dB, dBo)):
            big = y > 1e-10 * y.sum()
            assert np.max(np.abs(x[big] / y[big] - 1)) < 2e-12, T
            assert abs(x.sum() / y.sum() - 1) < 1e-14, T
