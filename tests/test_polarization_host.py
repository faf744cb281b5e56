"""The polarization functions of the transport kernels (transport.cuh: pol_scatter, pol_observer; host
and device code), with the sampling table of the scattering angle that mcrt_set_mueller builds
(tables.h), compiled for the host with nvcc and compared with the oracle's on random packets, for
the exact Rayleigh matrix and a polarized Henyey-Greenstein matrix: FP64 to 1e-11, FP32 to 2e-5 (float
rounding of the geometry and of the table interpolation, ~1e-6, and the FP32 Newton tolerance of the
plane azimuth, 1e-6, which moves the direction and the Stokes vector by a few 1e-6)."""
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
def shim(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = tmp_path_factory.mktemp("polar") / "libpolar.so"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_0902_3092_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "hostshim", "polar_shim.cu"), "-o", str(out)])
    return C.CDLL(str(out))


@pytest.mark.parametrize("which", ["rayleigh", "hg"])
def test_kernel_polarization_functions_match_oracle(shim, oracle, which):
    tab = disks.rayleigh_mueller(1, 181)[0] if which == "rayleigh" else disks.hg_polarized_mueller([0.5], [0.6], 181)[0]
    t = np.ascontiguousarray(tab)
    P = lambda a: a.ctypes.data_as(C.c_void_p)
    rng = np.random.default_rng(1)
    for k in range(500):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        e = np.cross(u, rng.normal(size=3))
        e /= np.linalg.norm(e)
        p, ang = rng.uniform(0, 1), rng.uniform(0, math.pi)
        st = np.array([p * math.cos(2 * ang), p * math.sin(2 * ang), 0.0]) if k % 2 else np.zeros(3)
        w1, w2 = rng.random(2)
        uo, eo, so = oracle.pol_scatter(t, u, e, st, w1, w2)
        qo, uuo = oracle.pol_observer(uo, eo, so)
        for f, g, tol in ((shim.pol_scatter_d, shim.pol_observer_d, 1e-11), (shim.pol_scatter_f, shim.pol_observer_f, 2e-5)):
            uu, ee, ss = u.copy(), e.copy(), st.copy()
            f(C.c_int(181), P(t), P(uu), P(ee), P(ss), C.c_double(w1), C.c_double(w2))
            assert np.abs(uu - uo).max() < tol and np.abs(ee - eo).max() < tol and np.abs(ss - so).max() < tol, (k, tol)
            q, qu = C.c_double(), C.c_double()
            g(P(uo), P(eo), P(so), C.byref(q), C.byref(qu))
            assert abs(q.value - qo) < tol and abs(qu.value - uuo) < tol
