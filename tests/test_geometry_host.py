"""The cell geometry of the transport kernels (common.cuh: next_face and d_min, with the branch-free FP32
versions; host and device code) compiled for the host with nvcc and compared with the oracle's on the
benchmark's 200 x 120 rim-refined grid, at random points inside random cells and random directions:
distance to the cell boundary and the face crossed, and d_min of Eq. 11. FP64 to 1e-12 of the radius;
FP32 to 1e-5 of the radius (positions carry 6e-8 of the radius, a near-grazing cone root a few 1e-7
relative), with the same exit face."""
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
    out = tmp_path_factory.mktemp("geom") / "libgeom.so"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_0902_3092_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "hostshim", "geom_shim.cu"), "-o", str(out)])
    L = C.CDLL(str(out))
    for f in ("next_face_f", "next_face_d", "dmin_f", "dmin_d"):
        getattr(L, f).restype = C.c_double
    return L


def test_kernel_geometry_matches_oracle(shim, oracle):
    d = disks.config_thick_gray(200, 120, 1e6)
    l = d.r_faces_cm[0]
    rf = np.ascontiguousarray(d.r_faces_cm / l)
    tf = np.ascontiguousarray(d.theta_faces)
    P = lambda a: a.ctypes.data_as(C.c_void_p)
    rng = np.random.default_rng(2)
    for _ in range(2000):
        ir, it = int(rng.integers(d.nr)), int(rng.integers(d.ntheta))
        r = (rf[ir] ** 3 + rng.random() * (rf[ir + 1] ** 3 - rf[ir] ** 3)) ** (1 / 3)
        c1, c2 = math.cos(tf[it]), math.cos(tf[it + 1])
        mu = c1 + rng.random() * (c2 - c1)
        ph, s = rng.uniform(0, 2 * math.pi), math.sqrt(1 - mu * mu)
        p = np.array([r * s * math.cos(ph), r * s * math.sin(ph), r * mu])
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        cells, lens = oracle.march(d, p * l, u, ir, it, nmax=2)
        nxt = int(cells[1]) if len(cells) > 1 else -1
        dm = oracle.dmin(d, p * l, ir, it) / l
        for f_face, f_dmin, tol, tol_d in ((shim.next_face_d, shim.dmin_d, 1e-12, 1e-13),
                                           (shim.next_face_f, shim.dmin_f, 1e-5, 1e-6)):
            face = C.c_int()
            s_k = f_face(d.nr, d.ntheta, P(rf), P(tf), ir, it, P(p), P(u), C.byref(face))
            assert abs(s_k - lens[0] / l) < tol * r
            assert abs(f_dmin(d.nr, d.ntheta, P(rf), P(tf), ir, it, P(p)) - dm) < tol_d * r
            f = face.value
            want = {0: (ir - 1) * d.ntheta + it, 1: (ir + 1) * d.ntheta + it, 2: ir * d.ntheta + it - 1,
                    3: ir * d.ntheta + it + 1}[f]
            if f == 1 and ir + 1 >= d.nr:
                want = -1
            if not (f == 0 and ir == 0):  # into the cavity: the oracle's march stops there
                assert want == nxt
