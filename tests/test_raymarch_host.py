"""The ray march of the ray-tracing kernel (paper_0902_3092_gb300/csrc/raymarch.cuh: closed-form
crossings of a straight ray with the grid's spheres and cones, one root per step) compiled for the host
and compared, cell by cell, with the oracle's segments (every crossing found in closed form, sorted,
pieces assigned by midpoint). FP64 to 1e-10 of the chord; FP32 to 3e-4 of the chord except for rays
within 1e-3 of the outer radius, where sqrt(r_out^2 - b^2) itself loses FP32 precision."""
import ctypes as C
import math
import os
import subprocess

import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = tmp_path_factory.mktemp("march") / "libmarch.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I",
                           os.path.join(ROOT, "paper_0902_3092_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "hostshim", "raymarch_shim.cpp"), "-o", str(out)])
    return C.CDLL(str(out))


def _march(L, d, incl, p, q, dt):
    rf = d.r_faces_cm / d.r_faces_cm[0]
    tf = d.theta_faces
    fk = np.where(np.abs(tf - np.pi / 2) < 1e-12, 0, np.where(tf < np.pi / 2, 1, -1)).astype(np.int8)
    fk[0] = fk[-1] = 2
    rf2, c2, s2, cf = (np.ascontiguousarray(x, dt) for x in (rf * rf, np.cos(tf) ** 2, np.sin(tf) ** 2, np.cos(tf)))
    cap = 8 * (d.nr + d.ntheta) + 64
    cells, Ls = np.zeros(cap, np.int32), np.zeros(cap)
    f, T = (L.march_d, C.c_double) if dt == np.float64 else (L.march_f, C.c_float)
    P = lambda a: a.ctypes.data_as(C.c_void_p)
    l = d.r_faces_cm[0]
    m = f(d.nr, d.ntheta, P(rf2), P(c2), P(s2), P(cf), P(fk), T(p / l), T(q / l), T(math.sin(incl)),
          T(math.cos(incl)), 4 * (d.nr + d.ntheta) + 64, P(cells), P(Ls), cap)
    assert m >= 0, "event guard"
    return cells[:m], Ls[:m] * l


@pytest.mark.parametrize("which", ["thick", "nongray"])
def test_march_matches_oracle_segments(shim, oracle, which):
    from oracle import raytrace as R
    d = disks.config_thick_gray(60, 40, 1e5) if which == "thick" else disks.config_nongray(20, 16, 1e3)
    rf = d.r_faces_cm
    rng = np.random.default_rng(7)
    n = d.nr * d.ntheta
    for k in range(300):
        incl = [0.0, math.pi, math.pi / 2, rng.uniform(0, math.pi)][k % 4]
        b = rf[-1] * min(rng.uniform(0, 1) ** 2, 0.9995)
        phi = rng.uniform(0, 2 * math.pi)
        p, q = b * math.cos(phi), b * math.sin(phi)
        oc, oL = R.segments(d, incl, p, q)
        ref = np.bincount(oc, weights=oL, minlength=n)
        chord = max(oL.sum(), 1e-300)
        for dt, tol in ((np.float64, 1e-10), (np.float32, 3e-4)):
            if dt == np.float32 and b > 0.999 * rf[-1]:
                continue
            cells, L = _march(shim, d, incl, p, q, dt)
            got = np.bincount(cells, weights=L, minlength=n)
            assert np.max(np.abs(got - ref)) <= tol * chord, (k, incl, b / rf[-1], dt)
