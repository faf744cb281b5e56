"""The ray tracer's source function and the mean-intensity read-out (source.cuh: k_source,
k_mean_intensity; host and device code) compiled for the host and fed the oracle's path lengths of a
Monte Carlo run of non-gray, scattering dust: J equal to the oracle's mean intensity to 1e-13, and the
source function, thermal kappa Bbar(T) / chi plus the scattered sigma J / chi, equal to the oracle's to
1e-12 in FP64 and to FP32 rounding (2e-7 of each bin's largest value; 0 below FP32's smallest normal)
in FP32, with and without the scattered light."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if not shutil.which("g++") or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers not found")
    out = tmp_path_factory.mktemp("source") / "libhostsource.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I", CUDA_INC,
                           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_0902_3092_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "hostshim", "source_shim.cpp"), "-o", str(out)])
    return C.CDLL(str(out))


def test_mean_intensity_and_source_match_oracle(lib, oracle):
    from oracle import raytrace as R
    d = disks.config_nongray(10, 8, 30.0)
    op = d.opacity
    n = 20_000
    ref = oracle.Run(d).run(n, seed=6, want_j=True)
    Jo = ref.mean_intensity()
    T, _ = ref.temperatures()
    P = lambda a: None if a is None else np.ascontiguousarray(a, np.float64).ctypes.data_as(C.c_void_p)
    jlen = np.ascontiguousarray(ref.jtally / d.r_faces_cm[0])  # cm -> the library's internal length unit
    Lpkt = ref.packet_lum
    nc = d.nr * d.ntheta
    J = np.zeros(nc * op.nlam)
    lib.host_mean_intensity(d.nr, d.ntheta, op.nlam, P(d.r_faces_cm), P(d.theta_faces), P(jlen), C.c_double(Lpkt),
                            C.c_double(n), P(J))
    J = J.reshape(Jo.shape)
    assert Jo.max() > 0 and np.all(np.abs(J - Jo) <= 1e-13 * np.abs(Jo))
    for with_j in (True, False):
        want = R.source(d, T, J=Jo if with_j else None)
        for prec, tol in ((64, 1e-12), (32, 2e-7)):
            S = np.zeros(nc * op.nlam)
            lib.host_source(d.nr, d.ntheta, op.nlam, P(d.r_faces_cm), P(d.theta_faces), P(T.ravel()),
                            P(op.lam_edges_um), P(op.kappa_abs), P(op.kappa_sca), P(op.g), C.c_double(d.star.T_K),
                            P(jlen if with_j else None), C.c_double(Lpkt), C.c_double(n), C.c_int(prec), P(S))
            S = S.reshape(want.shape)
            if prec == 32:  # of each bin's largest value; values below FP32's smallest normal become 0
                bound = tol * np.abs(want).max(axis=0, keepdims=True) + 1.2e-38
            else:
                bound = tol * np.abs(want)
            assert np.all(np.abs(S - want) <= bound), (with_j, prec)
