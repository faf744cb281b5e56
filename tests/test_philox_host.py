"""Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011), the counter-based generator that both sides draw
every random number from: the oracle's (plain C) and the transport kernels' (common.cuh, host build)
against an independent implementation, Triton's tl.philox run by its CPU interpreter, on random
counters and keys including the all-zero and all-ones words. Bit-exact."""
import ctypes as C
import json
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = 16

_TRITON = r'''
import json, sys
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(c0p, c1p, c2p, c3p, k0p, k1p, o0, o1, o2, o3, N: tl.constexpr):
    i = tl.arange(0, N)
    seed = (tl.load(k1p + i).to(tl.uint32).to(tl.uint64) << 32) | tl.load(k0p + i).to(tl.uint32).to(tl.uint64)
    a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i), 10)
    tl.store(o0 + i, a)
    tl.store(o1 + i, b)
    tl.store(o2 + i, c)
    tl.store(o3 + i, d)

x = np.array(json.loads(sys.stdin.read()), dtype=np.uint64)  # rows c0 c1 c2 c3 k0 k1
n = x.shape[1]
t = [torch.tensor(r.astype(np.uint32).view(np.int32)) for r in x]
o = [torch.zeros(n, dtype=torch.int32) for _ in range(4)]
k[(1,)](*t, *o, N=n)
print(json.dumps([[int(v) & 0xFFFFFFFF for v in r.tolist()] for r in o]))
'''


def test_philox_matches_independent_implementation(oracle, tmp_path):
    pytest.importorskip("triton")
    rng = np.random.default_rng(11)
    x = rng.integers(0, 2 ** 32, (6, N), dtype=np.uint64)
    x[:, 0] = 0
    x[:, 1] = 0xFFFFFFFF
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _TRITON], input=json.dumps(x.tolist()), capture_output=True,
                       text=True, env=env, timeout=600)
    if r.returncode != 0:
        pytest.skip("Triton's CPU interpreter is not available: " + r.stderr.strip().splitlines()[-1])
    ref = np.array(json.loads(r.stdout.strip().splitlines()[-1]), dtype=np.uint64)
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    lib = None
    if os.path.exists(nvcc):
        so = tmp_path / "libphilox.so"
        subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                               "-I", os.path.join(ROOT, "paper_0902_3092_gb300", "csrc"),
                               os.path.join(ROOT, "tests", "hostshim", "philox_shim.cu"), "-o", str(so)])
        lib = C.CDLL(str(so))
    for j in range(N):
        ctr, key = [int(v) for v in x[:4, j]], [int(v) for v in x[4:, j]]
        want = [int(v) for v in ref[:, j]]
        assert list(oracle.philox(ctr, key)) == want, j
        if lib is not None:
            out = (C.c_uint * 4)()
            lib.philox_host((C.c_uint * 4)(*ctr), (C.c_uint * 2)(*key), out)
            assert list(out) == want, j
