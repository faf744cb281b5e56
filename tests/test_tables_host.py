"""The tables the library's kernels read (tables.h, host code), compiled for the host and compared with
the oracle: the MRW escape-time inverse, and the dust tables on the temperature grid (built when the
opacities are set), against the oracle's exact quantities at grid temperatures from 1 K to 1e4 K: Q(T) = 4 pi sum_b kappa_b Bbar_b(T) and
its logarithmic slope; the cumulative re-emission spectrum kappa_b Bbar_b(T) (Bjorkman & Wood, Sect. 2.1)
and MRW exit spectrum dBbar_b/dT / chi'_b; chi_R = 1 / (3 rho D) with D of Eq. 12-15 and kappa_bar of
Eq. 10, both at the oracle's iterated fixed point of Eq. 13; the J weights eta_b / chi'_b normalised.
FP32 entries to 1e-6 relative (their rounding; the cumulative spectra to 1e-6 of their total, which
is what sampling from them sees), FP64 ones to 1e-12."""
import ctypes as C
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NT, TMIN, TMAX = 1024, 1.0, 1.0e4


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = tmp_path_factory.mktemp("tables") / "libtables.so"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_0902_3092_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "hostshim", "tables_shim.cu"), "-o", str(out)])
    return C.CDLL(str(out))


def tables(shim, op):
    nlam = op.nlam
    chip = np.ascontiguousarray(op.kappa_abs + (1 - op.g) * op.kappa_sca)
    f = lambda n: np.zeros(n, np.float32)
    out = dict(lQk=f(NT), cbw=f(NT * nlam), cexit=f(NT * nlam), chiR=f(NT), kbar=f(NT), jw=f(NT * nlam),
               lQ64=np.zeros(NT), slQ64=np.zeros(NT))
    P = lambda a: np.ascontiguousarray(a).ctypes.data_as(C.c_void_p)
    shim.tables_host(C.c_int(nlam), P(op.lam_edges_um), P(op.kappa_abs), P(chip), C.c_int(NT), C.c_double(TMIN),
                     C.c_double(TMAX), *(P(out[k]) for k in ("lQk", "cbw", "cexit", "chiR", "kbar", "jw", "lQ64", "slQ64")))
    for k in ("cbw", "cexit", "jw"):
        out[k] = out[k].reshape(NT, nlam)
    return out, chip


@pytest.mark.parametrize("kind", ["nongray", "gray_hg"])
def test_tables_match_oracle(shim, oracle, kind):
    if kind == "nongray":
        d = disks.config_nongray(8, 8, 100.0)
    else:
        d = disks.config_plain_gray(8, 8, 100.0)
        d.opacity = disks.gray_opacity(nlam=60, albedo=0.6, g=0.5)
    op = d.opacity
    t, chip = tables(shim, op)
    dln = math.log(TMAX / TMIN) / (NT - 2)
    for k in list(range(1, NT, 37)) + [NT - 1]:
        T = TMIN * math.exp((k - 1) * dln)
        B, dB = oracle.planck_bins(op.lam_edges_um, T), oracle.dplanck_bins(op.lam_edges_um, T)
        q = 4 * math.pi * (op.kappa_abs * B).sum()
        assert abs(t["lQ64"][k] - math.log(q)) < 1e-12 * abs(math.log(q)) + 1e-13
        assert abs(t["lQk"][k] - math.log(q)) < 2e-6 * abs(math.log(q)) + 1e-6
        h = 1e-4
        slope = (math.log((op.kappa_abs * oracle.planck_bins(op.lam_edges_um, T * math.exp(h))).sum())
                 - math.log((op.kappa_abs * oracle.planck_bins(op.lam_edges_um, T * math.exp(-h))).sum())) / (2 * h)
        assert abs(t["slQ64"][k] / slope - 1) < 1e-6
        for tab, ref in (("cbw", np.cumsum(op.kappa_abs * B)), ("cexit", np.cumsum(dB / chip))):
            assert np.all(np.abs(t[tab][k] - ref) <= 1e-6 * ref[-1]), (tab, k)  # of the CDF's total
        D, kb = oracle.diffusion(d, T, 1.0)
        assert abs(t["chiR"][k] * 3 * D - 1) < 1e-6 and abs(t["kbar"][k] / kb - 1) < 1e-6, k
        w = oracle.eta_iterate(d, T) / chip
        w /= w.sum()
        assert np.max(np.abs(t["jw"][k] - w)) < 1e-7, k
        assert abs(float(t["jw"][k].astype(np.float64).sum()) - 1) < 1e-5
    assert np.isneginf(t["lQk"][0]) and not t["cbw"][0].any()


def test_mrw_escape_time_table_matches_oracle(shim, oracle):
    """The inverse of the MRW escape-time law P(x) (Eq. 7-8) that the kernels interpolate: nodes
    u = 2^-24 .. 1/2 evenly in log u, x with P(x) = u and 1/x with P(x) = 1 - u, against the oracle's
    bisection of the series: the nodes to their FP32 rounding (1e-7), and halfway between nodes the
    kernels' linear interpolation in log u within 3e-6 of the exact inverse."""
    n = 2048
    tab = np.zeros(2 * n, np.float32)
    t0, dt = C.c_float(), C.c_float()
    assert shim.mrw_table_host(tab.ctypes.data_as(C.c_void_p), C.byref(t0), C.byref(dt)) == n
    t0, dt = np.float64(t0.value), np.float64(dt.value)
    assert abs(t0 - math.log(2.0 ** -24)) < 1e-6 and abs(t0 + (n - 1) * dt - math.log(0.5)) < 1e-4
    lo, hi = tab[:n].astype(np.float64), tab[n:].astype(np.float64)
    for frac, tol in ((0.0, 1e-7), (0.5, 3e-6)):
        i = np.arange(0, n - 1, 7)
        u = np.exp(t0 + (i + frac) * dt)
        xl = (1 - frac) * lo[i] + frac * lo[i + 1]
        xh = 1.0 / ((1 - frac) * hi[i] + frac * hi[i + 1])
        assert np.max(np.abs(xl / [oracle.mrw_x(x) for x in u] - 1)) < tol, frac
        assert np.max(np.abs(xh / [oracle.mrw_x(1 - x) for x in u] - 1)) < tol, frac


def test_pda_half_resistances_match_oracle(shim, oracle):
    """The PDA's geometric half-cell resistances (Sect. 2.2.1, exact for constant D) and cell extents on
    the rim-refined 200 x 120 grid against the oracle's: 1e-12, except the faces on the polar axis, which
    carry no flux (infinite in the library)."""
    d = disks.config_thick_gray(200, 120, 1e6)
    nr, nt = d.nr, d.ntheta
    out = [np.zeros(nr * nt) for _ in range(5)]
    P = lambda a: np.ascontiguousarray(a, np.float64).ctypes.data_as(C.c_void_p)
    shim.half_resistances_host(nr, nt, P(d.r_faces_cm), P(d.theta_faces), *(P(x) for x in out))
    hi, ho, tl, th, el = (x.reshape(nr, nt) for x in out)
    ri, ro, rl, rh = oracle.half_resistances(d.r_faces_cm, d.theta_faces)
    for got, want in ((hi, ri), (ho, ro), (tl[:, 1:], rl[:, 1:]), (th[:, :-1], rh[:, :-1])):
        assert np.max(np.abs(got / want - 1)) < 1e-12
    assert np.all(np.isinf(tl[:, 0])) and np.all(np.isinf(th[:, -1]))
    ext = oracle.cell_extent(d)
    assert np.max(np.abs(el / ext - 1)) < 1e-12
