"""The C-ABI library builds, loads and exports every function that include/mcrt.h declares, and the
ctypes structs have the C layout. No compute calls: these run without a GPU."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mcrt.h")


@pytest.fixture(scope="module")
def L():
    from paper_0902_3092_gb300 import build, mcrt
    build.build()
    return mcrt.lib()


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mcrt_[a-z_0-9]+)\s*\(", src)))


def test_all_declared_symbols_exported(L):
    names = declared()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", L._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (mcrt_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    from paper_0902_3092_gb300 import mcrt
    assert sorted(mcrt.EXPORTS) == names


def test_struct_layouts_match_c(L, tmp_path):
    import ctypes as C

    from paper_0902_3092_gb300 import mcrt
    prog = tmp_path / "sz.c"
    prog.write_text('#include "mcrt.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                    'sizeof(mcrt_grid),sizeof(mcrt_star),sizeof(mcrt_run_opts),sizeof(mcrt_run_stats),sizeof(mcrt_pda_opts),'
                    'offsetof(mcrt_run_stats,seconds),offsetof(mcrt_pda_opts,kappa_R),sizeof(mcrt_hydro_opts),'
                    'offsetof(mcrt_hydro_opts,shell_mass_g),offsetof(mcrt_run_stats,guard_cell),'
                    'offsetof(mcrt_run_stats,guard_dir));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(mcrt.Grid), C.sizeof(mcrt.Star), C.sizeof(mcrt.RunOpts), C.sizeof(mcrt.RunStats),
            C.sizeof(mcrt.PdaOpts), mcrt.RunStats.seconds.offset, mcrt.PdaOpts.kappa_R.offset,
            C.sizeof(mcrt.HydroOpts), mcrt.HydroOpts.shell_mass_g.offset, mcrt.RunStats.guard_cell.offset,
            mcrt.RunStats.guard_dir.offset]
    assert got == want


def test_defaults_and_host_validation(L):
    import ctypes as C

    from paper_0902_3092_gb300 import mcrt
    o = mcrt.RunOpts()
    L.mcrt_default_run_opts(C.byref(o))
    assert o.precision == 32 and o.mrw_min_interactions == 20 and o.gamma == 2.0 and o.want_sed == 1
    p = mcrt.PdaOpts()
    L.mcrt_default_pda_opts(C.byref(p))
    assert p.min_visits == 30 and p.max_rel_err == 0.05
    h = mcrt.HydroOpts()
    L.mcrt_default_hydro_opts(C.byref(h))
    assert h.mu == 2.3 and abs(h.M_star_g / 1.98892e33 - 2.5) < 1e-12 and h.which == mcrt.T_PDA
    # invalid input is rejected on the host before any device work
    h = C.c_void_p()
    assert L.mcrt_disk_create(None, None, 0, None, C.byref(h)) == 1
    assert b"NULL" in L.mcrt_last_error(None)
    assert L.mcrt_set_rays(None, 0.5, 1e20, 1, None, None, None) == 1
    assert L.mcrt_raytrace(None, 0, 32, None, None, None, None) == 1
    assert L.mcrt_visibilities(None, 1, None, None, None, 1, None) == 1
    assert L.mcrt_set_sources(None, None) == 1
    assert L.mcrt_set_mueller(None, 181, None) == 1
    assert L.mcrt_sed_stokes(None, 10, None, None, None) == 1
    assert L.mcrt_keep_mean_intensity(None, 1) == 1
    assert L.mcrt_mean_intensity(None, None) == 1
    L.mcrt_disk_destroy(None)


def test_binding_fails_loudly_without_library(monkeypatch):
    from paper_0902_3092_gb300 import mcrt
    monkeypatch.setattr(mcrt, "_lib", None)
    monkeypatch.setattr(mcrt, "LIB_PATH", "/nonexistent/libmcrt.so")
    with pytest.raises(RuntimeError):
        mcrt.lib()


def test_disk_create_validates_on_the_host(L):
    """mcrt_disk_create checks the grid and star before it touches a device: each bad input gives
    MCRT_EINVAL and a message naming it; a valid one gets past the checks (here MCRT_ECUDA without a
    device, or a disk on a GPU machine)."""
    import ctypes as C
    import math

    import numpy as np

    from paper_0902_3092_gb300 import mcrt
    rf0 = np.array([1e13, 2e13, 4e13])
    tf0 = np.array([0.0, math.pi / 2, math.pi])
    rho0 = np.full(4, 1e-15)

    def create(rf=rf0, tf=tf0, rho=rho0, T=5000.0, R=1e11, nr=2, nt=2):
        rf, tf, rho = (np.ascontiguousarray(x, np.float64) for x in (rf, tf, rho))
        p = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        g = mcrt.Grid(nr, nt, p(rf), p(tf), p(rho))
        s = mcrt.Star(T, R)
        h = C.c_void_p()
        st = L.mcrt_disk_create(C.byref(g), C.byref(s), 0, None, C.byref(h))
        if st == 0:
            L.mcrt_disk_destroy(h)
        return st, (L.mcrt_last_error(None) or b"").decode()

    st, _ = create()
    assert st in (0, 3)
    bad = [(dict(rf=[1e13, 1e13, 4e13]), "r_faces"), (dict(rf=[-1.0, 2e13, 4e13]), "r_faces"),
           (dict(rf=[1e13, math.nan, 4e13]), "r_faces"), (dict(tf=[0.1, math.pi / 2, math.pi]), "0 to pi"),
           (dict(tf=[0.0, math.pi / 2, 3.0]), "0 to pi"), (dict(tf=[0.0, 0.0, math.pi]), "theta_faces"),
           (dict(rho=[1e-15, -1.0, 0.0, 0.0]), "rho"), (dict(rho=[1e-15, math.inf, 0.0, 0.0]), "rho"),
           (dict(T=0.0), "star"), (dict(R=math.inf), "star"), (dict(nr=0), "grid sizes")]
    for kw, word in bad:
        st, msg = create(**kw)
        assert st == 1 and word in msg, (kw, st, msg)
