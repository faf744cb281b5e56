"""Plain FP64 CPU oracle for the transport + MRW + PDA path of Min et al. 2009.

TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
benchmark's CPU-baseline leg use this module. It shares no code with the CUDA
library: the Monte Carlo part is the plain C file next to this one (compiled
with `build()`), the diffusion part is numpy/scipy below.

Sections, equations and the readings taken where the paper is silent:

* Transport, BW re-emission, MRW: Sect. 2.1, 2.2.2 (Eq. 5-11), see mcrt_oracle.c.
* Diffusion coefficient and mean opacities: Sect. 2.2.3 (Eq. 12-16).
* PDA: Sect. 2.2.1, Eq. 4 -- div(D grad T^4) = 0 in the cells that fewer than 30
  packets entered or whose statistical temperature error exceeds 5 % (Sect. 3.1),
  with the Monte Carlo temperatures of all other cells as Dirichlet values. Reading:
  only optically thick cells take part (the diffusion equation is used "in regions of
  high optical depth", Sect. 2.2.1); see pda_mask.
  Discretisation (a reading; the paper gives none): finite volumes on the (r, theta)
  cells, face conductance = series resistance of the two half cells, exact for
  piecewise-constant D in spherical geometry; zero flux through grid edges and
  into cells without dust. D = 1/(3 rho chi_R) (Eq. 2), frozen at the Monte Carlo
  temperature so the system is linear.
* Adjoint of the PDA solve: derivative of J = sum_i w_i T_i with respect to
  log rho_i and kappa_R,i (the Rosseland mean entering D), with the Monte Carlo
  boundary temperatures held fixed.
* Internal sources (viscous heating, Sect. 5) and polarized transport with a full
  Mueller matrix per scattering (Sect. 2.3): see mcrt_oracle.c; ray-traced
  observables: raytrace.py; vertical structure: hydro.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mcrt_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

EUNIT = 65536
NINC = 10
SIGMA_SB = 2 * 3.141592653589793 ** 5 * 1.380649e-16 ** 4 / (15 * 6.62607015e-27 ** 3 * 2.99792458e10 ** 2)
EV_NAMES = ["launch", "cross", "scatter", "absorb", "mrw", "escape", "capped"]


def build(force: bool = False) -> str:
    """Compile the C oracle (plain gcc, no FP contraction so x86 and Arm agree)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread",
               "-o", LIB, SRC, "-lm"]
        subprocess.check_call(cmd)
    return LIB


_lib = None


class _Model(C.Structure):
    _fields_ = [("nr", C.c_int), ("nt", C.c_int), ("nlam", C.c_int),
                ("rf", C.POINTER(C.c_double)), ("tf", C.POINTER(C.c_double)), ("rho", C.POINTER(C.c_double)),
                ("lam_e", C.POINTER(C.c_double)), ("kabs", C.POINTER(C.c_double)),
                ("ksca", C.POINTER(C.c_double)), ("g", C.POINTER(C.c_double)),
                ("Tstar", C.c_double), ("Rstar", C.c_double), ("Lsrc", C.POINTER(C.c_double)),
                ("mueller", C.POINTER(C.c_double)), ("nmu", C.c_int)]


class _Opts(C.Structure):
    _fields_ = [("mrw", C.c_int), ("gamma", C.c_double), ("nmin", C.c_int), ("max_events", C.c_uint64),
                ("want_sed", C.c_int), ("mrw_exit_dir", C.c_int)]


class _State(C.Structure):
    _fields_ = [("tally", C.POINTER(C.c_uint64)), ("visits", C.POINTER(C.c_uint64)),
                ("nabs", C.POINTER(C.c_uint64)), ("sed", C.POINTER(C.c_uint64)),
                ("sed_q", C.POINTER(C.c_int64)), ("sed_u", C.POINTER(C.c_int64)),
                ("Tcell", C.POINTER(C.c_double)), ("cnt", C.c_uint64 * 10),
                ("trace_packets", C.c_int), ("trace_max", C.c_int),
                ("tr_type", C.POINTER(C.c_int32)), ("tr_cell", C.POINTER(C.c_int32)),
                ("tr_lam", C.POINTER(C.c_int32)), ("tr_n", C.POINTER(C.c_int32)),
                ("tr_pos", C.POINTER(C.c_double)), ("jtally", C.POINTER(C.c_double)),
                ("sed_sca", C.POINTER(C.c_uint64))]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        d, pd = C.c_double, C.POINTER(C.c_double)
        L.oracle_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.oracle_uniforms.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_int, pd]
        L.oracle_G3.restype = d; L.oracle_G3.argtypes = [d]
        L.oracle_G4.restype = d; L.oracle_G4.argtypes = [d]
        L.oracle_planck_bins.argtypes = [pd, C.c_int, d, pd]
        L.oracle_dplanck_bins.argtypes = [pd, C.c_int, d, pd]
        L.oracle_T_of_q.restype = d; L.oracle_T_of_q.argtypes = [C.POINTER(_Model), d]
        L.oracle_temperatures.argtypes = [C.POINTER(_Model), C.POINTER(C.c_uint64), d, pd, pd]
        L.oracle_eta_iterate.argtypes = [C.POINTER(_Model), d, C.c_int, pd]
        L.oracle_diffusion.argtypes = [C.POINTER(_Model), d, d, pd, pd]
        L.oracle_mrw_P.restype = d; L.oracle_mrw_P.argtypes = [d]
        L.oracle_mrw_x.restype = d; L.oracle_mrw_x.argtypes = [d]
        L.oracle_dmin.restype = d; L.oracle_dmin.argtypes = [C.POINTER(_Model), pd, C.c_int, C.c_int]
        L.oracle_run.restype = C.c_int
        L.oracle_run.argtypes = [C.POINTER(_Model), C.POINTER(_Opts), C.POINTER(_State), C.c_uint64, C.c_uint64,
                                 C.c_uint64, C.c_uint64, C.c_uint32]
        L.oracle_run_par.restype = C.c_int
        L.oracle_run_par.argtypes = [C.POINTER(_Model), C.POINTER(_Opts), C.POINTER(_State), C.c_uint64, C.c_uint64,
                                     C.c_uint64, C.c_uint64, C.c_uint32, C.c_int]
        L.oracle_star_bin.restype = C.c_int; L.oracle_star_bin.argtypes = [C.POINTER(_Model), d]
        L.oracle_packet_lum.restype = d; L.oracle_packet_lum.argtypes = [C.POINTER(_Model)]
        L.oracle_pol_sample_theta.restype = d; L.oracle_pol_sample_theta.argtypes = [pd, C.c_int, d]
        L.oracle_pol_sample_phi.restype = d; L.oracle_pol_sample_phi.argtypes = [d, d, d, d]
        L.oracle_pol_scatter.argtypes = [pd, C.c_int, pd, pd, pd, d, d]
        L.oracle_pol_observer.argtypes = [pd, pd, pd, pd, pd]
        for f in ("oracle_cone_exit",):
            getattr(L, f).restype = d
            getattr(L, f).argtypes = [pd, pd, d, C.c_int]
        for f in ("oracle_sphere_far", "oracle_sphere_near"):
            getattr(L, f).restype = d
            getattr(L, f).argtypes = [pd, pd, d]
        L.oracle_hg_mu.restype = d; L.oracle_hg_mu.argtypes = [d, d]
        L.oracle_march.restype = C.c_int
        L.oracle_march.argtypes = [C.POINTER(_Model), pd, pd, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int32), pd]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _up(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


class Model:
    """Holds the arrays of a disk (keeps them alive for the C side)."""

    def __init__(self, disk, sources=None, mueller=None):
        self.disk = disk
        self.rf = np.ascontiguousarray(disk.r_faces_cm, np.float64)
        self.tf = np.ascontiguousarray(disk.theta_faces, np.float64)
        self.rho = np.ascontiguousarray(disk.rho, np.float64).ravel()
        op = disk.opacity
        self.lam_e = np.ascontiguousarray(op.lam_edges_um, np.float64)
        self.kabs = np.ascontiguousarray(op.kappa_abs, np.float64)
        self.ksca = np.ascontiguousarray(op.kappa_sca, np.float64)
        self.g = np.ascontiguousarray(op.g, np.float64)
        self.nr, self.nt, self.nlam = disk.nr, disk.ntheta, op.nlam
        # internal source luminosity per cell (erg/s; viscous heating), or none
        self.Lsrc = None if sources is None else np.ascontiguousarray(sources, np.float64).ravel()
        # Mueller matrix per bin for polarized transport: (nlam, 4, nmu) = S11, S12, S33, S34 on
        # theta_k = k pi / (nmu - 1), or none
        self.mueller = None if mueller is None else np.ascontiguousarray(mueller, np.float64)
        nmu = 0 if self.mueller is None else self.mueller.shape[-1]
        self.c = _Model(self.nr, self.nt, self.nlam, _dp(self.rf), _dp(self.tf), _dp(self.rho), _dp(self.lam_e),
                        _dp(self.kabs), _dp(self.ksca), _dp(self.g), disk.star.T_K, disk.star.R_cm,
                        None if self.Lsrc is None else _dp(self.Lsrc),
                        None if self.mueller is None else _dp(self.mueller), nmu)

    @property
    def ptr(self):
        return C.byref(self.c)


class Run:
    """Tallies of an oracle Monte Carlo run (may be continued: resume). sources: luminosity (erg/s) of
    internal sources per cell (viscous heating), released by absorption-like events (see mcrt_oracle.c)."""

    def __init__(self, disk, sources=None, mueller=None):
        self.model = Model(disk, sources, mueller)
        n = self.model.nr * self.model.nt
        self.tally = np.zeros(n, np.uint64)
        self.visits = np.zeros(n, np.uint64)
        self.nabs = np.zeros(n, np.uint64)
        self.sed = np.zeros(self.model.nlam * NINC, np.uint64)
        self.jtally = None
        self.sed_sca = np.zeros(self.model.nlam * NINC, np.uint64)
        self.sed_q = np.zeros(self.model.nlam * NINC, np.int64)
        self.sed_u = np.zeros(self.model.nlam * NINC, np.int64)
        self.Tcell = np.zeros(n, np.float64)
        self.counters = np.zeros(10, np.uint64)
        self.trace = None

    def run(self, n_packets, seed=1, first_id=0, n_total=None, mrw=False, gamma=2.0, nmin=20,
            max_events=10 ** 9, want_sed=True, mrw_exit_dir=0, model_id=0, trace_packets=0, trace_max=0,
            want_j=False, threads=1):
        """want_j: keep the path-length estimator of the mean intensity (see mean_intensity). threads > 1:
        the packets on that many host threads (shared atomic energy tallies; no trace or J tally; gray
        runs give the serial tallies, counts and escapes per inclination bit for bit, non-gray runs the
        same method with the re-emission temperatures of each deposit's own tally value)."""
        L = lib()
        opts = _Opts(int(mrw), float(gamma), int(nmin), int(max_events), int(want_sed), int(mrw_exit_dir))
        st = _State()
        st.tally, st.visits, st.nabs, st.sed = _up(self.tally), _up(self.visits), _up(self.nabs), _up(self.sed)
        st.sed_q = self.sed_q.ctypes.data_as(C.POINTER(C.c_int64))
        st.sed_u = self.sed_u.ctypes.data_as(C.POINTER(C.c_int64))
        st.Tcell = _dp(self.Tcell)
        if want_j and self.jtally is None:
            self.jtally = np.zeros(self.model.nr * self.model.nt * self.model.nlam)
        if self.jtally is not None:
            st.jtally = _dp(self.jtally)
        st.sed_sca = _up(self.sed_sca)
        for i in range(10):
            st.cnt[i] = int(self.counters[i])
        tr = None
        if trace_packets:
            tr = dict(type=np.full((trace_packets, trace_max), -1, np.int32),
                      cell=np.full((trace_packets, trace_max), -1, np.int32),
                      lam=np.full((trace_packets, trace_max), -1, np.int32),
                      n=np.zeros(trace_packets, np.int32),
                      pos=np.zeros((trace_packets, trace_max, 3), np.float64))
            st.trace_packets, st.trace_max = trace_packets, trace_max
            st.tr_type, st.tr_cell, st.tr_lam = _ip(tr["type"]), _ip(tr["cell"]), _ip(tr["lam"])
            st.tr_n, st.tr_pos = _ip(tr["n"]), _dp(tr["pos"])
        n_total = n_packets if n_total is None else n_total
        if threads > 1:
            if trace_packets or self.jtally is not None:
                raise ValueError("a packet-parallel run keeps no trace and no mean-intensity tally")
            rc = L.oracle_run_par(self.model.ptr, C.byref(opts), C.byref(st), int(n_packets), int(first_id),
                                  int(n_total), int(seed), int(model_id), int(threads))
            if rc != 0:
                raise RuntimeError("oracle_run_par failed")
        else:
            L.oracle_run(self.model.ptr, C.byref(opts), C.byref(st), int(n_packets), int(first_id), int(n_total),
                         int(seed), int(model_id))
        self.counters = np.array([st.cnt[i] for i in range(10)], np.uint64)
        self.trace = tr
        self.n_total = n_total
        return self

    @property
    def stats(self):
        k = ["packets", "events", "absorptions", "scatterings", "crossings", "mrw_jumps", "capped", "escaped",
             "deposit_sum", "error_flags"]
        return {a: int(b) for a, b in zip(k, self.counters)}

    def temperatures(self):
        L = lib()
        n = self.model.nr * self.model.nt
        T = np.zeros(n)
        e = np.zeros(n)
        L.oracle_temperatures(self.model.ptr, _up(self.tally), float(self.n_total), _dp(T), _dp(e))
        return T.reshape(self.model.nr, self.model.nt), e.reshape(self.model.nr, self.model.nt)

    def mean_intensity(self):
        """Mean intensity per cell and bin (erg s^-1 cm^-2 sr^-1, integrated over the bin), shape
        (nr, ntheta, nlam): J = E_pkt (sum of path lengths) / (4 pi V), the path-length estimator;
        flights count in the packet's bin, an MRW walk's c t over the bins with the weights of Eq. 10
        (see mcrt_oracle.c)."""
        if self.jtally is None:
            raise ValueError("run with want_j=True")
        rf, tf = self.model.rf, self.model.tf
        V = (2 * np.pi / 3) * (rf[1:] ** 3 - rf[:-1] ** 3)[:, None] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :]
        e = self.packet_lum / self.n_total
        jt = self.jtally.reshape(self.model.nr, self.model.nt, self.model.nlam)
        return e * jt / (4 * np.pi * V[:, :, None])

    @property
    def packet_lum(self):
        """Luminosity the packets carry (erg/s): the star plus the internal sources."""
        return float(lib().oracle_packet_lum(self.model.ptr))

    def sed_stokes(self):
        """Escaped luminosity per (wavelength bin, inclination bin) as Stokes I, Q, U (erg/s) in the sky
        frame whose reference is the projected disk axis (Q > 0: polarized along it)."""
        e = self.packet_lum / self.n_total
        sh = (self.model.nlam, NINC)
        return (self.sed.reshape(sh).astype(np.float64) * e, self.sed_q.reshape(sh) / 1048576.0 * e,
                self.sed_u.reshape(sh) / 1048576.0 * e)

    def sed_scattered_lum(self):
        """Escaped luminosity of the packets that scattered at least once, per (bin, inclination), erg/s."""
        return self.sed_sca.reshape(self.model.nlam, NINC).astype(np.float64) * self.packet_lum / self.n_total

    def sed_lum(self):
        """Escaped luminosity per (wavelength bin, inclination bin), erg/s."""
        return self.sed.reshape(self.model.nlam, NINC).astype(np.float64) * self.packet_lum / self.n_total


# ----------------------------------------------------------------------------- small helpers

def philox(ctr, key):
    L = lib()
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    L.oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniforms(seed, model, packet, n):
    out = np.zeros(n)
    lib().oracle_uniforms(seed, model, packet, n, _dp(out))
    return out


def pol_sample_theta(S11, xi):
    S11 = np.ascontiguousarray(S11, np.float64)
    return float(lib().oracle_pol_sample_theta(_dp(S11), len(S11), float(xi)))


def pol_sample_phi(a, q, u, xi):
    return float(lib().oracle_pol_sample_phi(float(a), float(q), float(u), float(xi)))


def pol_scatter(table, u, e, st, w1, w2):
    """One polarized scattering (table: (4, nmu) Mueller elements of a bin); returns (u, e, st)."""
    t = np.ascontiguousarray(table, np.float64)
    u, e, st = (np.array(x, np.float64) for x in (u, e, st))
    lib().oracle_pol_scatter(_dp(t), t.shape[-1], _dp(u), _dp(e), _dp(st), float(w1), float(w2))
    return u, e, st


def pol_observer(u, e, st):
    u, e, st = (np.ascontiguousarray(x, np.float64) for x in (u, e, st))
    q, uu = C.c_double(), C.c_double()
    lib().oracle_pol_observer(_dp(u), _dp(e), _dp(st), C.byref(q), C.byref(uu))
    return q.value, uu.value


def planck_bins(lam_e, T):
    lam_e = np.ascontiguousarray(lam_e, np.float64)
    out = np.zeros(len(lam_e) - 1)
    lib().oracle_planck_bins(_dp(lam_e), len(lam_e) - 1, float(T), _dp(out))
    return out


def dplanck_bins(lam_e, T):
    lam_e = np.ascontiguousarray(lam_e, np.float64)
    out = np.zeros(len(lam_e) - 1)
    lib().oracle_dplanck_bins(_dp(lam_e), len(lam_e) - 1, float(T), _dp(out))
    return out


def mrw_P(x):
    return lib().oracle_mrw_P(float(x))


def mrw_x(P0):
    return lib().oracle_mrw_x(float(P0))


def eta_iterate(disk, T, iters=500):
    m = Model(disk)
    out = np.zeros(m.nlam)
    lib().oracle_eta_iterate(m.ptr, float(T), int(iters), _dp(out))
    return out


def diffusion(disk, T, rho):
    m = Model(disk)
    D, kb = C.c_double(), C.c_double()
    lib().oracle_diffusion(m.ptr, float(T), float(rho), C.byref(D), C.byref(kb))
    return D.value, kb.value


def T_of_q(disk, q):
    m = Model(disk)
    return lib().oracle_T_of_q(m.ptr, float(q))


def march(disk, p, u, ir, it, nmax=100000):
    """Segments (cells, lengths) of a straight ray through the grid."""
    m = Model(disk)
    pp = np.ascontiguousarray(p, np.float64)
    uu = np.ascontiguousarray(u, np.float64)
    cells = np.zeros(nmax, np.int32)
    lens = np.zeros(nmax)
    n = lib().oracle_march(m.ptr, _dp(pp), _dp(uu), int(ir), int(it), int(nmax), _ip(cells), _dp(lens))
    return cells[:n], lens[:n]


def dmin(disk, p, ir, it):
    m = Model(disk)
    pp = np.ascontiguousarray(p, np.float64)
    return lib().oracle_dmin(m.ptr, _dp(pp), int(ir), int(it))


# ----------------------------------------------------------------------------- PDA (Sect. 2.2.1)

def rosseland_chi(disk, T):
    """Eq. 3 with chi' = kappa + (1-g) sigma (Eq. 16, g' = 0), bins integrated."""
    op = disk.opacity
    chi = op.kappa_abs + (1.0 - op.g) * op.kappa_sca
    if disk.opacity.is_gray():
        return float(chi[0])
    dB = dplanck_bins(op.lam_edges_um, max(T, 1.0))
    return float(dB.sum() / np.sum(dB / chi))


def cell_extent(disk):
    """Smallest extent of each cell, min(dr, r_c dtheta) (cm)."""
    rf, tf = disk.r_faces_cm, disk.theta_faces
    rc = 0.5 * (rf[:-1] + rf[1:])
    return np.minimum((rf[1:] - rf[:-1])[:, None], rc[:, None] * (tf[1:] - tf[:-1])[None, :])


def pda_mask(disk, visits, relerr, min_visits=30, max_rel_err=0.05, min_cell_tau=1.0):
    """PDA cells -- Sect. 3.1: fewer than 30 packet entries or a statistical temperature error above
    5 %; Sect. 2.2.1: only where the diffusion equation holds, i.e. in optically thick cells. Reading:
    a cell is thick when rho * max_b chi'_b * min(dr, r dtheta) >= min_cell_tau (default 1)."""
    op = disk.opacity
    chi_max = float(np.max(op.kappa_abs + (1.0 - op.g) * op.kappa_sca))
    thick = disk.rho * chi_max * cell_extent(disk) >= min_cell_tau
    return (disk.rho > 0) & thick & ((visits < min_visits) | (relerr > max_rel_err))


def dirichlet_mask(disk, pda, tally):
    """Cells whose Monte Carlo temperature bounds the PDA region: dust that absorbed energy. Reading:
    a cell outside the PDA region that absorbed nothing has no temperature estimate and, like a
    dust-free cell, carries no flux."""
    return (disk.rho > 0) & (~pda) & (np.asarray(tally).reshape(disk.rho.shape) > 0)


def _borders(mask):
    """Cells that share a face with a cell of `mask`."""
    out = np.zeros_like(mask)
    out[1:] |= mask[:-1]
    out[:-1] |= mask[1:]
    out[:, 1:] |= mask[:, :-1]
    out[:, :-1] |= mask[:, 1:]
    return out


def reference_T_for_D(T_mc, tally, mask, rho):
    """T at which D is frozen: the MC temperature where the cell absorbed energy, otherwise
    the mean MC temperature of the Dirichlet cells that border the PDA region."""
    nr, nt = T_mc.shape
    bnd = _borders(mask) & (~mask) & (rho > 0) & (np.asarray(tally).reshape(nr, nt) > 0)
    Tb = float(T_mc[bnd].mean()) if bnd.any() else float(T_mc[rho > 0].mean())
    return np.where(np.asarray(tally).reshape(nr, nt) > 0, T_mc, Tb)


def half_resistances(r_faces, theta_faces):
    """Geometric half-cell resistances (multiply by 1/D):
    hr_in[i,j]  cell centre -> face r_i,   hr_out[i,j] cell centre -> face r_{i+1},
    ht_lo[i,j]  cell centre -> face th_j,  ht_hi[i,j]  cell centre -> face th_{j+1}.
    Radial: flux through a shell portion of solid angle Omega is -D r^2 Omega du/dr, so the
    resistance of [a, b] is (1/a - 1/b)/(D Omega). Polar: flux through a cone face is
    -2 pi D sin(theta) (r2 - r1) du/dtheta, so [t1, t2] has resistance
    (ln tan(t2/2) - ln tan(t1/2)) / (2 pi D (r2 - r1))."""
    rf = np.asarray(r_faces, np.float64)
    tf = np.asarray(theta_faces, np.float64)
    rc = 0.5 * (rf[:-1] + rf[1:])
    tc = 0.5 * (tf[:-1] + tf[1:])
    omega = 2 * np.pi * (np.cos(tf[:-1]) - np.cos(tf[1:]))
    dr = rf[1:] - rf[:-1]
    hr_in = ((1 / rf[:-1] - 1 / rc)[:, None]) / omega[None, :]
    hr_out = ((1 / rc - 1 / rf[1:])[:, None]) / omega[None, :]
    with np.errstate(divide="ignore"):
        lt_f = np.log(np.tan(tf / 2))
    lt_c = np.log(np.tan(tc / 2))
    ht_lo = (lt_c - lt_f[:-1])[None, :] / (2 * np.pi * dr[:, None])
    ht_hi = (lt_f[1:] - lt_c)[None, :] / (2 * np.pi * dr[:, None])
    return hr_in, hr_out, ht_lo, ht_hi


def conductances(disk, D, part=None):
    """Face conductances Cr[i,j] between (i,j)-(i+1,j) and Ct[i,j] between (i,j)-(i,j+1);
    zero where either cell does not take part (no dust, or `part` False)."""
    hr_in, hr_out, ht_lo, ht_hi = half_resistances(disk.r_faces_cm, disk.theta_faces)
    dust = (disk.rho > 0) if part is None else part
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):  # D -> 0: no conductance
        Cr = 1.0 / (hr_out[:-1] / D[:-1] + hr_in[1:] / D[1:])
        Ct = 1.0 / (ht_hi[:, :-1] / D[:, :-1] + ht_lo[:, 1:] / D[:, 1:])
    Cr = np.where(dust[:-1] & dust[1:], Cr, 0.0)
    Ct = np.where(dust[:, :-1] & dust[:, 1:], Ct, 0.0)
    return Cr, Ct


def assemble(Cr, Ct, mask, u_bnd):
    """Sparse system A x = b over the PDA cells (mask); Dirichlet values u_bnd elsewhere."""
    import scipy.sparse as sp
    nr, nt = mask.shape
    idx = -np.ones((nr, nt), np.int64)
    idx[mask] = np.arange(int(mask.sum()))
    n = int(mask.sum())
    rows, cols, vals = [], [], []
    diag = np.zeros(n)
    b = np.zeros(n)
    has_dir = np.zeros(n, bool)

    def face(Cf, ia, ib, ua, ub, ma, mb):
        # faces between cell arrays a and b with conductance Cf
        sel = (Cf > 0) & (ma | mb)
        for a_pda, b_pda in ((True, True), (True, False), (False, True)):
            s = sel & (ma == a_pda) & (mb == b_pda)
            if not s.any():
                continue
            c = Cf[s]
            if a_pda and b_pda:
                i, j = ia[s], ib[s]
                np.add.at(diag, i, c)
                np.add.at(diag, j, c)
                rows.extend([i, j]); cols.extend([j, i]); vals.extend([-c, -c])
            elif a_pda:
                i = ia[s]
                np.add.at(diag, i, c)
                np.add.at(b, i, c * ub[s])
                has_dir[i] = True
            else:
                j = ib[s]
                np.add.at(diag, j, c)
                np.add.at(b, j, c * ua[s])
                has_dir[j] = True

    face(Cr, idx[:-1], idx[1:], u_bnd[:-1], u_bnd[1:], mask[:-1], mask[1:])
    face(Ct, idx[:, :-1], idx[:, 1:], u_bnd[:, :-1], u_bnd[:, 1:], mask[:, :-1], mask[:, 1:])
    rows.append(np.arange(n)); cols.append(np.arange(n)); vals.append(diag)
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return A, b, idx, has_dir


def check_components(A, b_has_dirichlet):
    """Every connected PDA component must touch a Dirichlet cell, or the system is singular."""
    import scipy.sparse.csgraph as cg
    ncomp, lab = cg.connected_components(A, directed=False)
    ok = np.zeros(ncomp, bool)
    np.logical_or.at(ok, lab, b_has_dirichlet)
    return bool(ok.all())


def solve_pda(disk, T_mc, tally, visits, relerr, min_visits=30, max_rel_err=0.05, kappa_R=None, min_cell_tau=1.0,
              rho_D=None):
    """Partial diffusion approximation, Sect. 2.2.1 (Eq. 4): returns (T_final, mask, u, info)."""
    import scipy.sparse.linalg as spla
    nr, nt = disk.nr, disk.ntheta
    visits = np.asarray(visits).reshape(nr, nt)
    relerr = np.asarray(relerr).reshape(nr, nt)
    mask = pda_mask(disk, visits, relerr, min_visits, max_rel_err, min_cell_tau)
    T_mc = np.asarray(T_mc, np.float64).reshape(nr, nt)
    if kappa_R is None:
        Tref = reference_T_for_D(T_mc, np.asarray(tally), mask, disk.rho)
        kappa_R = np.vectorize(lambda t: rosseland_chi(disk, t))(Tref) if not disk.opacity.is_gray() \
            else np.full((nr, nt), rosseland_chi(disk, 0.0))
    kappa_R = np.asarray(kappa_R, np.float64).reshape(nr, nt)
    rho_D = disk.rho if rho_D is None else np.asarray(rho_D, np.float64).reshape(nr, nt)
    with np.errstate(divide="ignore", over="ignore"):
        D = np.where(disk.rho > 0, 1.0 / (3.0 * rho_D * kappa_R), 0.0)
    part = mask | dirichlet_mask(disk, mask, tally)
    Cr, Ct = conductances(disk, D, part)
    u_bnd = np.where(mask, 0.0, T_mc ** 4)
    A, b, idx, has_dir = assemble(Cr, Ct, mask, u_bnd)
    info = dict(n_pda=int(mask.sum()), Cr=Cr, Ct=Ct, D=D, kappa_R=kappa_R, A=A, b=b, idx=idx)
    T = T_mc.copy()
    u = u_bnd.copy()
    if mask.any():
        if not check_components(A, has_dir):
            raise ValueError("PDA region has a component with no Monte Carlo boundary cell")
        x = spla.spsolve(A.tocsc(), b)
        u[mask] = x
        T[mask] = np.maximum(x, 0.0) ** 0.25
    return T, mask, u, info


def pda_adjoint(disk, u, mask, info, w):
    """Gradient of J = sum w_i T_i (T = u^(1/4) in PDA cells, fixed elsewhere) with respect to
    log rho and kappa_R per cell, by the adjoint of the PDA system (A symmetric)."""
    import scipy.sparse.linalg as spla
    nr, nt = mask.shape
    A = info["A"]
    D = info["D"]
    Cr, Ct = info["Cr"], info["Ct"]
    w = np.asarray(w, np.float64).reshape(nr, nt)
    g = np.zeros(int(mask.sum()))
    um = u[mask]
    with np.errstate(divide="ignore"):
        g[:] = np.where(um > 0, w[mask] * 0.25 * np.abs(um) ** (-0.75), 0.0)
    lam_v = spla.spsolve(A.tocsc(), g) if g.size else g
    lam = np.zeros((nr, nt))
    lam[mask] = lam_v
    hr_in, hr_out, ht_lo, ht_hi = half_resistances(disk.r_faces_cm, disk.theta_faces)
    dJdD = np.zeros((nr, nt))
    # radial faces
    dJdC = -(lam[:-1] - lam[1:]) * (u[:-1] - u[1:])
    act = (Cr > 0) & (mask[:-1] | mask[1:])
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        ta = np.where(act, dJdC * Cr ** 2 * hr_out[:-1] / D[:-1] ** 2, 0.0)
        tb = np.where(act, dJdC * Cr ** 2 * hr_in[1:] / D[1:] ** 2, 0.0)
    dJdD[:-1] += ta
    dJdD[1:] += tb
    dJdC = -(lam[:, :-1] - lam[:, 1:]) * (u[:, :-1] - u[:, 1:])
    act = (Ct > 0) & (mask[:, :-1] | mask[:, 1:])
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        ta = np.where(act, dJdC * Ct ** 2 * ht_hi[:, :-1] / D[:, :-1] ** 2, 0.0)
        tb = np.where(act, dJdC * Ct ** 2 * ht_lo[:, 1:] / D[:, 1:] ** 2, 0.0)
    dJdD[:, :-1] += ta
    dJdD[:, 1:] += tb
    with np.errstate(invalid="ignore"):
        grad_logrho = np.where(dJdD != 0, -D * dJdD, 0.0)
        grad_kR = np.where(dJdD != 0, -D / info["kappa_R"] * dJdD, 0.0)
    return grad_logrho, grad_kR, lam


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
