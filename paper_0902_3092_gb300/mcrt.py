"""ctypes binding of libmcrt.so (include/mcrt.h): argument marshalling only.

Every step of the transport, temperature and diffusion path runs in the CUDA library; this module
converts numpy arrays to pointers and C structs and raises on a non-zero status. It fails loudly
when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmcrt.so")

EUNIT = 65536
NINC = 10
T_MC, T_PDA = 0, 1
WITH_SCATTERING = 4
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV", 5: "ETIMEOUT", 6: "EOVERFLOW", 7: "ESTATE"}
EXPORTS = ["mcrt_disk_create", "mcrt_set_opacity", "mcrt_default_run_opts", "mcrt_run_photons", "mcrt_run_batch",
           "mcrt_reset", "mcrt_temperatures", "mcrt_temperatures_dev", "mcrt_get_tallies", "mcrt_sed",
           "mcrt_default_pda_opts", "mcrt_solve_pda", "mcrt_pda_adjoint", "mcrt_pda_adjoint_dev",
           "mcrt_trace_packets", "mcrt_checkpoint", "mcrt_restore", "mcrt_debug_uniforms", "mcrt_debug_mrw_x",
           "mcrt_pda_solve_static", "mcrt_disk_info", "mcrt_launch_count", "mcrt_last_error",
           "mcrt_disk_destroy", "mcrt_batch_create", "mcrt_batch_run", "mcrt_batch_config", "mcrt_batch_destroy",
           "mcrt_default_hydro_opts", "mcrt_hydrostatic_density", "mcrt_set_density", "mcrt_set_rays",
           "mcrt_raytrace", "mcrt_visibilities", "mcrt_set_sources", "mcrt_set_mueller", "mcrt_sed_stokes",
           "mcrt_keep_mean_intensity", "mcrt_mean_intensity"]


class McrtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(C.Structure):
    _fields_ = [("nr", C.c_int), ("ntheta", C.c_int), ("r_faces_cm", C.POINTER(C.c_double)),
                ("theta_faces", C.POINTER(C.c_double)), ("rho_gcm3", C.POINTER(C.c_double))]


class Star(C.Structure):
    _fields_ = [("T_star_K", C.c_double), ("R_star_cm", C.c_double)]


class RunOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("mrw", C.c_int), ("gamma", C.c_double), ("mrw_min_interactions", C.c_int),
                ("mrw_exit_dir", C.c_int), ("max_events_per_packet", C.c_uint64), ("n_total_packets", C.c_uint64),
                ("block_size", C.c_int), ("refill_interval", C.c_int), ("want_sed", C.c_int),
                ("tail_warps_per_sm", C.c_int), ("interact_batch", C.c_int), ("max_in_flight", C.c_uint64)]


class RunStats(C.Structure):
    _fields_ = [("packets", C.c_uint64), ("events", C.c_uint64), ("absorptions", C.c_uint64),
                ("scatterings", C.c_uint64), ("crossings", C.c_uint64), ("mrw_jumps", C.c_uint64),
                ("capped", C.c_uint64), ("escaped", C.c_uint64), ("deposit_sum", C.c_uint64),
                ("error_flags", C.c_uint32), ("seconds", C.c_double), ("max_packet_steps", C.c_uint64),
                ("longest_packet", C.c_uint64), ("guarded", C.c_uint64), ("guard_packet", C.c_uint64),
                ("guard_kind", C.c_int32), ("guard_in_tail", C.c_int32), ("guard_cell", C.c_int32 * 2),
                ("guard_events", C.c_uint64), ("guard_steps", C.c_uint64), ("guard_pos_cm", C.c_double * 3),
                ("guard_dir", C.c_double * 3)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if isinstance(v, C.Array) else v
        return out


class PdaOpts(C.Structure):
    _fields_ = [("min_visits", C.c_int), ("max_rel_err", C.c_double), ("tol", C.c_double), ("inner_tol", C.c_double),
                ("max_outer", C.c_int), ("max_inner", C.c_int), ("min_cell_tau", C.c_double),
                ("kappa_R", C.POINTER(C.c_double)), ("rho", C.POINTER(C.c_double))]


class HydroOpts(C.Structure):
    _fields_ = [("M_star_g", C.c_double), ("mu", C.c_double), ("T_floor_K", C.c_double), ("which", C.c_int),
                ("shell_mass_g", C.POINTER(C.c_double)), ("relax", C.POINTER(C.c_double))]


_lib = None


def lib():
    """Loads libmcrt.so; raises if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_0902_3092_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    P, pd, pu, pi = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_uint64), C.POINTER(C.c_int32)
    st = C.c_int
    sig = {
        "mcrt_disk_create": (st, [C.POINTER(Grid), C.POINTER(Star), C.c_int, P, C.POINTER(P)]),
        "mcrt_set_opacity": (st, [P, C.c_int, pd, pd, pd, pd]),
        "mcrt_default_run_opts": (None, [C.POINTER(RunOpts)]),
        "mcrt_run_photons": (st, [P, C.c_uint64, C.c_uint64, C.c_uint64, C.POINTER(RunOpts), C.POINTER(RunStats)]),
        "mcrt_run_batch": (st, [C.POINTER(P), C.c_int, pu, C.c_uint64, C.POINTER(RunOpts), C.POINTER(RunStats)]),
        "mcrt_reset": (st, [P]),
        "mcrt_temperatures": (st, [P, C.c_int, pd, pd, pu]),
        "mcrt_temperatures_dev": (st, [P, C.c_int, P, P]),
        "mcrt_get_tallies": (st, [P, pu, pu, pu]),
        "mcrt_sed": (st, [P, C.c_int, pd]),
        "mcrt_default_pda_opts": (None, [C.POINTER(PdaOpts)]),
        "mcrt_solve_pda": (st, [P, C.POINTER(PdaOpts), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "mcrt_pda_adjoint": (st, [P, pd, pd, pd]),
        "mcrt_pda_adjoint_dev": (st, [P, P, P, P]),
        "mcrt_trace_packets": (st, [P, C.c_uint64, C.c_uint64, C.c_uint64, C.POINTER(RunOpts), C.c_int, pi, pi, pi, pd,
                                    pi]),
        "mcrt_checkpoint": (st, [P, P, C.POINTER(C.c_size_t)]),
        "mcrt_restore": (st, [P, P, C.c_size_t]),
        "mcrt_debug_uniforms": (st, [C.c_int, C.c_uint64, C.c_uint32, C.c_uint64, C.c_int, pd]),
        "mcrt_debug_mrw_x": (st, [C.c_int, C.c_int, pd, pd]),
        "mcrt_disk_info": (st, [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "mcrt_launch_count": (st, [P, C.POINTER(C.c_uint64)]),
        "mcrt_pda_solve_static": (st, [C.c_int, C.c_int, C.c_int, P, P, P, P, C.POINTER(PdaOpts), P,
                                       C.POINTER(C.c_int)]),
        "mcrt_last_error": (C.c_char_p, [P]),
        "mcrt_batch_create": (st, [C.POINTER(P), C.c_int, pu, C.POINTER(RunOpts), C.POINTER(P)]),
        "mcrt_batch_run": (st, [P, C.c_uint64, C.POINTER(RunStats)]),
        "mcrt_batch_config": (st, [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_double)]),
        "mcrt_batch_destroy": (None, [P]),
        "mcrt_disk_destroy": (None, [P]),
        "mcrt_default_hydro_opts": (None, [C.POINTER(HydroOpts)]),
        "mcrt_hydrostatic_density": (st, [P, C.POINTER(HydroOpts), pd]),
        "mcrt_set_density": (st, [P, pd]),
        "mcrt_set_rays": (st, [P, C.c_double, C.c_double, C.c_int64, pd, pd, pd]),
        "mcrt_set_sources": (st, [P, pd]),
        "mcrt_set_mueller": (st, [P, C.c_int, pd]),
        "mcrt_sed_stokes": (st, [P, C.c_int, pd, pd, pd]),
        "mcrt_keep_mean_intensity": (st, [P, C.c_int]),
        "mcrt_mean_intensity": (st, [P, pd]),
        "mcrt_raytrace": (st, [P, C.c_int, C.c_int, pd, pd, pd, pu]),
        "mcrt_visibilities": (st, [P, C.c_int, pi, pd, pd, C.c_int, pd]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _up(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _check(status, handle=None):
    if status != 0:
        msg = lib().mcrt_last_error(handle)
        raise McrtError(status, msg.decode() if msg else "")


def run_opts(precision=32, mrw=False, gamma=2.0, nmin=20, exit_dir=0, max_events=100_000_000, n_total=0,
             block_size=0, refill=0, want_sed=True, tail_warps=0, interact_batch=0, max_in_flight=0):
    o = RunOpts()
    lib().mcrt_default_run_opts(C.byref(o))
    o.precision, o.mrw, o.gamma, o.mrw_min_interactions, o.mrw_exit_dir = precision, int(mrw), gamma, nmin, exit_dir
    o.max_events_per_packet, o.n_total_packets = int(max_events), int(n_total)
    o.block_size, o.refill_interval, o.want_sed = block_size, refill, int(want_sed)
    o.tail_warps_per_sm = tail_warps
    o.interact_batch = interact_batch
    o.max_in_flight = int(max_in_flight)
    return o


class Disk:
    """One disk model on one GPU (owns the library handle)."""

    def __init__(self, r_faces_cm, theta_faces, rho, T_star_K, R_star_cm, device=0, stream=None):
        L = lib()
        self._rf = np.ascontiguousarray(r_faces_cm, np.float64)
        self._tf = np.ascontiguousarray(theta_faces, np.float64)
        self._rho = np.ascontiguousarray(rho, np.float64).ravel()
        self.nr, self.ntheta = len(self._rf) - 1, len(self._tf) - 1
        g = Grid(self.nr, self.ntheta, _dp(self._rf), _dp(self._tf), _dp(self._rho))
        s = Star(float(T_star_K), float(R_star_cm))
        h = C.c_void_p()
        _check(L.mcrt_disk_create(C.byref(g), C.byref(s), int(device), stream, C.byref(h)))
        self._h = h
        self.nlam = 0

    @classmethod
    def from_model(cls, d, device=0, stream=None):
        """From a paper_0902_3092_gb300.disks.Disk (grid, star and dust)."""
        x = cls(d.r_faces_cm, d.theta_faces, d.rho, d.star.T_K, d.star.R_cm, device, stream)
        op = d.opacity
        x.set_opacity(op.lam_edges_um, op.kappa_abs, op.kappa_sca, op.g)
        return x

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().mcrt_disk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_opacity(self, lam_edges_um, kappa_abs, kappa_sca, g=None):
        e = np.ascontiguousarray(lam_edges_um, np.float64)
        ka = np.ascontiguousarray(kappa_abs, np.float64)
        ks = np.ascontiguousarray(kappa_sca, np.float64)
        gg = None if g is None else np.ascontiguousarray(g, np.float64)
        self.nlam = len(ka)
        _check(lib().mcrt_set_opacity(self._h, self.nlam, _dp(e), _dp(ka), _dp(ks), None if gg is None else _dp(gg)),
               self._h)

    def run_photons(self, n_packets, seed=1, first_id=0, **kw):
        o = run_opts(**kw)
        s = RunStats()
        try:
            _check(lib().mcrt_run_photons(self._h, int(n_packets), int(seed), int(first_id), C.byref(o),
                                          C.byref(s)), self._h)
        except McrtError as e:
            e.stats = s.as_dict()  # filled when the run completed (a step guard dropped packets)
            raise
        return s.as_dict()

    def trace(self, n_packets, seed=1, first_id=0, max_events=1000, **kw):
        o = run_opts(**kw)
        m = n_packets * max_events
        tr = dict(type=np.full(m, -1, np.int32), cell=np.full(m, -1, np.int32), lam=np.full(m, -1, np.int32),
                  pos=np.zeros((m, 3)), n=np.zeros(n_packets, np.int32))
        _check(lib().mcrt_trace_packets(self._h, int(n_packets), int(seed), int(first_id), C.byref(o), int(max_events),
                                        _ip(tr["type"]), _ip(tr["cell"]), _ip(tr["lam"]), _dp(tr["pos"]),
                                        _ip(tr["n"])), self._h)
        for k in ("type", "cell", "lam"):
            tr[k] = tr[k].reshape(n_packets, max_events)
        tr["pos"] = tr["pos"].reshape(n_packets, max_events, 3)
        return tr

    def reset(self):
        _check(lib().mcrt_reset(self._h), self._h)

    def hydrostatic_density(self, M_star_g=None, mu=None, T_floor=None, which=T_PDA, shell_mass=None, relax=None):
        """Density in hydrostatic equilibrium with the disk's temperatures (Sect. 2.5, Eq. 20), nr x ntheta;
        relax (nr factors): a damped step per shell from the disk's current density (see mcrt.h)."""
        o = HydroOpts()
        lib().mcrt_default_hydro_opts(C.byref(o))
        if M_star_g is not None:
            o.M_star_g = M_star_g
        if mu is not None:
            o.mu = mu
        if T_floor is not None:
            o.T_floor_K = T_floor
        o.which = which
        sm = None
        if shell_mass is not None:
            sm = np.ascontiguousarray(shell_mass, np.float64)
            o.shell_mass_g = _dp(sm)
        rl = None
        if relax is not None:
            rl = np.ascontiguousarray(relax, np.float64)
            if rl.shape != (self.nr,):
                raise ValueError("relax needs one factor per radial shell")
            o.relax = _dp(rl)
        out = np.zeros(self.nr * self.ntheta)
        _check(lib().mcrt_hydrostatic_density(self._h, C.byref(o), _dp(out)), self._h)
        return out.reshape(self.nr, self.ntheta)

    def set_sources(self, L_cell=None):
        """Internal source luminosity per cell (erg/s, nr x ntheta; None: none), e.g. viscous heating
        from disks.viscous_sources; resets the tallies."""
        if L_cell is None:
            _check(lib().mcrt_set_sources(self._h, None), self._h)
            self.L_src = 0.0
            return
        L = np.ascontiguousarray(L_cell, np.float64).ravel()
        _check(lib().mcrt_set_sources(self._h, _dp(L)), self._h)
        self.L_src = float(L.sum())

    def set_mueller(self, table=None):
        """Polarized transport with a Mueller matrix per wavelength bin (nlam x 4 x nmu: S11, S12, S33,
        S34 on theta_k = k pi / (nmu - 1), e.g. disks.rayleigh_mueller); None turns it off. Resets the
        tallies."""
        if table is None:
            _check(lib().mcrt_set_mueller(self._h, 0, None), self._h)
            return
        t = np.ascontiguousarray(table, np.float64)
        _check(lib().mcrt_set_mueller(self._h, int(t.shape[-1]), _dp(t)), self._h)

    def sed_stokes(self, n_incl=NINC):
        """Escaped luminosity per (wavelength bin, inclination group) as Stokes I, Q, U (erg/s); Q > 0
        for light polarized along the projected disk axis."""
        I, Q, U = (np.zeros(self.nlam * n_incl) for _ in range(3))
        _check(lib().mcrt_sed_stokes(self._h, int(n_incl), _dp(I), _dp(Q), _dp(U)), self._h)
        sh = (self.nlam, n_incl)
        return I.reshape(sh), Q.reshape(sh), U.reshape(sh)

    def keep_mean_intensity(self, keep=True):
        """Path-length estimator of the mean intensity in the following runs (flights in their bin, MRW
        walks spread with the weights of Eq. 10); resets the tallies."""
        _check(lib().mcrt_keep_mean_intensity(self._h, int(bool(keep))), self._h)

    def mean_intensity(self):
        """Mean intensity per cell and bin, (nr, ntheta, nlam), erg s^-1 cm^-2 sr^-1 integrated over the
        bin."""
        J = np.zeros(self.nr * self.ntheta * self.nlam)
        _check(lib().mcrt_mean_intensity(self._h, _dp(J)), self._h)
        return J.reshape(self.nr, self.ntheta, self.nlam)

    def set_density(self, rho):
        """Replaces the density (g/cm^3) and resets the tallies."""
        r = np.ascontiguousarray(rho, np.float64).ravel().copy()
        _check(lib().mcrt_set_density(self._h, _dp(r)), self._h)
        self._rho = r

    def density(self):
        """The density the disk holds (g/cm^3, nr x ntheta): the one it was created or last set with."""
        return self._rho.reshape(self.nr, self.ntheta).copy()

    def temperatures(self, which=T_MC):
        n = self.nr * self.ntheta
        T, e, v = np.zeros(n), np.zeros(n), np.zeros(n, np.uint64)
        _check(lib().mcrt_temperatures(self._h, int(which), _dp(T), _dp(e), _up(v)), self._h)
        sh = (self.nr, self.ntheta)
        return T.reshape(sh), e.reshape(sh), v.reshape(sh)

    def temperatures_dev(self, T_ptr, relerr_ptr=None, which=T_MC):
        _check(lib().mcrt_temperatures_dev(self._h, int(which), T_ptr, relerr_ptr), self._h)

    def tallies(self):
        n = self.nr * self.ntheta
        t, v, a = np.zeros(n, np.uint64), np.zeros(n, np.uint64), np.zeros(n, np.uint64)
        _check(lib().mcrt_get_tallies(self._h, _up(t), _up(v), _up(a)), self._h)
        return t, v, a

    def sed(self, n_incl=NINC):
        L = np.zeros(self.nlam * n_incl)
        _check(lib().mcrt_sed(self._h, int(n_incl), _dp(L)), self._h)
        return L.reshape(self.nlam, n_incl)

    def solve_pda(self, min_visits=30, max_rel_err=0.05, tol=1e-12, inner_tol=1e-5, max_outer=50, max_inner=20000,
                  kappa_R=None, min_cell_tau=1.0, rho=None, allow_notconv=False):
        """PDA solve (Sect. 2.2.1, Eq. 4); returns (PDA cells, CG iterations). With allow_notconv an
        exhausted iteration budget returns normally instead of raising McrtError(ENOTCONV)."""
        o = PdaOpts()
        lib().mcrt_default_pda_opts(C.byref(o))
        o.min_visits, o.max_rel_err, o.tol, o.inner_tol = min_visits, max_rel_err, tol, inner_tol
        o.min_cell_tau = min_cell_tau
        o.max_outer, o.max_inner = max_outer, max_inner
        kr = rr = None
        if kappa_R is not None:
            kr = np.ascontiguousarray(kappa_R, np.float64).ravel()
            o.kappa_R = _dp(kr)
        if rho is not None:
            rr = np.ascontiguousarray(rho, np.float64).ravel()
            o.rho = _dp(rr)
        npda, it = C.c_int(), C.c_int()
        s = lib().mcrt_solve_pda(self._h, C.byref(o), C.byref(npda), C.byref(it))
        if not (allow_notconv and s == 4):
            _check(s, self._h)
        return npda.value, it.value

    def pda_adjoint(self, w):
        w = np.ascontiguousarray(w, np.float64).ravel()
        n = self.nr * self.ntheta
        gl, gk = np.zeros(n), np.zeros(n)
        _check(lib().mcrt_pda_adjoint(self._h, _dp(w), _dp(gl), _dp(gk)), self._h)
        sh = (self.nr, self.ntheta)
        return gl.reshape(sh), gk.reshape(sh)

    def pda_adjoint_dev(self, w_ptr, g_lr_ptr, g_kr_ptr):
        _check(lib().mcrt_pda_adjoint_dev(self._h, w_ptr, g_lr_ptr, g_kr_ptr), self._h)

    def launch_count(self) -> int:
        n = C.c_uint64()
        _check(lib().mcrt_launch_count(self._h, C.byref(n)), self._h)
        return n.value

    def set_rays(self, incl, dist_cm, rays):
        """Sky-plane rays of the observables (paper_0902_3092_gb300.disks.Rays, cm) for an observer at
        inclination incl (rad) and distance dist_cm."""
        self._rays = tuple(np.ascontiguousarray(x, np.float64) for x in (rays.p, rays.q, rays.w))
        p, q, w = self._rays
        _check(lib().mcrt_set_rays(self._h, float(incl), float(dist_cm), len(p), _dp(p), _dp(q), _dp(w)), self._h)

    def raytrace(self, which=T_MC, precision=32, want_image=False, scattering=False):
        """Ray-traced SED of the current rays: dict with F (disk + star, erg/s/cm^2 per wavelength bin),
        F_star, segments (ray segments through dust) and, with want_image, I (rays x bins intensities,
        erg/s/cm^2/sr per bin). scattering: add the scattered light of the mean-intensity tally."""
        F, Fs = np.zeros(self.nlam), np.zeros(self.nlam)
        rays = getattr(self, "_rays", None)
        n = len(rays[0]) if rays is not None else 0
        I = np.zeros(n * self.nlam) if want_image else None
        seg = np.zeros(1, np.uint64)
        w = int(which) | (WITH_SCATTERING if scattering else 0)
        _check(lib().mcrt_raytrace(self._h, w, int(precision), _dp(F), _dp(Fs),
                                   None if I is None else _dp(I), _up(seg)), self._h)
        out = {"F": F, "F_star": Fs, "segments": int(seg[0])}
        if I is not None:
            out["I"] = I.reshape(n, self.nlam)
        return out

    def visibilities(self, bins, baseline_cm, pa_rad, with_star=True):
        """|V| of the last ray-traced image at wavelength bins `bins`, baselines (cm) and position angles
        (rad, from the projected major axis), the star included as an unresolved source."""
        b = np.ascontiguousarray(bins, np.int32).ravel()
        B = np.ascontiguousarray(np.broadcast_to(baseline_cm, b.shape), np.float64)
        pa = np.ascontiguousarray(np.broadcast_to(pa_rad, b.shape), np.float64)
        out = np.zeros(b.size)
        _check(lib().mcrt_visibilities(self._h, b.size, _ip(b), _dp(B), _dp(pa), int(bool(with_star)), _dp(out)),
               self._h)
        return out

    def checkpoint(self) -> bytes:
        n = C.c_size_t()
        _check(lib().mcrt_checkpoint(self._h, None, C.byref(n)), self._h)
        buf = C.create_string_buffer(n.value)
        _check(lib().mcrt_checkpoint(self._h, C.cast(buf, C.c_void_p), C.byref(n)), self._h)
        return buf.raw

    def restore(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(lib().mcrt_restore(self._h, C.cast(buf, C.c_void_p), len(blob)), self._h)


def run_batch(disks, n_packets, seed=1, **kw):
    o = run_opts(**kw)
    n = len(disks)
    hs = (C.c_void_p * n)(*[d.handle for d in disks])
    npk = np.ascontiguousarray(n_packets, np.uint64)
    stats = (RunStats * n)()
    _check(lib().mcrt_run_batch(hs, n, _up(npk), int(seed), C.byref(o), stats))
    return [s.as_dict() for s in stats]


def pda_solve_static(nr, ntheta, mask_ptr, Cr_ptr, Ct_ptr, u_ptr, device=0, stream=None, tol=1e-12,
                     inner_tol=1e-5, max_outer=50, max_inner=20000):
    """PDA solve on caller-owned device buffers with no device allocation (see include/mcrt.h)."""
    o = PdaOpts()
    lib().mcrt_default_pda_opts(C.byref(o))
    o.tol, o.inner_tol, o.max_outer, o.max_inner = tol, inner_tol, max_outer, max_inner
    it = C.c_int()
    _check(lib().mcrt_pda_solve_static(int(device), int(nr), int(ntheta), mask_ptr, Cr_ptr, Ct_ptr, u_ptr,
                                        C.byref(o), stream, C.byref(it)))
    return it.value


class Batch:
    """Disks transported together by one persistent launch, replayed from a captured CUDA graph."""

    def __init__(self, disks, n_packets, **kw):
        o = run_opts(**kw)
        self.disks = list(disks)
        self.n = len(self.disks)
        hs = (C.c_void_p * self.n)(*[d.handle for d in self.disks])
        self._npk = np.ascontiguousarray(n_packets, np.uint64)
        h = C.c_void_p()
        _check(lib().mcrt_batch_create(hs, self.n, _up(self._npk), C.byref(o), C.byref(h)))
        self._h = h

    def run(self, seed=1):
        stats = (RunStats * self.n)()
        _check(lib().mcrt_batch_run(self._h, int(seed), stats))
        return [s.as_dict() for s in stats]

    def config(self):
        b, r, g, t = C.c_int(), C.c_int(), C.c_int(), C.c_double()
        _check(lib().mcrt_batch_config(self._h, C.byref(b), C.byref(r), C.byref(g), C.byref(t)))
        return {"block_size": b.value, "refill_interval": r.value, "grid": g.value, "tune_seconds": t.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().mcrt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_uniforms(seed, model, packet, n, device=0):
    out = np.zeros(n)
    _check(lib().mcrt_debug_uniforms(int(device), int(seed), int(model), int(packet), int(n), _dp(out)))
    return out


def debug_mrw_x(P0, device=0):
    P0 = np.ascontiguousarray(P0, np.float64)
    out = np.zeros_like(P0)
    _check(lib().mcrt_debug_mrw_x(int(device), len(P0), _dp(P0), _dp(out)))
    return out
