"""Seeded synthetic disk models: grids, densities, star and dust opacities.

This module only builds input arrays. It holds none of the transport, temperature
or diffusion arithmetic, so that both the CUDA library and the CPU oracle can take
the same inputs from it.

Disk density follows Sect. 2.4, Eq. 17-18:

    rho(R, z) = rho0 * (R/AU)^(-1-p) * exp(-(z/h(R))^2),   h(R) = h1 * (R/AU)^p,

for R_in < R < R_out (cylindrical R), zero elsewhere. Instead of the dust mass, the
constant rho0 is fixed by the closed-form midplane radial optical depth of Eq. 19,
evaluated with the extinction at the reference wavelength. Surface density then
goes as R^-1 (Sect. 2.4, item 1).

All quantities are cgs at this boundary: lengths in cm, density in g cm^-3, mass
opacities in cm^2 g^-1, wavelengths in micron.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

AU_CM = 1.495978707e13
RSUN_CM = 6.957e10
H_PLANCK = 6.62607015e-27
C_LIGHT = 2.99792458e10
K_BOLTZ = 1.380649e-16
SIGMA_SB = 2 * math.pi ** 5 * K_BOLTZ ** 4 / (15 * H_PLANCK ** 3 * C_LIGHT ** 2)  # erg cm^-2 s^-1 K^-4


@dataclasses.dataclass
class Star:
    T_K: float
    R_cm: float

    @property
    def L(self) -> float:
        """Blackbody luminosity 4 pi R^2 sigma T^4 (erg/s)."""
        return 4.0 * math.pi * self.R_cm ** 2 * SIGMA_SB * self.T_K ** 4


@dataclasses.dataclass
class Opacity:
    lam_edges_um: np.ndarray  # nlam+1, increasing
    kappa_abs: np.ndarray     # nlam, cm^2/g
    kappa_sca: np.ndarray     # nlam, cm^2/g
    g: np.ndarray             # nlam, Henyey-Greenstein asymmetry

    @property
    def nlam(self) -> int:
        return len(self.kappa_abs)

    def is_gray(self) -> bool:
        return bool(np.all(self.kappa_abs == self.kappa_abs[0])
                    and np.all(self.kappa_sca == self.kappa_sca[0])
                    and np.all(self.g == self.g[0]))


@dataclasses.dataclass
class Disk:
    r_faces_cm: np.ndarray     # nr+1
    theta_faces: np.ndarray    # ntheta+1, radians, 0..pi, pi/2 is a face
    rho: np.ndarray            # (nr, ntheta), g/cm^3
    star: Star
    opacity: Opacity
    name: str = ""
    params: dict = dataclasses.field(default_factory=dict)

    @property
    def nr(self) -> int:
        return len(self.r_faces_cm) - 1

    @property
    def ntheta(self) -> int:
        return len(self.theta_faces) - 1


# ----------------------------------------------------------------------------- grids

def log_r_faces(r_in_au: float, r_out_au: float, nr: int) -> np.ndarray:
    return np.geomspace(r_in_au, r_out_au, nr + 1) * AU_CM


def rim_refined_r_faces(r_in_au: float, r_out_au: float, nr: int, n_fine: int = 20,
                        dr1_frac: float = 1e-3, growth: float = 1.3) -> np.ndarray:
    """First n_fine cells grow geometrically from dr1 = dr1_frac*r_in by `growth`,
    the remaining nr-n_fine cells are log-spaced out to r_out."""
    f = [r_in_au]
    dr = dr1_frac * r_in_au
    for _ in range(n_fine):
        f.append(f[-1] + dr)
        dr *= growth
    rest = np.geomspace(f[-1], r_out_au, nr - n_fine + 1)
    return np.concatenate([np.array(f[:-1]), rest]) * AU_CM


def midplane_refined_theta_faces(ntheta: int) -> np.ndarray:
    """ntheta even; faces at pi/2 -/+ (pi/2)(k/(ntheta/2))^2, k = 0..ntheta/2, so that
    pi/2 is a face and spacing is finest at the midplane."""
    if ntheta % 2:
        raise ValueError("ntheta must be even so that the midplane is a face")
    half = ntheta // 2
    k = np.arange(half + 1, dtype=np.float64)
    off = (math.pi / 2) * (k / half) ** 2
    upper = math.pi / 2 - off[::-1]   # 0 .. pi/2
    lower = math.pi / 2 + off[1:]     # .. pi
    t = np.concatenate([upper, lower])
    t[0] = 0.0
    t[-1] = math.pi
    return t


def cell_centres(r_faces_cm: np.ndarray, theta_faces: np.ndarray):
    """Arithmetic mid-points in r and theta."""
    rc = 0.5 * (r_faces_cm[:-1] + r_faces_cm[1:])
    tc = 0.5 * (theta_faces[:-1] + theta_faces[1:])
    return rc, tc


# ----------------------------------------------------------------------------- density

def rho0_for_tau(tau_mid: float, chi_ref: float, p: float, R_in_au: float, R_out_au: float) -> float:
    """rho0 such that Eq. 19's closed form  tau = rho0 chi AU (R_in^-p - R_out^-p)/p
    (R in AU) equals tau_mid."""
    return tau_mid / (chi_ref * AU_CM * (R_in_au ** (-p) - R_out_au ** (-p)) / p)


def density(R_cm, z_cm, rho0, h1_au, p, R_in_au, R_out_au):
    """Eq. 17-18 with the cylindrical truncation R_in < R < R_out."""
    R_au = np.asarray(R_cm, dtype=np.float64) / AU_CM
    h_cm = h1_au * AU_CM * np.power(np.maximum(R_au, 1e-300), p)
    inside = (R_au > R_in_au) & (R_au < R_out_au)
    with np.errstate(over="ignore", under="ignore", divide="ignore", invalid="ignore"):
        val = rho0 * np.power(np.maximum(R_au, 1e-300), -1.0 - p) * np.exp(-(np.asarray(z_cm) / h_cm) ** 2)
    return np.where(inside, val, 0.0)


def disk_mass_eq17(rho0, h1_au, R_in_au, R_out_au) -> float:
    """Mass implied by Eq. 17's prefactor: M = 2 pi sqrt(pi) h1 rho0 (R_out-R_in) AU^3."""
    return 2.0 * math.pi * math.sqrt(math.pi) * h1_au * rho0 * (R_out_au - R_in_au) * AU_CM ** 3


# ----------------------------------------------------------------------------- opacities

def lam_edges(nlam: int = 100, lo_um: float = 0.1, hi_um: float = 1000.0) -> np.ndarray:
    return np.geomspace(lo_um, hi_um, nlam + 1)


def gray_opacity(nlam: int = 100, albedo: float = 0.5, chi: float = 1.0e3, g: float = 0.0) -> Opacity:
    e = lam_edges(nlam)
    ka = np.full(nlam, chi * (1.0 - albedo))
    ks = np.full(nlam, chi * albedo)
    return Opacity(e, ka, ks, np.full(nlam, g))


def powerlaw_opacity(nlam: int = 100, kappa0: float = 1.0e3, g: float = 0.6) -> Opacity:
    """kappa_abs flat below 1 micron and ~1/lambda beyond; albedo 0.5 for lambda <= 1 um,
    0.5(1 - log10(lambda/um)/2) for 1-100 um and 0 beyond; kappa_sca = kappa_abs w/(1-w).
    Evaluated at the geometric bin centre."""
    e = lam_edges(nlam)
    lc = np.sqrt(e[:-1] * e[1:])
    ka = np.where(lc <= 1.0, kappa0, kappa0 / lc)
    w = np.where(lc <= 1.0, 0.5, np.where(lc < 100.0, 0.5 * (1.0 - np.log10(lc) / 2.0), 0.0))
    w = np.clip(w, 0.0, 0.5)
    ks = ka * w / (1.0 - w)
    return Opacity(e, ka, ks, np.full(nlam, g))


def extinction_at(op: Opacity, lam_um: float) -> float:
    b = int(np.searchsorted(op.lam_edges_um, lam_um, side="right") - 1)
    b = min(max(b, 0), op.nlam - 1)
    return float(op.kappa_abs[b] + op.kappa_sca[b])


# ----------------------------------------------------------------------------- models

def make_disk(r_faces_cm, theta_faces, star: Star, op: Opacity, tau_mid: float,
              h1_au: float = 0.05, p: float = 9.0 / 7.0, R_in_au=None, R_out_au=None,
              lam_ref_um: float = 0.55, name: str = "") -> Disk:
    R_in_au = r_faces_cm[0] / AU_CM if R_in_au is None else R_in_au
    R_out_au = r_faces_cm[-1] / AU_CM if R_out_au is None else R_out_au
    chi_ref = extinction_at(op, lam_ref_um)
    rho0 = rho0_for_tau(tau_mid, chi_ref, p, R_in_au, R_out_au)
    rc, tc = cell_centres(r_faces_cm, theta_faces)
    R = rc[:, None] * np.sin(tc)[None, :]
    z = rc[:, None] * np.cos(tc)[None, :]
    rho = density(R, z, rho0, h1_au, p, R_in_au, R_out_au)
    return Disk(np.asarray(r_faces_cm, np.float64), np.asarray(theta_faces, np.float64),
                np.ascontiguousarray(rho), star, op, name,
                dict(tau_mid=tau_mid, h1_au=h1_au, p=p, R_in_au=R_in_au, R_out_au=R_out_au,
                     rho0=rho0, chi_ref=chi_ref, lam_ref_um=lam_ref_um))


def paper_star() -> Star:
    """T* = 4000 K blackbody, R* = 2 R_sun."""
    return Star(4000.0, 2.0 * RSUN_CM)


def config_plain_gray(nr=40, ntheta=40, tau_mid=100.0) -> Disk:
    """Gray dust, albedo 0.5, isotropic, r 0.1-100 AU log-spaced, tau_mid = 100."""
    return make_disk(log_r_faces(0.1, 100.0, nr), midplane_refined_theta_faces(ntheta),
                     paper_star(), gray_opacity(), tau_mid, name=f"gray{nr}x{ntheta}_tau{tau_mid:g}")


def config_nongray(nr=100, ntheta=60, tau_mid=1e5) -> Disk:
    """Power-law absorption, falling albedo, HG g=0.6, tau_mid(0.55um) = 1e5."""
    return make_disk(log_r_faces(0.1, 100.0, nr), midplane_refined_theta_faces(ntheta),
                     paper_star(), powerlaw_opacity(), tau_mid, name=f"nongray{nr}x{ntheta}_tau{tau_mid:g}")


def config_thick_gray(nr=200, ntheta=120, tau_mid=1e6) -> Disk:
    """Gray dust (albedo 0.5, isotropic) at tau_mid = 1e6 with a rim-refined radial grid."""
    return make_disk(rim_refined_r_faces(0.1, 100.0, nr), midplane_refined_theta_faces(ntheta),
                     paper_star(), gray_opacity(), tau_mid, name=f"thickgray{nr}x{ntheta}_tau{tau_mid:g}")


def config_pda_adjoint(nr=400, ntheta=200, tau_mid=1e6) -> Disk:
    """400 x 200 grid, tau_mid = 1e6, non-gray power-law dust."""
    return make_disk(log_r_faces(0.1, 100.0, nr), midplane_refined_theta_faces(ntheta),
                     paper_star(), powerlaw_opacity(), tau_mid, name=f"pda{nr}x{ntheta}_tau{tau_mid:g}")


def batch_sweep(n_models=64, seed=1, max_nr=300, max_ntheta=180):
    """Models of uneven size: nr ~ U{50..300}, ntheta ~ U{30..180} even, tau_mid log-uniform
    1e2-1e6, flaring exponent beta ~ U(1/7, 3/7) with h/r = 0.05 (r/AU)^beta, packet budgets
    log-uniform 1e5-1e7. Returns (disks, packets)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    disks, packets = [], []
    for m in range(n_models):
        nr = int(rng.integers(50, max_nr + 1))
        nt = 2 * int(rng.integers(15, max_ntheta // 2 + 1))
        tau = float(10 ** rng.uniform(2, 6))
        beta = float(rng.uniform(1 / 7, 3 / 7))
        npk = int(10 ** rng.uniform(5, 7))
        d = make_disk(log_r_faces(0.1, 100.0, nr), midplane_refined_theta_faces(nt), paper_star(),
                      powerlaw_opacity(), tau, h1_au=0.05, p=1.0 + beta, name=f"batch{m}")
        disks.append(d)
        packets.append(npk)
    return disks, packets


@dataclasses.dataclass
class Rays:
    """Sky-plane sampling of an image: points (p, q) in cm along the axes of the projected disk (p along
    its major axis) and the sky-plane area w (cm^2) each point stands for."""
    p: np.ndarray
    q: np.ndarray
    w: np.ndarray

    @property
    def n(self) -> int:
        return int(self.p.size)


def polar_rays(r_faces_cm: np.ndarray, n_sub: int = 4, n_phi: int = 64, n_inner: int = 8) -> Rays:
    """Rings of rays in the sky plane: n_inner rings inside the inner radius and n_sub rings across every
    radial cell (edges equally spaced between the radial faces), n_phi rays per ring at the mid-radius
    of the ring and equally spaced azimuths; each ray stands for its share of the ring's area."""
    rf = np.asarray(r_faces_cm, np.float64)
    inner = np.linspace(0.0, rf[0], n_inner + 1)
    cells = (rf[:-1, None] + (rf[1:] - rf[:-1])[:, None] * (np.arange(n_sub) / n_sub)[None, :]).ravel()
    edges = np.concatenate([inner[:-1], cells, rf[-1:]])
    b = 0.5 * (edges[:-1] + edges[1:])
    area = np.pi * (edges[1:] ** 2 - edges[:-1] ** 2) / n_phi
    phi = (np.arange(n_phi) + 0.5) * (2.0 * np.pi / n_phi)
    p = (b[:, None] * np.cos(phi)[None, :]).ravel()
    q = (b[:, None] * np.sin(phi)[None, :]).ravel()
    w = np.repeat(area, n_phi)
    return Rays(p, q, w)


G_CGS = 6.67430e-8        # cm^3 g^-1 s^-2
MSUN_G = 1.98892e33
YEAR_S = 3.15576e7


def viscous_sources(d: Disk, mdot_msun_yr: float = 1e-8, M_star_msun: float = 2.5) -> np.ndarray:
    """Internal source luminosity per cell (erg/s, nr x ntheta) for viscous heating, which the paper
    leaves to future work (Sect. 5). Reading: the steady accretion-disk dissipation, 3 G M Mdot /
    (8 pi R^3) (1 - sqrt(R_in / R)) per unit area of each face, released in proportion to the dust
    mass of the column, so a cell at cylindrical radius R releases m_cell Q(R) / Sigma(R) with Q twice
    the one-face rate and Sigma(R) = sqrt(pi) h1 rho0 AU / (R / AU) the surface density of Eq. 17."""
    prm = d.params
    R_in = prm["R_in_au"] * AU_CM
    rc, tc = cell_centres(d.r_faces_cm, d.theta_faces)
    R = rc[:, None] * np.sin(tc)[None, :]
    rf, tf = d.r_faces_cm, d.theta_faces
    V = (2 * math.pi / 3) * (rf[1:] ** 3 - rf[:-1] ** 3)[:, None] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :]
    mdot = mdot_msun_yr * MSUN_G / YEAR_S
    GM = G_CGS * M_star_msun * MSUN_G
    with np.errstate(divide="ignore", invalid="ignore"):
        F = np.where(R > R_in, 3 * GM * mdot / (8 * math.pi * R ** 3) * (1 - np.sqrt(R_in / R)), 0.0)
        sigma = math.sqrt(math.pi) * prm["h1_au"] * AU_CM * prm["rho0"] / (R / AU_CM)
        L = np.where((d.rho > 0) & (sigma > 0), d.rho * V * 2 * F / sigma, 0.0)
    return np.ascontiguousarray(L)


def rayleigh_mueller(nlam: int = 100, nmu: int = 181) -> np.ndarray:
    """Mueller matrix of small (Rayleigh) particles on theta_k = k pi / (nmu - 1), every bin alike:
    (nlam, 4, nmu) = S11, S12, S33, S34 with S11 = (3/4)(1 + mu^2), S12 = (3/4)(mu^2 - 1),
    S33 = (3/2) mu, S34 = 0 (mu = cos theta; normalised so S11 averages to 1 over the sphere)."""
    mu = np.cos(np.linspace(0.0, math.pi, nmu))
    t = np.stack([0.75 * (1 + mu ** 2), 0.75 * (mu ** 2 - 1), 1.5 * mu, np.zeros(nmu)])
    return np.ascontiguousarray(np.broadcast_to(t, (nlam, 4, nmu)))


def hg_polarized_mueller(g: np.ndarray, p_lin: np.ndarray, nmu: int = 181) -> np.ndarray:
    """Synthetic Mueller matrix per bin in the form White (1979, ApJ 229, 954) gives for dust: a
    Henyey-Greenstein S11 of asymmetry g, S12 = -p_lin S11 (1 - mu^2) / (1 + mu^2) and
    S33 = S11 2 mu / (1 + mu^2), no circular term (S34 = 0). g = 0 and p_lin = 1 give the Rayleigh
    polarization with an isotropic S11. (nlam, 4, nmu) on theta_k = k pi / (nmu - 1)."""
    g = np.atleast_1d(np.asarray(g, np.float64))[:, None]
    p = np.atleast_1d(np.asarray(p_lin, np.float64))[:, None]
    mu = np.cos(np.linspace(0.0, math.pi, nmu))[None, :]
    s11 = (1 - g ** 2) / (1 + g ** 2 - 2 * g * mu) ** 1.5
    out = np.stack([s11, -p * s11 * (1 - mu ** 2) / (1 + mu ** 2), s11 * 2 * mu / (1 + mu ** 2),
                    np.zeros_like(s11)], axis=1)
    return np.ascontiguousarray(out)
