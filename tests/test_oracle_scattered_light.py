"""Pins of the oracle's mean-intensity estimator and of the scattered-light source function of its ray
tracer (Sect. 2.3: the observables come from the computed source function, scattering included): the
path-length estimator against the closed form of an optically thin absorbing shell and, with MRW
walks, against radiative equilibrium, and the ray-traced scattered flux of a purely scattering disk against the Monte Carlo escape spectrum of the
packets that scattered."""
import math

import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

AU = disks.AU_CM
PC = 3.0856775814913673e18


def test_mean_intensity_of_thin_absorbing_shell(oracle):
    """Absorbing shell (albedo 0) of radial optical depth 0.3 around the point star: in the stellar bins
    J = L_b exp(-tau(r)) / (16 pi^2 r^2), whose volume average over a shell (r1, r2) is
    L_b / (16 pi^2) (e^-tau(r1) - e^-tau(r2)) / a * 3 / (r2^3 - r1^3) (a = rho chi). Every radial shell,
    every bin that received at least 5000 packets, within four counting errors."""
    rf = np.geomspace(1.0, 3.0, 7) * AU
    tf = np.linspace(0.0, math.pi, 9)
    op = disks.gray_opacity(nlam=12, albedo=0.0)
    chi = op.kappa_abs[0] + op.kappa_sca[0]
    rho = np.full((6, 8), 0.3 / (chi * (rf[-1] - rf[0])))
    d = disks.Disk(rf, tf, rho, disks.paper_star(), op, "shell")
    n = 200_000
    r = oracle.Run(d).run(n, seed=4, want_j=True)
    J = r.mean_intensity()
    Bs = oracle.planck_bins(op.lam_edges_um, d.star.T_K)
    Lb = 4 * math.pi ** 2 * d.star.R_cm ** 2 * Bs
    n_b = n * Bs / Bs.sum()
    lc = np.sqrt(op.lam_edges_um[:-1] * op.lam_edges_um[1:])
    sel = (n_b >= 5000) & (lc < 3.0)
    assert sel.sum() >= 2
    V = (2 * math.pi / 3) * (rf[1:] ** 3 - rf[:-1] ** 3)[:, None] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :]
    a = rho[0, 0] * chi
    for i in range(6):
        Js = (J[i] * V[i][:, None]).sum(axis=0) / V[i].sum()
        t1, t2 = a * (rf[i] - rf[0]), a * (rf[i + 1] - rf[0])
        ref = Lb / (16 * math.pi ** 2) * (math.exp(-t1) - math.exp(-t2)) / a * 3 / (rf[i + 1] ** 3 - rf[i] ** 3)
        assert np.all(np.abs(Js[sel] / ref[sel] - 1) < 4 / np.sqrt(n_b[sel]) + 2e-3), (i, Js[sel] / ref[sel])


@pytest.mark.parametrize("kind,n", [("gray", 20_000), ("nongray", 8_000)])
def test_mean_intensity_balances_absorption_with_mrw(oracle, kind, n):
    """Radiative equilibrium: a cell's absorbed energy, which sets its temperature, equals
    4 pi m sum_b kappa_b J_b, the absorption the path-length J implies; with MRW walks (Eq. 9-10) the
    walk's c t must count in J with the weights of Eq. 10, else the MRW cells break the balance (the
    diffusion-flux spectrum dB/dT / chi' instead would put this dust's kappa_bar 27 % low, spreading at
    the end-of-run temperature 10 % high). Every cell with 100 or more packet energies, within four
    counting errors sqrt(n_abs) / (absorbed packet energies) plus 1e-3; cells where the walks deposit
    over 40 % take part."""
    d = disks.config_plain_gray(16, 16, 1e4) if kind == "gray" else disks.config_nongray(16, 16, 1e4)
    r = oracle.Run(d).run(n, seed=5, mrw=True, gamma=2.0, nmin=5, want_j=True)
    J = r.mean_intensity()
    T, _ = r.temperatures()
    op = d.opacity
    units = r.tally.reshape(d.nr, d.ntheta) / 65536.0
    nabs = r.nabs.reshape(d.nr, d.ntheta).astype(float)
    n_mrw_cells = 0
    for i, j in zip(*np.nonzero(units >= 100)):
        absorbed = (op.kappa_abs * J[i, j]).sum()
        emitted = (op.kappa_abs * oracle.planck_bins(op.lam_edges_um, T[i, j])).sum()
        assert abs(absorbed / emitted - 1) < 4 * math.sqrt(nabs[i, j]) / units[i, j] + 1e-3, (i, j)
        n_mrw_cells += nabs[i, j] < 0.6 * units[i, j]
    assert r.stats["mrw_jumps"] > 300 and n_mrw_cells >= 2


def test_ray_traced_scattered_light_matches_monte_carlo(oracle):
    """Pure isotropic scattering (albedo 1, gray) in a thin disk of h/r = 0.2 and midplane optical depth
    0.05: the flux of the rays through the source function J (sigma J / chi with kappa = 0), averaged over
    each inclination bin, equals the Monte Carlo escape luminosity of the scattered packets in that bin
    over 4 pi d^2 and the bin's solid-angle fraction 0.1, within four counting errors plus 3 % (ray
    sampling)."""
    from oracle import raytrace as R
    op = disks.gray_opacity(nlam=4, albedo=1.0)
    d = disks.make_disk(disks.log_r_faces(0.1, 100.0, 16), disks.midplane_refined_theta_faces(16),
                        disks.paper_star(), op, 0.05, h1_au=0.2, p=1.0, name="thin_scatter")
    n = 4_000_000
    r = oracle.Run(d).run(n, seed=7, want_j=True)
    J = r.mean_intensity()
    Lsca = r.sed_scattered_lum().sum(axis=0)
    nsca = r.sed_sca.reshape(op.nlam, 10).sum(axis=0)
    dist = 100 * PC
    rays = disks.polar_rays(d.r_faces_cm, n_sub=2, n_phi=32, n_inner=4)
    T = np.zeros(d.rho.shape)
    for k in (0, 3, 6, 9):
        rt = np.mean([R.sed(d, T, math.acos(mu), dist, rays.p, rays.q, rays.w, J=J)[1].sum()
                      for mu in (k / 10 + 0.025, k / 10 + 0.075)])
        mc = Lsca[k] / (4 * math.pi * dist ** 2 * 0.1)
        assert nsca[k] > 2000
        assert abs(mc / rt - 1) < 4 / math.sqrt(nsca[k]) + 0.03, (k, mc / rt)


def test_source_without_mean_intensity_unchanged(oracle):
    from oracle import raytrace as R
    d = disks.config_nongray(8, 8, 100.0)
    rc, tc = disks.cell_centres(d.r_faces_cm, d.theta_faces)
    T = 300.0 * (rc[:, None] / AU) ** -0.5 * np.ones(d.rho.shape)
    a = R.source(d, T)
    b = R.source(d, T, J=np.zeros((d.nr, d.ntheta, d.opacity.nlam)))
    assert np.array_equal(a, b)
