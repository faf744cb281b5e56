"""Pins of the vertical-structure oracle (Sect. 2.5, Eq. 20) against closed forms of the hydrostatic
balance along a radial shell."""
import numpy as np

from paper_0902_3092_gb300 import disks

from oracle import hydro as H

AU = 1.495978707e13


def _grid(nt, r1=1.0 * AU, r2=1.02 * AU):
    return np.array([r1, r2]), np.linspace(0.0, np.pi, nt + 1)


def _profile_error(nt, T_of_theta, closed):
    rf, tf = _grid(nt)
    th = 0.5 * (tf[:-1] + tf[1:])
    T = T_of_theta(th)[None, :]
    mask = np.ones((1, nt), bool)
    rho = H.hydrostatic_density(rf, tf, mask, T, np.array([1e25]))[0]
    ref = closed(rf, tf, th)
    sel = ref > 1e-8 * ref.max()
    a = rho[sel] / rho[sel].max()
    b = ref[sel] / ref[sel].max()
    return np.max(np.abs(a / b - 1.0))


def test_isothermal_shell_matches_closed_form_second_order():
    T0 = 300.0
    closed = lambda rf, tf, th: H.isothermal_shell_density(rf, tf, 0, T0)
    e1 = _profile_error(400, lambda th: np.full_like(th, T0), closed)
    e2 = _profile_error(800, lambda th: np.full_like(th, T0), closed)
    assert e1 < 2e-3
    assert 3.0 < e1 / e2 < 5.0  # trapezoid rule: error falls as (dtheta)^2


def test_temperature_inverse_sine_closed_form():
    """T = T0 / sin(theta): Eq. 20 along the shell integrates to rho proportional to sin^(K+1)(theta)
    with K = G M mu m_u / (k_B r T0), which exercises both the gravity term and the 1/T factor."""
    T0 = 400.0

    def closed(rf, tf, th):
        rc = 0.5 * (rf[0] + rf[1])
        K = H.G_CGS * 2.5 * H.M_SUN * 2.3 * H.M_U / (H.K_B * rc * T0)
        return np.sin(th) ** (K + 1.0)

    e1 = _profile_error(400, lambda th: T0 / np.sin(th), closed)
    e2 = _profile_error(800, lambda th: T0 / np.sin(th), closed)
    assert e1 < 5e-3
    assert 3.0 < e1 / e2 < 5.0


def test_shell_mass_kept_and_empty_cells_stay_empty():
    rng = np.random.default_rng(5)
    rf = AU * np.geomspace(0.5, 5.0, 9)
    tf = np.linspace(0.0, np.pi, 31)
    T = rng.uniform(50, 800, size=(8, 30))
    mask = np.ones((8, 30), bool)
    mask[:, :3] = mask[:, -3:] = False
    mask[2] = False
    M = rng.uniform(1e24, 1e26, size=8)
    rho = H.hydrostatic_density(rf, tf, mask, T, M)
    got = H.shell_masses(rf, tf, rho)
    ok = np.arange(8) != 2
    assert np.allclose(got[ok], M[ok], rtol=1e-12, atol=0)
    assert np.all(rho[~mask] == 0) and got[2] == 0
    # the density peaks at the midplane for a flat temperature and falls monotonically away from it
    r = H.hydrostatic_density(rf, tf, mask, np.full((8, 30), 2000.0), M)[7]
    up, down = r[3:15], r[15:27]
    assert np.all(np.diff(up[up > 1e-250]) > 0) and np.all(np.diff(down[down > 1e-250]) < 0)
    assert up[-1] > 0 and down[0] > 0


def test_convergence_statistic():
    T = np.array([100.0, 200.0, 300.0, 0.0])
    e = np.array([0.01, 0.01, 0.01, 0.01])
    assert H.convergence(T, e, T, e) == 0.0
    f = 1 + 0.03
    T2 = T * f  # |dT| = 0.03 T against sigma = 0.01 T sqrt(1 + f^2)
    assert abs(H.convergence(T, e, T2, e) - 3.0 / np.sqrt(1 + f * f)) < 1e-12


def test_relaxed_density_limits_and_mass():
    """The damped step: a = 1 gives the Eq. 20 density, a = 0 the current density (both already at the
    shell's mass), a = 1/2 the normalised geometric mean; every shell keeps its mass."""
    from oracle import hydro as H
    d = disks.config_thick_gray(20, 16, 1e4)
    rng = np.random.default_rng(9)
    shell = H.shell_masses(d.r_faces_cm, d.theta_faces, d.rho)
    rc = 0.5 * (d.r_faces_cm[1:] + d.r_faces_cm[:-1])
    T = 200.0 * (rc[:, None] / disks.AU_CM) ** -0.5 * np.exp(0.2 * rng.standard_normal(d.rho.shape))
    rho_h = H.hydrostatic_density(d.r_faces_cm, d.theta_faces, d.rho > 0, T, shell)
    one = H.relaxed_density(d.r_faces_cm, d.theta_faces, d.rho, rho_h, np.ones(d.nr), shell)
    assert np.array_equal(one, rho_h)
    zero = H.relaxed_density(d.r_faces_cm, d.theta_faces, d.rho, rho_h, np.zeros(d.nr), shell)
    ok = (d.rho > 0) & (rho_h > 0)
    assert np.allclose(zero[ok], d.rho[ok], rtol=1e-12, atol=0)
    half = H.relaxed_density(d.r_faces_cm, d.theta_faces, d.rho, rho_h, np.full(d.nr, 0.5), shell)
    with np.errstate(divide="ignore"):
        gm = np.where(ok, np.exp(0.5 * np.log(d.rho) + 0.5 * np.log(rho_h)), 0.0)  # sqrt(rho rho_h) without underflow
    V = H.cell_volumes(d.r_faces_cm, d.theta_faces)
    gm *= (shell / (gm * V).sum(1))[:, None]
    assert np.allclose(half, gm, rtol=1e-12, atol=0)
    for x in (one, zero, half):
        assert np.allclose(H.shell_masses(d.r_faces_cm, d.theta_faces, x), shell, rtol=1e-12, atol=0)
