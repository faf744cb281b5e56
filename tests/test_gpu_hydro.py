"""Vertical hydrostatic structure on the GPU (Sect. 2.5, Eq. 20) against the FP64 oracle, and the
iteration's 3-sigma convergence."""
import numpy as np
import pytest

import mcstate as S
from paper_0902_3092_gb300 import disks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_0902_3092_gb300 import build, mcrt
    build.build()
    mcrt.lib()
    return mcrt


def test_hydrostatic_density_matches_oracle(M, oracle):
    """The same Monte Carlo state on both sides (tallies for a smooth 40-1300 K field in the dusty cells
    heavy enough to hold one tally unit, restored into the disk; the others take T_floor) -> the same
    Eq. 20 density to 1e-9, with the temperatures each side computes from the tallies."""
    from oracle import hydro as H
    d = disks.config_thick_gray(40, 30, 1e4)
    n_total = 200_000
    t, v = S.state_for(d, S.wanted_T(d), np.zeros(d.rho.shape, bool), n_total, thick_only=False)
    g = M.Disk.from_model(d)
    g.restore(S.blob(d, t, v, n_total))
    r = oracle.Run(d)
    r.tally[:] = t
    r.n_total = n_total
    T, _ = r.temperatures()
    assert (T > 0).sum() > 300
    Ms = 2.5 * H.M_SUN
    shell = H.shell_masses(d.r_faces_cm, d.theta_faces, d.rho)
    rho_g = g.hydrostatic_density(M_star_g=Ms, mu=2.3, T_floor=10.0, which=M.T_MC)
    rho_o = H.hydrostatic_density(d.r_faces_cm, d.theta_faces, d.rho > 0, T, shell, M_star=Ms, mu=2.3, T_floor=10.0)
    assert np.array_equal(rho_g > 0, rho_o > 0) or np.all(np.abs(rho_g - rho_o) <= 1e-200)
    big = rho_o > 1e-200 * rho_o.max()
    assert big.sum() > 200
    assert np.max(np.abs(rho_g[big] / rho_o[big] - 1)) < 1e-9
    # the new density keeps every shell's mass, and installing it keeps the shells' masses too
    assert np.allclose(H.shell_masses(d.r_faces_cm, d.theta_faces, rho_g), shell, rtol=1e-12, atol=0)
    g.set_density(rho_g)
    t, v, a = g.tallies()
    assert t.sum() == 0 and v.sum() == 0
    rho_g2 = g.hydrostatic_density(M_star_g=Ms, which=M.T_MC, shell_mass=shell)
    assert np.all(np.isfinite(rho_g2)) and rho_g2.max() > 0


def test_iteration_settles(M):
    """Plain Monte Carlo (whose per-cell error is the counting error the criterion uses): the change of
    the temperatures between iterations, in units of their errors, falls from its first value and the
    driver stops once it is below the threshold. On this small disk it settles near 3-6 sigma (the density
    follows the noisy temperatures of the previous iteration), so the threshold here is 8."""
    from paper_0902_3092_gb300 import hydro
    d = disks.config_thick_gray(40, 30, 1e3)
    _, hist = hydro.iterate(d, 100_000, max_iter=12, seed=7, mrw=False, tol_sigma=8.0)
    changes = [h["change_sigma"] for h in hist]
    assert len(hist) >= 2 and changes[-1] < 8.0, changes
    assert len(hist) < 12  # stopped by the criterion
    assert all(h["transport_s"] > 0 for h in hist)
