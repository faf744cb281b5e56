"""Differentiable PDA (torch.autograd.Function over the CUDA adjoint) on the 400 x 200, tau_mid = 1e6
non-gray disk: d(mean midplane T)/d(log rho, kappa_R) against the FP64 oracle's adjoint and against
central finite differences on 50 random cells (seed 1).

Both sides start from one synthetic Monte Carlo state, restored into the disk: no entries in the
~11,000 cells deeper than 100 optical depths from the nearer pole (the PDA region of a long run on
this disk has ~12,000), and tallies for a smooth temperature field in the thick cells around them.
The Rosseland opacity is a seeded field, log-uniform within a factor e^0.5 of 26 cm^2/g (this dust's
Rosseland mean near 100 K), given to both sides. The PDA threshold is 3000 entries, as for the
1e7-packet runs (Sect. 3.1)."""
import numpy as np
import pytest

import mcstate as S
from paper_0902_3092_gb300 import disks

pytestmark = pytest.mark.gpu
MINV = 3000
N_TOTAL = 10_000_000


@pytest.fixture(scope="module")
def setup(oracle):
    torch = pytest.importorskip("torch")
    from paper_0902_3092_gb300 import build, mcrt
    build.build()
    d = disks.config_pda_adjoint(400, 200, 1e6)
    t, v = S.state_for(d, S.wanted_T(d), S.deep_band(d, 100.0), N_TOTAL)
    kR = 26.0 * np.exp(np.random.default_rng(7).uniform(-0.5, 0.5, d.rho.shape))
    g = mcrt.Disk.from_model(d)
    g.restore(S.blob(d, t, v, N_TOTAL))
    r = oracle.Run(d)
    r.tally[:] = t
    r.n_total = N_TOTAL
    T_mc, err = r.temperatures()
    To, mo, uo, info = oracle.solve_pda(d, T_mc, t, v, err, min_visits=MINV, kappa_R=kR)
    return torch, mcrt, d, g, kR, (To, mo, uo, info)


def midplane_weights(d):
    w = np.zeros((d.nr, d.ntheta))
    j = d.ntheta // 2
    w[:, j - 1:j + 1] = 1.0 / (2 * d.nr)
    return w


def test_forward_matches_oracle(setup):
    torch, mcrt, d, g, kR, (To, mo, uo, info) = setup
    from paper_0902_3092_gb300.pda_torch import pda_temperature
    assert mo.sum() > 10_000
    lr = torch.tensor(np.log(np.where(d.rho > 0, d.rho, 1.0)), dtype=torch.float64, device="cuda")
    kr = torch.tensor(kR, dtype=torch.float64, device="cuda")
    T = pda_temperature(g, lr, kr, min_visits=MINV).cpu().numpy()
    assert np.max(np.abs(T[mo] / To[mo] - 1)) < 1e-6


def test_gradient_matches_oracle_adjoint(setup, oracle):
    torch, mcrt, d, g, kR, (To, mo, uo, info) = setup
    from paper_0902_3092_gb300.pda_torch import pda_temperature
    w = midplane_weights(d)
    lr = torch.tensor(np.log(np.where(d.rho > 0, d.rho, 1.0)), dtype=torch.float64, device="cuda",
                      requires_grad=True)
    kr = torch.tensor(kR, dtype=torch.float64, device="cuda", requires_grad=True)
    J = (pda_temperature(g, lr, kr, min_visits=MINV) * torch.tensor(w, device="cuda")).sum()
    J.backward()
    gl, gk = lr.grad.cpu().numpy(), kr.grad.cpu().numpy()
    ol, ok_, _ = oracle.pda_adjoint(d, uo, mo, info, w)
    assert np.abs(ol).max() > 0
    assert np.max(np.abs(gl - ol)) <= 1e-6 * np.abs(ol).max()
    assert np.max(np.abs(gk - ok_)) <= 1e-6 * np.abs(ok_).max()


def test_gradient_against_finite_differences(setup):
    torch, mcrt, d, g, kR, (To, mo, uo, info) = setup
    from paper_0902_3092_gb300.pda_torch import pda_temperature
    w = midplane_weights(d)
    wt = torch.tensor(w, device="cuda")
    lr0 = np.log(np.where(d.rho > 0, d.rho, 1.0))
    kr0 = kR.copy()

    def J(lr, kr):
        with torch.no_grad():
            T = pda_temperature(g, torch.tensor(lr, device="cuda"), torch.tensor(kr, device="cuda"), min_visits=MINV)
            return float((T * wt).sum())

    lr = torch.tensor(lr0, device="cuda", requires_grad=True)
    kr = torch.tensor(kr0, device="cuda", requires_grad=True)
    (pda_temperature(g, lr, kr, min_visits=MINV) * wt).sum().backward()
    gl, gk = lr.grad.cpu().numpy(), kr.grad.cpu().numpy()
    cand = np.argwhere(np.abs(gl) > 1e-3 * np.abs(gl).max())
    assert len(cand) >= 50
    rng = np.random.default_rng(1)
    pick = cand[rng.choice(len(cand), size=min(50, len(cand)), replace=False)]
    # central differences: O(h^2) truncation plus the solve's FP64 residual floor divided by h, hence
    # 5e-4 relative (and 1e-6 of the largest component for the smallest ones)
    h = 1e-3
    for i, j in pick:
        a, b = lr0.copy(), lr0.copy()
        a[i, j] += h
        b[i, j] -= h
        fd = (J(a, kr0) - J(b, kr0)) / (2 * h)
        assert abs(fd - gl[i, j]) <= 5e-4 * abs(gl[i, j]) + 1e-6 * np.abs(gl).max(), (i, j, fd, gl[i, j])
        a, b = kr0.copy(), kr0.copy()
        hk = h * kr0[i, j]
        a[i, j] += hk
        b[i, j] -= hk
        fdk = (J(lr0, a) - J(lr0, b)) / (2 * hk)
        assert abs(fdk - gk[i, j]) <= 5e-4 * abs(gk[i, j]) + 1e-6 * np.abs(gk).max(), (i, j, fdk, gk[i, j])
