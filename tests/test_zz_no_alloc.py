"""mcrt_pda_solve_static: the PDA solve for callers that may not allocate device memory while running
(their device memory is owned by a pool or fixed at start-up). It must give the same temperatures as
mcrt_solve_pda, and the oracle's sparse direct solve, call after call, from one fixed scratch array.

The system (PDA mask, face conductances, boundary values) is assembled here with the CPU reference's
own assembly routines and handed over in torch device buffers; mcrt_solve_pda assembles the same
system inside the library from the same Monte Carlo state."""
import numpy as np
import pytest

import mcstate as S
from paper_0902_3092_gb300 import disks

pytestmark = pytest.mark.gpu


def _state(d):
    """Monte Carlo state (tallies, visit counts) with a PDA band around the midplane."""
    n_total = 10 ** 6
    tally, visits = S.state_for(d, S.wanted_T(d), S.midplane_band(d), n_total)
    return tally, visits, n_total


def test_static_scratch_solve_matches_solve_pda(oracle):
    torch = pytest.importorskip("torch")
    from paper_0902_3092_gb300 import build, mcrt
    build.build()
    d = disks.config_plain_gray(24, 20, 1e6)
    tally, visits, n_total = _state(d)

    # existing entry point: the library assembles and solves from the Monte Carlo state
    g = mcrt.Disk.from_model(d)
    g.restore(S.blob(d, tally, visits, n_total))
    g.solve_pda()
    T_ref, _, _ = g.temperatures(mcrt.T_PDA)
    g.close()

    # the same system for the no-allocation entry point
    r = oracle.Run(d)
    r.tally[:] = tally
    r.n_total = n_total
    T_mc, err = r.temperatures()
    pda = oracle.pda_mask(d, visits.reshape(d.rho.shape), err)
    fixed = oracle.dirichlet_mask(d, pda, tally)
    kR = oracle.rosseland_chi(d, 0.0)
    with np.errstate(divide="ignore", over="ignore"):  # (near-empty cells: D overflows to inf, as in the oracle)
        D = np.where(d.rho > 0, 1.0 / (3.0 * d.rho * kR), 0.0)
    Cr, Ct = oracle.conductances(d, D, pda | fixed)
    Cr_full = np.zeros(d.rho.shape)
    Cr_full[:-1] = Cr
    Ct_full = np.zeros(d.rho.shape)
    Ct_full[:, :-1] = Ct
    mask = np.where(pda, 2, np.where(fixed, 1, 0)).astype(np.int8)
    u0 = np.where(fixed, T_mc ** 4, 0.0)
    assert pda.sum() > 20
    To, mo, _, _ = oracle.solve_pda(d, T_mc, tally, visits, err)
    assert np.array_equal(mo, pda)

    dev = torch.device("cuda:0")
    t_mask = torch.from_numpy(mask.ravel()).to(dev)
    t_cr = torch.from_numpy(Cr_full.ravel()).to(dev)
    t_ct = torch.from_numpy(Ct_full.ravel()).to(dev)
    for call in range(2):  # two calls in a row share the scratch array
        t_u = torch.from_numpy(u0.ravel().copy()).to(dev)
        torch.cuda.synchronize()
        it = mcrt.pda_solve_static(d.nr, d.ntheta, t_mask.data_ptr(), t_cr.data_ptr(), t_ct.data_ptr(),
                                   t_u.data_ptr(), device=0)
        u = t_u.cpu().numpy().reshape(d.rho.shape)
        assert it > 0
        T = np.where(pda, np.maximum(u, 0.0) ** 0.25, T_mc)
        assert np.max(np.abs(T[pda] / T_ref[pda] - 1)) < 1e-6, call
        assert np.max(np.abs(T[pda] / To[pda] - 1)) < 1e-6, call
        assert np.array_equal(u[~pda], u0[~pda])
    # a third call from a starting guess far from the solution: the tolerance is relative to the
    # right-hand side, not to the first residual, so it lands on the same solution
    guess = np.where(pda, 3.0 * u, u0)
    t_u = torch.from_numpy(guess.ravel().copy()).to(dev)
    torch.cuda.synchronize()
    mcrt.pda_solve_static(d.nr, d.ntheta, t_mask.data_ptr(), t_cr.data_ptr(), t_ct.data_ptr(), t_u.data_ptr(),
                          device=0)
    u3 = t_u.cpu().numpy().reshape(d.rho.shape)
    T3 = np.where(pda, np.maximum(u3, 0.0) ** 0.25, T_mc)
    assert np.max(np.abs(T3[pda] / To[pda] - 1)) < 1e-6
    assert torch.cuda.current_device() == 0


def test_static_scratch_size_limit():
    pytest.importorskip("torch")
    from paper_0902_3092_gb300 import build, mcrt
    build.build()
    with pytest.raises(mcrt.McrtError) as e:
        mcrt.pda_solve_static(400, 400, 1, 1, 1, 1, device=0)  # 160000 cells > 131072
    assert e.value.status == 1
    assert b"131072" in mcrt.lib().mcrt_last_error(None)
