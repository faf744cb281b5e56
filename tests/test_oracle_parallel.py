"""Pins of the oracle's packet-parallel mode (oracle_run_par): the same packets on several host threads,
shared atomic energy tallies, per-thread counts summed at the end.

Gray dust: the trajectories do not depend on the temperatures (Sect. 2.1: the wavelength only shapes the
escape spectrum, and gray re-emission is isotropic whatever the temperature), and the tallies are integer
sums, so a parallel run must equal the serial run bit for bit -- energy tallies, entries, absorptions,
counters and the escapes per inclination -- with MRW (Sect. 2.2.2) and with internal sources (Sect. 5).
Only the wavelength bins of the escapes differ: they come from the re-emission temperatures, which
depend on the order of the deposits. Non-gray dust: each re-emission sees the tally its
own deposit followed, which other threads move, so the histories fork; the integer bookkeeping must stay
exact (every packet escapes or is capped, the summed deposits equal the tallies) and the temperatures must
agree with independent serial runs within their counting errors (1/(4 sqrt N) per cell, Sect. 3.1; without
the MRW, whose jumps deposit many packet energies at once so that the counting error understates a cell's
scatter -- the gray pins cover the MRW exactly)."""
import numpy as np
import pytest

from oracle import oracle
from paper_0902_3092_gb300 import disks


def _same(a, b):
    for k in ("tally", "visits", "nabs"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    ninc = oracle.NINC
    assert np.array_equal(a.sed.reshape(-1, ninc).sum(0), b.sed.reshape(-1, ninc).sum(0))
    assert a.stats == b.stats


@pytest.mark.parametrize("mrw,sources,want_sed", [(False, False, True), (True, False, True), (True, True, True),
                                                  (True, False, False)])
def test_gray_parallel_run_equals_serial_run(mrw, sources, want_sed):
    """(Without the escape spectrum each thread keeps a tally of its own, added at the end.)"""
    d = disks.make_disk(disks.rim_refined_r_faces(0.1, 100.0, 24), disks.midplane_refined_theta_faces(16),
                        disks.paper_star(), disks.gray_opacity(nlam=20), 3e3)
    L = None
    if sources:
        L = disks.viscous_sources(d)
        L *= 0.5 * d.star.L / L.sum()
    n = 4000
    ser = oracle.Run(d, sources=L).run(n, seed=5, mrw=mrw, gamma=2.0, want_sed=want_sed, max_events=10 ** 5)
    par = oracle.Run(d, sources=L).run(n, seed=5, mrw=mrw, gamma=2.0, want_sed=want_sed, max_events=10 ** 5,
                                       threads=4)
    _same(ser, par)
    assert ser.stats["escaped"] + ser.stats["capped"] == n
    if mrw:
        assert ser.stats["mrw_jumps"] > 0
    # a continued run: the parallel call leaves the cell temperatures of its tallies
    T1, _ = par.temperatures()
    assert np.array_equal(par.Tcell.reshape(T1.shape), T1)


def test_nongray_parallel_run_keeps_exact_bookkeeping_and_agrees_with_serial():
    d = disks.make_disk(disks.log_r_faces(0.1, 100.0, 12), disks.midplane_refined_theta_faces(10),
                        disks.paper_star(), disks.powerlaw_opacity(nlam=16), 3e3)
    n = 20000
    pars = [oracle.Run(d).run(n, seed=11 + k, want_sed=True, threads=4) for k in range(4)]
    for par in pars:
        st = par.stats
        assert st["packets"] == n and st["escaped"] + st["capped"] == n and st["error_flags"] == 0
        assert int(par.tally.sum(dtype=np.uint64)) == st["deposit_sum"]
        assert int(par.sed.sum()) == st["escaped"] and int(par.nabs.sum()) == st["absorptions"]
    # independent serial runs (other seeds) against the parallel ones, cell by cell; the scatter of a cell
    # is measured from the runs themselves (in thick cells one packet is absorbed many times, so the
    # counting error 1/(4 sqrt N) understates it)
    sers = [oracle.Run(d).run(n, seed=31 + k, want_sed=True) for k in range(4)]
    Tp = np.array([r.temperatures()[0] for r in pars])
    Ts = np.array([r.temperatures()[0] for r in sers])
    nab = np.minimum(pars[0].nabs, sers[0].nabs).reshape(Tp.shape[1:])
    sd = np.sqrt((Tp.var(0, ddof=1) + Ts.var(0, ddof=1)) / 2)
    sel = (nab >= 100) & (sd > 0)
    assert sel.sum() >= 6
    z = np.abs(Tp.mean(0)[sel] - Ts.mean(0)[sel]) / (sd[sel] * np.sqrt(2 / 4))
    assert np.max(z) < 5.0, np.sort(z)[-5:]
