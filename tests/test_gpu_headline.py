"""The production FP32 MRW transport on the benchmark disk itself (200x120 rim-refined, gray, tau_mid = 1e6,
gamma = 2, 1e6-event cap), as the benchmark runs it: no packet may trip a step guard, and the packet and
energy bookkeeping is exact."""
import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

pytestmark = pytest.mark.gpu

# Packet 1306294732 of seed 1 reached the inner radius moving along it (p.u / r = +6e-9); in FP32 p.u
# rounded to a negative value and |p| onto the face, so it stepped between cell 0 and the inner cavity
# without moving until the guard of 1e5 crossings without an interaction dropped it (FP32, single lane).
TANGENT_PACKET = 1306294732


@pytest.fixture(scope="module")
def M():
    from paper_0902_3092_gb300 import build, mcrt
    build.build()
    mcrt.lib()
    return mcrt


@pytest.fixture(scope="module")
def disk():
    return disks.config_thick_gray(200, 120, 1e6)


def test_recorded_tangent_packet_escapes(M, disk):
    """The packet alone, run by the transport kernel without the tail kernel (where it was dropped): it
    must end (escape or the event cap) with no step-guard flag."""
    g = M.Disk.from_model(disk)
    st = g.run_photons(1, seed=1, first_id=TANGENT_PACKET, n_total=10 ** 8, mrw=True, gamma=2.0, want_sed=True,
                       max_events=10 ** 6, tail_warps=-1)
    g.close()
    assert st["error_flags"] == 0 and st["guarded"] == 0
    assert st["escaped"] + st["capped"] == 1 and st["crossings"] < 10_000


def test_headline_disk_beyond_the_benchmark_ids(M, disk):
    """1e8 packets with ids 2.5e9 .. 2.6e9 (past every id the 25-step benchmark uses): status OK, no step
    guard, every packet escaped or capped at the event cap, the tallies grew by exactly the deposit sum,
    and the capped fraction is the small one of the 1e6-event cap (~1e-5)."""
    g = M.Disk.from_model(disk)
    n = 10 ** 8
    st = g.run_photons(n, seed=1, first_id=25 * 10 ** 8, n_total=n, mrw=True, gamma=2.0, want_sed=True,
                       max_events=10 ** 6)
    t, v, a = g.tallies()
    blob = np.frombuffer(g.checkpoint(), np.uint64)  # header, tally, visits, absorptions, escape counts
    nc = disk.nr * disk.ntheta
    sed = blob[8 + 3 * nc:8 + 3 * nc + disk.opacity.nlam * 10]
    g.close()
    assert st["error_flags"] == 0 and st["guarded"] == 0, (st["guard_packet"], st["guard_kind"], st["guard_cell"])
    assert st["packets"] == n and st["escaped"] + st["capped"] == n
    assert int(t.astype(np.uint64).sum(dtype=np.uint64)) == st["deposit_sum"]
    assert st["capped"] < 1e-4 * n
    assert st["mrw_jumps"] > 0
    assert int(sed.sum()) == st["escaped"]
