"""Batched transport (many disks, one persistent launch, CUDA graph replay, autotuned launch shape)."""
import math

import numpy as np
import pytest

from paper_0902_3092_gb300 import disks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_0902_3092_gb300 import build, mcrt
    build.build()
    mcrt.lib()
    return mcrt


def test_first_model_equals_single_disk_run(M):
    """Model 0 of a batch uses the same Philox counters as mcrt_run_photons, and the integer tallies do
    not depend on the order in which packets deposit: bitwise equal for gray dust."""
    a = disks.config_plain_gray(20, 20, 100.0)
    b = disks.config_nongray(30, 24, 1e3)
    c = disks.config_thick_gray(40, 30, 1e4)
    ga, gb, gc = M.Disk.from_model(a), M.Disk.from_model(b), M.Disk.from_model(c)
    # without the tail kernel (its batched interactions sum positions in another floating-point order)
    B = M.Batch([ga, gb, gc], [60_000, 40_000, 30_000], mrw=True, gamma=2.0, max_events=10 ** 6, tail_warps=-1)
    cfg = B.config()
    assert cfg["block_size"] in (64, 128, 256) and cfg["refill_interval"] in (1, 4, 16)  # the tuner's candidates
    st = B.run(seed=5)
    for s, n in zip(st, (60_000, 40_000, 30_000)):
        assert s["packets"] == n and s["escaped"] + s["capped"] == n and s["error_flags"] == 0
    for g in (ga, gb, gc):
        t, _, _ = g.tallies()
    single = M.Disk.from_model(a)
    # without the tail kernel: its batched interactions sum positions in another floating-point order
    single.run_photons(60_000, seed=5, mrw=True, gamma=2.0, max_events=10 ** 6, tail_warps=-1)
    for x, y in zip(ga.tallies(), single.tallies()):
        assert np.array_equal(x, y)
    # sum of tallies equals the sum of per-packet deposits in every model
    for g, s in zip((ga, gb, gc), st):
        t, _, _ = g.tallies()
        assert int(t.sum()) == s["deposit_sum"]
    B.close()


def test_replay_with_new_seed(M, oracle):
    """Replays accumulate; a new seed gives new streams; model 1 matches the oracle run with model id 1
    statistically (gray dust, same Philox counters)."""
    a = disks.config_plain_gray(16, 16, 100.0)
    b = disks.config_plain_gray(16, 16, 300.0)
    ga, gb = M.Disk.from_model(a), M.Disk.from_model(b)
    B = M.Batch([ga, gb], [200_000, 200_000], block_size=256, refill=4, tail_warps=-1)  # bitwise replays
    assert B.config()["block_size"] == 256
    B.run(seed=1)
    t1, _, _ = gb.tallies()
    gb.reset()
    ga.reset()
    B.run(seed=2)
    t2, _, _ = gb.tallies()
    assert not np.array_equal(t1, t2)
    gb.reset()
    B.run(seed=1)
    t3, v3, n3 = gb.tallies()
    assert np.array_equal(t1, t3)
    ref = oracle.Run(b).run(200_000, seed=1, model_id=1, want_sed=False)
    T, _, _ = gb.temperatures()
    To, _ = ref.temperatures()
    sel = n3.reshape(T.shape) >= 1000
    assert sel.sum() >= 5
    assert np.max(np.abs(T[sel] / To[sel] - 1)) < 0.02
    B.close()


def test_sweep_of_64_models(M):
    """The batched sweep: 64 models of uneven size, optical depth and packet budget (budgets scaled by
    1/100 to keep the test short), one autotuned graph launch; every model conserves packets."""
    ds, npk = disks.batch_sweep(64, seed=1)
    npk = [max(1000, n // 100) for n in npk]
    gs = [M.Disk.from_model(d) for d in ds]
    B = M.Batch(gs, npk, mrw=True, gamma=2.0, max_events=10 ** 5)
    for seed in (1, 2):  # a new seed updates both kernel nodes of the graph (transport and tail)
        for g in gs:
            g.reset()
        st = B.run(seed=seed)
        for g, s, n in zip(gs, st, npk):
            assert s["packets"] == n and s["escaped"] + s["capped"] == n
            assert s["error_flags"] == 0
            t, _, _ = g.tallies()
            assert int(t.sum(dtype=np.uint64)) == s["deposit_sum"]  # every deposit reached its model's tallies
    B.close()


def test_batch_model_with_sources_equals_single_disk_run(M):
    """A batched model that carries internal sources (viscous heating) draws its source choices from
    the same Philox counters as a single-disk run: bitwise equal gray tallies (without the tail kernel)."""
    a = disks.config_plain_gray(20, 20, 100.0)
    L = disks.viscous_sources(a)
    L *= 3.0 * a.star.L / L.sum()
    ga = M.Disk.from_model(a)
    ga.set_sources(L)
    gb = M.Disk.from_model(disks.config_nongray(30, 24, 1e3))
    B = M.Batch([ga, gb], [50_000, 30_000], mrw=True, gamma=2.0, max_events=10 ** 6, tail_warps=-1)
    st = B.run(seed=5)
    assert st[0]["packets"] == 50_000 and st[0]["escaped"] + st[0]["capped"] == 50_000
    single = M.Disk.from_model(a)
    single.set_sources(L)
    single.run_photons(50_000, seed=5, mrw=True, gamma=2.0, max_events=10 ** 6, tail_warps=-1)
    for x, y in zip(ga.tallies(), single.tallies()):
        assert np.array_equal(x, y)
    t, _, _ = ga.tallies()
    assert int(t.sum()) == st[0]["deposit_sum"]
    B.close()


def test_warp_wide_mrw_chains_equal_per_lane_chains(M):
    """A single gray FP32 disk's transport kernel makes the MRW chains of its lanes warp-wide (the random
    blocks of every chaining lane computed by the 32 lanes together, each lane's jumps read from the lanes
    that hold its blocks); the batch kernel makes each lane's chain alone. Same Philox counters, same
    arithmetic per jump: without the tail kernel, tallies, entries and absorption counts are bitwise equal,
    on a disk where MRW jumps are a large share of the events (Sect. 2.2.2, Eq. 9-11)."""
    d = disks.config_thick_gray(100, 60, 1e5)
    single = M.Disk.from_model(d)
    st = single.run_photons(200_000, seed=7, mrw=True, gamma=2.0, max_events=10 ** 6, tail_warps=-1, want_sed=False)
    assert st["mrw_jumps"] > 0.1 * st["events"], (st["mrw_jumps"], st["events"])
    g = M.Disk.from_model(d)
    B = M.Batch([g], [200_000], mrw=True, gamma=2.0, max_events=10 ** 6, tail_warps=-1, want_sed=False)
    (sb,) = B.run(seed=7)
    assert sb["mrw_jumps"] == st["mrw_jumps"] and sb["events"] == st["events"]
    for x, y in zip(single.tallies(), g.tallies()):
        assert np.array_equal(x, y)
    B.close()
    single.close()
    g.close()
