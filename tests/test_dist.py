"""Multi-rank host logic on the CPU (gloo, world size 2): each rank runs the oracle on its own packet
range; the integer all-reduce of their checkpoint blobs equals one run over all packets, bitwise."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _sources(d):
    from paper_0902_3092_gb300 import disks
    L = disks.viscous_sources(d)
    return L * (2.0 * d.star.L / L.sum())


def _rank(rank, world, port, out, with_sources=False):
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_0902_3092_gb300 import disks
    from paper_0902_3092_gb300 import dist as D
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = disks.config_plain_gray(12, 12, 50.0)
    per = 1500
    first, n = D.packet_range(rank, world, per)
    src = _sources(d) if with_sources else None
    r = O.Run(d, sources=src).run(n, seed=3, first_id=first, n_total=per * world, want_sed=True)
    blob = D.make_blob(d.nr, d.ntheta, d.opacity.nlam, r.tally, r.visits, r.nabs, r.sed, n, per * world)
    red = D.allreduce_blob(blob)
    if rank == 0:
        out.put(red)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("with_sources", [False, True])
def test_two_rank_tally_allreduce_is_exact(with_sources):
    """Also with internal sources (viscous heating): the source choices come from each packet's own
    counter-based stream, so sharding by packet id changes nothing."""
    from oracle import oracle as O
    from paper_0902_3092_gb300 import disks
    from paper_0902_3092_gb300 import dist as D
    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q, with_sources)) for r in range(2)]
    for p in ps:
        p.start()
    red = q.get(timeout=120)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    hdr, body = D.split_blob(red)
    d = disks.config_plain_gray(12, 12, 50.0)
    ref = O.Run(d, sources=_sources(d) if with_sources else None).run(3000, seed=3, first_id=0, n_total=3000,
                                                                         want_sed=True)
    n = d.nr * d.ntheta
    assert int(hdr[5]) == 3000
    assert np.array_equal(body[:n], ref.tally)
    assert np.array_equal(body[n:2 * n], ref.visits)
    assert np.array_equal(body[2 * n:3 * n], ref.nabs)
    # the BW wavelength depends on the tally seen at absorption time, so only totals of the spectrum agree
    assert int(body[3 * n:].sum()) == int(ref.sed.sum())


def test_packet_ranges_partition():
    from paper_0902_3092_gb300 import dist as D
    seen = set()
    for step in range(3):
        for rank in range(4):
            f, n = D.packet_range(rank, 4, 100, step)
            ids = set(range(f, f + n))
            assert not (ids & seen)
            seen |= ids
    assert seen == set(range(1200))
