"""Host logic of multi-GPU runs: one rank per GPU transports its own packet range with the same Philox
key; the Monte Carlo step then has one exchange, an exact integer sum of the tallies, visit counts,
absorption counts and escape spectrum over the ranks, before temperatures and the PDA.

The tallies travel as checkpoint blobs (the layout of mcrt_checkpoint: 8 uint64 header words, then
tally, visits, absorptions per cell and the spectrum counts), so the exchange is independent of where
the tallies live; with gray dust the summed state is bitwise that of a single run over all packets.

Each rank transports its share as a run of its own: n_total = its own packet count. The tallies count
packet energies, so that choice only sets the temperatures seen during the rank's run -- those of its own
tallies, which decide the Bjorkman-Wood re-emission spectra and the MRW coefficients of non-gray dust. A
rank whose share were weighed as 1/k of the whole run would see temperatures low by k^(1/4) and re-emit
at the wrong temperature. The exchange then rewrites the header to the total packet count, so the summed
state is k independent BW runs added together, read with the packet energy of the whole run.
"""
from __future__ import annotations

import numpy as np

MAGIC = 0x4D43525443484B31
HEADER_WORDS = 8


def packet_range(rank: int, world: int, per_rank: int, step: int = 0):
    """First packet id and count of `rank` in step `step` (ranks interleaved, steps consecutive)."""
    return (rank + world * step) * per_rank, per_rank


def _n_total_word(n_total: float) -> np.uint64:
    return np.frombuffer(np.array([float(n_total)]).tobytes(), np.uint64)[0]


def make_blob(nr, nt, nlam, tally, visits, nabs, sed, packets_done, n_total) -> bytes:
    hdr = np.array([MAGIC, 1, nr, nt, nlam, packets_done, _n_total_word(n_total), 0], np.uint64)
    parts = [hdr] + [np.ascontiguousarray(a, np.uint64).ravel() for a in (tally, visits, nabs, sed)]
    return np.concatenate(parts).tobytes()


def split_blob(blob: bytes):
    a = np.frombuffer(blob, np.uint64)
    hdr = a[:HEADER_WORDS]
    if int(hdr[0]) != MAGIC:
        raise ValueError("not a checkpoint blob")
    return hdr.copy(), a[HEADER_WORDS:].copy()


def combine_blobs(blobs) -> bytes:
    """The exchange without a process group: the integer states of several ranks' blobs summed, the header
    carrying the total packet count (what allreduce_blob leaves on every rank)."""
    hdrs, bodies = zip(*(split_blob(b) for b in blobs))
    hdr = hdrs[0].copy()
    body = np.sum(np.stack(bodies), axis=0, dtype=np.uint64)
    n = int(sum(int(h[5]) for h in hdrs))
    hdr[5] = n
    hdr[6] = _n_total_word(float(n))
    return hdr.tobytes() + body.tobytes()


def allreduce_blob(blob: bytes, group=None) -> bytes:
    """Sums the integer state of all ranks (torch.distributed, exact in int64: every tally stays below
    2^63). The header's packet counts become the totals of all ranks."""
    import torch
    import torch.distributed as dist
    hdr, body = split_blob(blob)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    x = torch.from_numpy(body.view(np.int64).copy()).to(dev)
    n = torch.tensor([int(hdr[5])], dtype=torch.int64, device=dev)
    dist.all_reduce(x, group=group)
    dist.all_reduce(n, group=group)
    hdr[5] = int(n.item())
    hdr[6] = _n_total_word(float(n.item()))
    return hdr.tobytes() + x.cpu().numpy().view(np.uint64).tobytes()
