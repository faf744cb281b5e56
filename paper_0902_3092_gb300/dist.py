"""Host logic of multi-GPU runs: one rank per GPU transports its own packet range with the same Philox
key; the Monte Carlo step then has one exchange, an exact integer sum of the tallies, visit counts,
absorption counts and escape spectrum over the ranks, before temperatures and the PDA.

The tallies travel as checkpoint blobs (the layout of mcrt_checkpoint: 8 uint64 header words, then
tally, visits, absorptions per cell and the spectrum counts), so the exchange is independent of where
the tallies live; with gray dust the summed state is bitwise that of a single run over all packets.
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
