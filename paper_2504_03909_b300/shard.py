"""One secure-histogram job split over the ranks of a torch.distributed group.

The paper's parties are distributed workers (Sec. II.A); the vertical secure
step of Sec. III.B is "the active party encrypts g/h, every passive party
accumulates the ciphertexts of its own features by bin, the active party
decrypts".  Over N GPUs of one node that step splits with exactly one
exchange:

* encryption: rank k encrypts the g and h of samples [k M / N, (k + 1) M / N)
  (the active party's share of the M x 2 encryptions of Sec. III.C);
* exchange: an all-gather of the ciphertext rows, so that every rank holds
  every encrypted g and h (the hand-off from the active to the passive
  parties; in the paper a gRPC message);
* aggregation: rank k builds the histograms of its own features
  [k F / N, (k + 1) F / N) over all M samples (passive parties own disjoint
  feature sets, Table II), so no histogram crosses ranks;
* decryption: rank k decrypts the cells it aggregated; the decrypted sums
  (F x K x 2 integers, a few hundred kilobytes) are gathered at the end.

The compute steps are passed in (``ops``), so that the same partition and
merge code drives the CUDA kernels over NCCL in ``bench.py`` and plain CPU
arithmetic over gloo in the tests.  Nothing here does Paillier arithmetic.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import Callable


def block_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """[lo, hi) of rank `rank` when n units are split in contiguous blocks over
    `world` ranks (sizes differ by at most one; the first n mod world ranks take
    the larger blocks)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n >= 0")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


@dataclass
class LevelOps:
    """The compute steps of one level, on whatever device the tensors live.

    encrypt(g_lo_hi: (lo, hi)) -> ct rows [2, hi - lo, 2L] (g rows then h rows)
    prepare(ct [2, M, 2L]) -> the aggregation's form of the ciphertexts
    aggregate(ctm, f_lo, f_hi) -> (hist [nodes, f_hi - f_lo, K, 2, 2L], count)
    decrypt(hist) -> sums [nodes, f_hi - f_lo, K, 2] (int64)
    empty_rows(rows) -> an uninitialised ct tensor [2, rows, 2L] on the exchange device
    """
    encrypt: Callable
    prepare: Callable
    aggregate: Callable
    decrypt: Callable
    empty_rows: Callable


def gather_rows(dist, local, M: int, world: int):
    """All-gather of the ranks' ciphertext blocks [2, m_k, 2L] into [2, M, 2L]
    (blocks padded to the largest block, so that every rank sends the same
    number of bytes; the padding is dropped on assembly)."""
    import torch
    width = local.shape[-1]
    blk = block_range(M, world, 0)[1]  # the largest block
    pad = torch.zeros((2, blk, width), dtype=local.dtype, device=local.device)
    pad[:, :local.shape[1]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    out = torch.empty((2, M, width), dtype=local.dtype, device=local.device)
    for k in range(world):
        lo, hi = block_range(M, world, k)
        out[:, lo:hi] = parts[k][:, :hi - lo]
    return out


def gather_features(dist, local, F: int, world: int):
    """All-gather of the ranks' decrypted feature blocks [nodes, f_k, K, 2] into
    [nodes, F, K, 2] (padded like gather_rows)."""
    import torch
    blk = block_range(F, world, 0)[1]
    shp = list(local.shape)
    shp[1] = blk
    pad = torch.zeros(shp, dtype=local.dtype, device=local.device)
    pad[:, :local.shape[1]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    shp[1] = F
    out = torch.empty(shp, dtype=local.dtype, device=local.device)
    for k in range(world):
        lo, hi = block_range(F, world, k)
        out[:, lo:hi] = parts[k][:, :hi - lo]
    return out


def run_level(ops: LevelOps, dist, world: int, rank: int, M: int, F: int, gather_sums: bool = True):
    """One sharded level step.  Returns (sums, counts, (f_lo, f_hi)): the
    decrypted sums of every feature when gather_sums (else of this rank's
    features only) and this rank's counts."""
    s_lo, s_hi = block_range(M, world, rank)
    f_lo, f_hi = block_range(F, world, rank)
    local = ops.encrypt((s_lo, s_hi))
    # with a process group the exchange runs even on one rank (the same code path)
    ct = gather_rows(dist, local, M, world) if dist is not None else local
    ctm = ops.prepare(ct)
    hist, count = ops.aggregate(ctm, f_lo, f_hi)
    sums = ops.decrypt(hist)
    if gather_sums and dist is not None:
        sums = gather_features(dist, sums, F, world)
    return sums, count, (f_lo, f_hi)
