"""The sharded level step of paper_2504_03909_b300.shard on CPU: two and three
gloo ranks run the partition (samples for encryption, features for
aggregation and decryption) and the exchange (all-gather of the ciphertext
rows, gather of the decrypted feature blocks) with the oracle doing the
arithmetic on each rank; the merged result must equal the single-rank
result of the same workload bit for bit: every gathered ciphertext row, every
rank's histogram cells, every decrypted sum and count."""

import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2504_03909_b300 import shard, synth  # noqa: E402

M, F, K, N_BITS, SEED, NODES = 91, 5, 8, 1024, 1, 2  # 91 samples: ragged blocks over 2 and 3 ranks


def test_block_range_partitions():
    for n in (0, 1, 5, 30, 250_000, 1_000_001):
        for world in (1, 2, 3, 8):
            parts = [shard.block_range(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in parts]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        shard.block_range(5, 2, 2)


def _workload():
    import oracle
    p, q = synth.gen_primes(N_BITS, SEED)
    pub, priv = oracle.keypair(p, q)
    gh = synth.gen_gh(M, SEED)
    r = synth.limbs_to_ints(synth.gen_r(p * q, N_BITS, 2 * M, SEED, p, q))
    m = [[oracle.encode(x) for x in gh[k]] for k in range(2)]
    bins = synth.gen_bins_uniform(F, M, K, SEED)
    node = synth.gen_tree_levels(M, 2, SEED)[1]
    return pub, priv, m, r, bins, node


def _ops(pub, priv, m, r, bins, node):
    """Oracle-backed compute steps on CPU tensors (int32 limb rows)."""
    import oracle
    L = N_BITS // 32

    def rows(vals, width):
        return torch.from_numpy(synth.ints_to_limbs(vals, width).view(np.int32))

    def ints(t):
        return synth.limbs_to_ints(t.numpy().view(np.uint32).reshape(-1, t.shape[-1]))

    def encrypt(rng_):
        lo, hi = rng_
        out = [rows([oracle.encrypt(pub, m[k][i], r[k * M + i]) for i in range(lo, hi)], 2 * L) for k in range(2)]
        return torch.stack(out)

    def aggregate(ct, f_lo, f_hi):
        cts = [ints(ct[k]) for k in range(2)]
        cells, counts = [], np.zeros((NODES, f_hi - f_lo, K), np.int32)
        for v in range(NODES):
            for f in range(f_lo, f_hi):
                for b in range(K):
                    counts[v, f - f_lo, b] = int(((node == v) & (bins[f] == b)).sum())
                    for k in range(2):
                        cells.append(oracle.encrypted_histogram_cell(pub, cts[k], bins, node, v, f, b))
        hist = rows(cells, 2 * L).view(NODES, f_hi - f_lo, K, 2, 2 * L)
        return hist, torch.from_numpy(counts)

    def decrypt(hist):
        vals = [oracle.decrypt(priv, c) for c in ints(hist.reshape(-1, 2 * L))]
        return torch.tensor(vals, dtype=torch.int64).view(hist.shape[:-1])

    return shard.LevelOps(encrypt=encrypt, prepare=lambda ct: ct, aggregate=aggregate, decrypt=decrypt,
                          empty_rows=lambda n: torch.empty((2, n, 2 * L), dtype=torch.int32))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ops = _ops(*_workload())
    captured = {}
    prepare = ops.prepare

    def keep(ct):
        captured["ct"] = ct.clone()
        return prepare(ct)

    ops.prepare = keep
    aggregate = ops.aggregate

    def keep_hist(ctm, f_lo, f_hi):
        h, c = aggregate(ctm, f_lo, f_hi)
        captured["hist"] = h.clone()
        return h, c

    ops.aggregate = keep_hist
    sums, count, frange = shard.run_level(ops, dist, world, rank, M, F)
    out[rank] = dict(sums=sums.numpy(), count=count.numpy(), frange=frange, ct=captured["ct"].numpy(),
                     hist=captured["hist"].numpy())
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_equal_one_rank(world):
    import oracle
    port = 29600 + (os.getpid() + 7 * world) % 1000
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    # the single-rank job of the same workload
    pub, priv, m, r, bins, node = _workload()
    ops = _ops(pub, priv, m, r, bins, node)
    sums1, count1, _ = shard.run_level(ops, None, 1, 0, M, F)
    ct1 = ops.encrypt((0, M))
    hist1, _ = ops.aggregate(ct1, 0, F)
    for rank in range(world):
        o = out[rank]
        f_lo, f_hi = o["frange"]
        assert (f_lo, f_hi) == shard.block_range(F, world, rank)
        assert np.array_equal(o["ct"], ct1.numpy())                   # every ciphertext row, gathered
        assert np.array_equal(o["hist"], hist1[:, f_lo:f_hi].numpy())  # this rank's cells
        assert np.array_equal(o["sums"], sums1.numpy())               # every decrypted sum, merged
        assert np.array_equal(o["count"], count1[:, f_lo:f_hi].numpy())
    # and the merged sums are the plaintext histogram
    ps, pc = oracle.plain_histogram_np(np.array(m[0], np.int64), np.array(m[1], np.int64), bins, node, NODES, K)
    assert np.array_equal(sums1.numpy(), ps)
