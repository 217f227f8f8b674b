"""Test helpers: a spawn-started process pool for oracle work, and tensor
conversion.  Only tests import this module."""

from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

import oracle

_POOL = None


def pool():
    """A process pool started with 'spawn' (safe after CUDA was initialised)."""
    global _POOL
    if _POOL is None:
        n = max(1, min(16, len(os.sched_getaffinity(0))))
        _POOL = mp.get_context("spawn").Pool(n)
    return _POOL


def _enc(args):
    n, m, r = args
    return oracle.encrypt(oracle.PublicKey(n), m, r)


def _dec(args):
    p, q, c = args
    return oracle.decrypt(oracle.PrivateKey(p, q), c)


def _dec_crt(args):
    p, q, c = args
    return oracle.decrypt_crt(oracle.PrivateKey(p, q), c)


def _prod(args):
    n, cts = args
    pub = oracle.PublicKey(n)
    acc = 1  # the empty cell
    for c in cts:
        acc = oracle.add(pub, acc, c)
    return acc


def oracle_products_many(n: int, groups):
    """The oracle's homomorphic sum (product mod n^2) of each list of ciphertexts."""
    return pool().map(_prod, [(n, [int(c) for c in g]) for g in groups], chunksize=4)


def _cells(args):
    folder, n, cells = args
    cts = np.load(os.path.join(folder, "cts.npy"), mmap_mode="r")  # [2][M] rows of 2L limbs
    bins = np.load(os.path.join(folder, "bins.npy"), mmap_mode="r")  # [F][M]
    nodes = np.load(os.path.join(folder, "nodes.npy"), mmap_mode="r")  # [levels][M]
    M = bins.shape[1]
    pub = oracle.PublicKey(n)
    out = []
    for lvl, v, f, b, k in cells:
        acc = 1  # the empty cell
        for i in np.flatnonzero((bins[f] == b) & (nodes[lvl] == v)):
            acc = oracle.add(pub, acc, int.from_bytes(np.ascontiguousarray(cts[k * M + i]).astype("<u4").tobytes(),
                                                      "little"))
        out.append(acc)
    return out


def oracle_cells_many(folder: str, n: int, cts, bins, nodes, cells, chunk: int = 32):
    """The oracle's encrypted-histogram cell (product mod n^2 of the g or h
    ciphertexts of the samples in node v with bin b of feature f) for every
    (level, v, f, b, k) of `cells`.  cts [2M][2L] uint32, bins [F][M], nodes
    [levels][M] go to the workers as memory-mapped files under `folder`."""
    np.save(os.path.join(folder, "cts.npy"), np.ascontiguousarray(cts, dtype=np.uint32))
    np.save(os.path.join(folder, "bins.npy"), np.ascontiguousarray(bins))
    np.save(os.path.join(folder, "nodes.npy"), np.ascontiguousarray(nodes, dtype=np.int32))
    parts = [(folder, n, cells[i:i + chunk]) for i in range(0, len(cells), chunk)]
    return [c for part in pool().map(_cells, parts, chunksize=1) for c in part]


def sample_cells(rng, levels, F: int, K: int, per_level: int):
    """Distinct (level, v, f, b, k) cells, `per_level` of each listed level
    (all of a level's cells if it has fewer)."""
    out = []
    for lvl in levels:
        total = (1 << lvl) * F * K * 2
        for c in sorted(rng.choice(total, size=min(per_level, total), replace=False).tolist()):
            v, rest = divmod(c, F * K * 2)
            f, rest = divmod(rest, K * 2)
            b, k = divmod(rest, 2)
            out.append((lvl, v, f, b, k))
    return out


def oracle_encrypt_many(n: int, ms, rs):
    return pool().map(_enc, [(n, int(m), int(r)) for m, r in zip(ms, rs)], chunksize=8)


def oracle_decrypt_many(p: int, q: int, cs, crt: bool = False):
    return pool().map(_dec_crt if crt else _dec, [(p, q, int(c)) for c in cs], chunksize=8)


def limbs(arr) -> list:
    a = np.ascontiguousarray(np.asarray(arr)).view(np.uint32)
    return [int.from_bytes(a[i].astype("<u4").tobytes(), "little") for i in range(a.shape[0])]
