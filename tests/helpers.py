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


def oracle_encrypt_many(n: int, ms, rs):
    return pool().map(_enc, [(n, int(m), int(r)) for m, r in zip(ms, rs)], chunksize=8)


def oracle_decrypt_many(p: int, q: int, cs, crt: bool = False):
    return pool().map(_dec_crt if crt else _dec, [(p, q, int(c)) for c in cs], chunksize=8)


def limbs(arr) -> list:
    a = np.ascontiguousarray(np.asarray(arr)).view(np.uint32)
    return [int.from_bytes(a[i].astype("<u4").tobytes(), "little") for i in range(a.shape[0])]
