"""Encryption as two launches (first stage mod p and mod q at half the lanes,
second stage mod p^2 and mod q^2) against one fused launch and against the
oracle: plaintexts of one and of two 64-bit words (g/h packing), a call large
enough to take the split path, sampled rows including the ragged tail."""

import numpy as np
import pytest
import torch

import oracle
from paper_2504_03909_b300 import native, paillier as P, synth

from helpers import oracle_encrypt_many

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def key2048():
    p, q = synth.gen_primes(2048, 31)
    return P.Key.from_primes(2048, p, q), p, q


def _sample(count, rng):
    idx = set(rng.choice(count, size=254, replace=False).tolist()) | {count - 2, count - 1}
    return sorted(idx)


@pytest.mark.parametrize("words", [1, 2])
def test_split_equals_fused_and_oracle(key2048, words):
    key, p, q = key2048
    n = p * q
    count = 4001  # ragged: not a multiple of the instances per warp or block
    rng = synth.rng_misc(40 + words)
    r = synth.gen_r(n, 2048, count, 40 + words, p, q)
    r_d = P.to_limb_tensor(r)
    if words == 1:
        ms = [int(x) for x in rng.integers(0, 1 << 62, size=count)]
        m_d = torch.tensor(ms, dtype=torch.int64, device="cuda")
        enc = lambda: P.encrypt(key, m_d, r_d)
    else:
        lo = rng.integers(0, 1 << 62, size=count)
        hi = rng.integers(0, 1 << 30, size=count)
        ms = [int(a) + (int(b) << 64) for a, b in zip(lo, hi)]
        m_d = torch.from_numpy(np.stack([lo, hi], axis=1).astype(np.int64)).cuda()
        enc = lambda: P.encrypt_gh(key, m_d, r_d)
    base = P.get_config(key, native.OP_ENCRYPT)
    assert base[0] == 4  # the configuration that runs as two launches at 2048-bit
    split = enc()
    P.set_config(key, native.OP_ENCRYPT, 8, base[1])  # one fused launch
    fused = enc()
    P.set_config(key, native.OP_ENCRYPT, *base)
    P.sync()
    assert torch.equal(split, fused)
    idx = _sample(count, rng)
    want = oracle_encrypt_many(n, [ms[i] for i in idx], synth.limbs_to_ints(r[idx]))
    assert synth.limbs_to_ints(P.from_limb_tensor(split[idx])) == want
