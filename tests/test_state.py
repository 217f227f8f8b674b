"""Checkpoint / resume of keys and ciphertext arrays (host side, no GPU)."""

import numpy as np
import torch

from paper_2504_03909_b300 import paillier as P, synth
from paper_2504_03909_b300.state import load_state, save_state


def test_private_key_and_arrays_roundtrip(tmp_path):
    p, q = synth.gen_primes(1024, 1)
    key = P.Key.from_primes(1024, p, q)
    ct = torch.from_numpy(synth.rng_misc(3).integers(-2**31, 2**31 - 1, size=(5, 64), dtype=np.int64)
                          .astype(np.int32))
    bins = torch.from_numpy(synth.gen_bins_uniform(3, 5, 16, 2))
    path = str(tmp_path / "state.npz")
    save_state(path, key, {"ct": ct, "bins": bins})
    key2, arrays = load_state(path)
    assert key2.export() == (p * q, p, q) and key2.is_private
    assert torch.equal(arrays["ct"], ct) and torch.equal(arrays["bins"], bins)


def test_public_key_roundtrip(tmp_path):
    p, q = synth.gen_primes(1024, 1)
    key = P.Key.public(1024, p * q)
    path = str(tmp_path / "pub.npz")
    save_state(path, key)
    key2, arrays = load_state(path)
    assert key2.export() == (p * q, None, None) and not key2.is_private and arrays == {}
