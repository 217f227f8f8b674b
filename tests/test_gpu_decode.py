"""A9 decode (Sec. III.B: the decrypted G/H sums go on to tree building)
against the oracle's exact rational decode.

paillier_decode maps a decrypted fixed-point sum S of `cnt` encoded values to
(S - cnt 2^24) / 2^24 in float64.  The oracle returns that value as an exact
Fraction; float() rounds it once to nearest, ties to even, which is what the
kernel's single int64 -> float64 conversion does (the scaling by 2^-24 is
exact), so the two must agree bit for bit.  Tolerance: none.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2504_03909_b300 import paillier as P, synth

pytestmark = pytest.mark.gpu

OFF = 1 << 24


def _check(sums, cnts):
    s = torch.tensor(np.array(sums, dtype=np.uint64).view(np.int64), device="cuda")
    c = torch.tensor(np.array(cnts, dtype=np.int32), device="cuda")
    got = P.decode(s, c)
    P.sync()
    want = [float(oracle.decode(int(a), int(b))) for a, b in zip(sums, cnts)]
    g = got.cpu().numpy()
    # compare the float64 bit patterns (so -0.0 / +0.0 and every ulp count)
    assert g.view(np.uint64).tolist() == np.array(want, dtype=np.float64).view(np.uint64).tolist()


def test_decode_hand_built_edges():
    sums, cnts = [], []
    # empty cell: count 0, sum 0 -> 0.0
    sums.append(0); cnts.append(0)
    # negative G: every value below the offset (g = -1 encodes to 0)
    sums.append(0); cnts.append(1000)
    sums.append(3 * OFF - 5); cnts.append(4)
    # exactly the offset per value -> 0
    sums.append(7 * OFF); cnts.append(7)
    # sums near the 2^45 bound of the level workload (250,000 values of at most 2^25)
    sums.append((1 << 45) - 1); cnts.append(250_000)
    sums.append(1 << 45); cnts.append(1_000_000)
    sums.append((1 << 45) + 12345); cnts.append(1)
    # one sample, extreme encodings (v = -1 -> 0, v = 1 -> 2^25)
    sums.append(1 << 25); cnts.append(1)
    sums.append(1); cnts.append(1)
    # differences above 2^53: float64 rounds, ties to even
    for d in ((1 << 54) + 2, (1 << 54) + 6, (1 << 54) + 1, (1 << 60) + (1 << 7), (1 << 62) + 3):
        sums.append(d); cnts.append(0)
    # largest counts the int32 count array can hold, with matching sums
    sums.append((2**31 - 1) * OFF); cnts.append(2**31 - 1)
    sums.append((2**31 - 1) * OFF - 1); cnts.append(2**31 - 1)
    _check(sums, cnts)


def test_decode_random_and_ragged():
    rng = synth.rng_misc(31)
    n = 4096 + 37  # several grid-stride tiles and a ragged tail
    cnts = rng.integers(0, 1 << 20, size=n).astype(np.int64)
    # sums of cnt encoded values lie in [0, cnt 2^25]
    sums = [int(rng.integers(0, int(c) * 2 * OFF + 1)) for c in cnts]
    _check(sums, cnts.tolist())


def test_decode_empty_call():
    out = P.decode(torch.empty(0, dtype=torch.int64, device="cuda"), torch.empty(0, dtype=torch.int32, device="cuda"))
    P.sync()
    assert out.numel() == 0
