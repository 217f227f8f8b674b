"""The serving loop's packing plan (include/paillier_serve.h, pl_request.pack_slots):
how many cells each packed ciphertext holds, and the modelled work that
classifies a request.  Host logic only (no GPU): the rule is checked on sizes
whose answers are worked out by hand below."""
import math

import pytest

from paper_2504_03909_b300 import native, paillier as P, synth


@pytest.fixture(scope="module")
def keys():
    out = {}
    for n_bits, seed in ((2048, 41), (3072, 42)):
        p, q = synth.gen_primes(n_bits, seed)
        out[n_bits] = P.Key.from_primes(n_bits, p, q)
    return out


def plan(key, M, F, K, **kw):
    return P.Server.request_plan(key, M, F, K, **kw)


def test_no_packing_without_pack_bits(keys):
    assert plan(keys[2048], 5000, 36, 160)[0] == 0


def test_small_requests_keep_at_least_1024_packed_ciphertexts(keys):
    k = keys[2048]
    # 36 x 160 x 2 = 11,520 cells -> ceil(11,520 / 1,024) = 12 cells per packed ciphertext
    assert plan(k, 5000, 36, 160, pack_bits=46)[0] == 12
    # 8 x 64 x 2 = 1,024 cells: one cell each, so no packing at all (cells decrypted directly)
    assert plan(k, 5000, 8, 64, pack_bits=46)[0] == 0
    # 64 x 256 x 2 = 32,768 cells -> 32 (below the 44 that fit at 46 bits)
    assert plan(k, 5000, 64, 256, pack_bits=46)[0] == 32
    # 3072-bit: (3070 // 46) = 66 fit; 11,520 cells -> 12
    assert plan(keys[3072], 5000, 36, 160, pack_bits=46)[0] == 12


def test_large_histogram_work_packs_as_many_as_fit(keys):
    # 2 x 1e6 x 64 products mod n^2 on 128 limbs: 8.4e12 modelled multiply-adds >= 3e12
    assert plan(keys[2048], 1_000_000, 64, 256, pack_bits=46)[0] == (2048 - 2) // 46
    # the threshold: 2 M F (4 * 128^2 + 128) against 3e12 at F = 8
    per = 2 * 8 * (4 * 128 ** 2 + 128)
    m_edge = math.ceil(3e12 / per)
    assert plan(keys[2048], m_edge, 8, 256, pack_bits=46)[0] == 44
    assert plan(keys[2048], m_edge - 1, 8, 256, pack_bits=46)[0] == 4  # 4,096 cells / 1,024


def test_explicit_pack_slots_caps_the_choice(keys):
    k = keys[2048]
    assert plan(k, 5000, 36, 160, pack_bits=46, pack_slots=5)[0] == 5
    assert plan(k, 5000, 36, 160, pack_bits=46, pack_slots=10_000)[0] == 44  # the most that fit
    assert plan(k, 5000, 36, 160, pack_bits=46, pack_slots=1)[0] == 0       # one per ciphertext: none
    with pytest.raises(native.PaillierError):
        plan(k, 5000, 36, 160, pack_bits=46, pack_slots=-1)


def test_gh_requests_pack_in_double_width_slots(keys):
    k = keys[2048]
    # one g/h-packed cell per (feature, bin): 36 x 160 = 5,760 cells -> 6; 2 x 45 = 90-bit slots, 22 fit
    assert plan(k, 5000, 36, 160, gh_bits=45, pack_bits=1)[0] == 6
    assert plan(k, 1_000_000, 64, 256, gh_bits=45, pack_bits=1)[0] == (2048 - 2) // 90


def test_work_model_counts_the_extra_decryptions(keys):
    k = keys[2048]
    L = 64
    mont = lambda nl: 4 * nl * nl + nl                     # CIOS product on nl limbs
    dec = 2 * (2048 / 2) * (7 / 6) * mont(L)               # two CRT halves, 6-bit windows
    hist = 2 * 5000 * 36 * mont(2 * L)
    cells = 2 * 36 * 160
    _, w0 = plan(k, 5000, 36, 160)
    assert w0 == pytest.approx(hist + cells * dec, rel=1e-12)
    s, w = plan(k, 5000, 36, 160, pack_bits=46)
    assert s == 12
    assert w == pytest.approx(hist + math.ceil(cells / s) * (s * 47 * mont(2 * L) + dec), rel=1e-12)
    _, wmax = plan(k, 5000, 36, 160, pack_bits=46, pack_slots=44)
    assert wmax < w < w0
