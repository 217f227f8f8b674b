"""Pins for the CPU oracle: checks against facts other than the oracle itself.

* brute force over toy primes (every plaintext, every unit r);
* the encryption map is a bijection Z_n x Z_n^* -> Z_{n^2}^*;
* additive homomorphism (Sec. III.B: ciphertexts are "added" into slots);
* lambda-form decryption == CRT-form decryption (Paillier 1999, Sec. 7);
* the fixed-point encoding against numpy's round-half-even and hand-derived ties;
* the plaintext histogram against np.bincount and a plain loop;
* the encrypted histogram decrypts to the plaintext histogram and is
  invariant under a shuffle of the samples;
* the paper's operation count (Sec. III.C: (M - K) x 2 x J additions);
* Miller-Rabin on known primes / composites; Montgomery REDC definition.
"""

import itertools
import os
import random
from fractions import Fraction
from math import gcd

import numpy as np
import pytest

import oracle
from paper_2504_03909_b300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
TOY_PRIMES = [5, 7, 11, 13, 17, 19, 23]


def _toy_keys():
    for p, q in itertools.combinations(TOY_PRIMES, 2):
        n = p * q
        if gcd(n, (p - 1) * (q - 1)) == 1:
            yield p, q


def test_encode_golden_ties():
    path = os.path.join(HERE, "golden", "encode_halves.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 10
    for k, want in rows:
        v = np.float32(int(k) * 2.0 ** -25)
        assert float(v) == int(k) * 2.0 ** -25  # the fixture value is exact in float32
        assert oracle.encode(v) - oracle.OFFSET == int(want), (k, want)


def test_encode_vs_numpy_rint():
    # every 9973rd float32 bit pattern whose value lies in [-1, 1]
    bits = np.arange(0, 1 << 32, 9973, dtype=np.uint64).astype(np.uint32)
    vals = bits.view(np.float32)
    vals = vals[np.isfinite(vals) & (np.abs(vals) <= 1.0)]
    assert vals.size > 100_000
    sample = vals[:: max(1, vals.size // 20000)]
    ref = np.rint(sample.astype(np.float64) * 2.0 ** 24).astype(np.int64)  # exact product, ties to even
    got = np.array([oracle.encode(v) - oracle.OFFSET for v in sample], dtype=np.int64)
    assert np.array_equal(got, ref)


def test_decode_of_sum():
    rng = synth.rng_misc(7)
    v = rng.standard_normal(500).astype(np.float32) * np.float32(0.4)
    ms = [oracle.encode(x) for x in v]
    exact = sum(Fraction(int(np.rint(np.float64(x) * 2 ** 24)), 2 ** 24) for x in v)
    assert oracle.decode(sum(ms), len(ms)) == exact
    # the decoded sum is within count * 2^-25 of the float sum
    assert abs(float(oracle.decode(sum(ms), len(ms))) - float(np.sum(v.astype(np.float64)))) <= len(v) * 2 ** -25


@pytest.mark.parametrize("p,q", list(_toy_keys()))
def test_bruteforce_toy_key(p, q):
    pub, priv = oracle.keypair(p, q)
    n, n2 = pub.n, pub.n2
    units = [r for r in range(1, n) if gcd(r, n) == 1]
    seen = set()
    for m in range(n):
        for r in units:
            c = oracle.encrypt(pub, m, r)
            assert gcd(c, n) == 1 and 0 < c < n2
            assert oracle.decrypt(priv, c) == m
            assert oracle.decrypt_crt(priv, c) == m
            seen.add(c)
    # bijection Z_n x Z_n^* -> Z_{n^2}^*: n * phi(n) distinct units mod n^2
    phi = (p - 1) * (q - 1)
    assert len(seen) == n * phi == sum(1 for x in range(n2) if gcd(x, n) == 1)


@pytest.mark.parametrize("p,q", [(7, 11), (13, 17), (19, 23)])
def test_toy_homomorphism_all_pairs(p, q):
    pub, priv = oracle.keypair(p, q)
    n = pub.n
    r1, r2 = 2, n - 1
    for m1 in range(n):
        c1 = oracle.encrypt(pub, m1, r1)
        for m2 in range(n):
            c2 = oracle.encrypt(pub, m2, r2)
            assert oracle.decrypt(priv, oracle.add(pub, c1, c2)) == (m1 + m2) % n


def test_generator_binomial_identity():
    # (n + 1)^m = 1 + m n (mod n^2): the closed form a kernel may use for g^m
    for p, q in _toy_keys():
        n = p * q
        for m in range(n):
            assert pow(n + 1, m, n * n) == (1 + m * n) % (n * n)
    p, q = synth.gen_primes(512, 3)
    n = p * q
    for m in (0, 1, 2 ** 25, 2 ** 45 + 12345, n - 1):
        assert pow(n + 1, m, n * n) == (1 + m * n) % (n * n)


@pytest.fixture(scope="module")
def key1024():
    p, q = synth.gen_primes(1024, 1)
    oracle.check_key(p, q, 1024)
    return oracle.keypair(p, q)


def test_large_roundtrip_crt_homomorphism(key1024):
    pub, priv = key1024
    rng = random.Random(5)
    cs, ms = [], []
    for _ in range(6):
        m = rng.randrange(pub.n)
        r = rng.randrange(1, pub.n)
        c = oracle.encrypt(pub, m, r)
        assert oracle.decrypt(priv, c) == m
        assert oracle.decrypt_crt(priv, c) == m
        cs.append(c)
        ms.append(m)
    prod = 1
    for c in cs:
        prod = oracle.add(pub, prod, c)
    assert oracle.decrypt_crt(priv, prod) == sum(ms) % pub.n
    # a tampered exponent (phi in place of lambda, but mu unchanged) breaks decryption
    bad = oracle.L(pow(cs[0], (priv.p - 1) * (priv.q - 1), pub.n2), pub.n) * priv.mu % pub.n
    assert bad != ms[0]


def test_plain_histogram_vs_bincount():
    rng = synth.rng_misc(11)
    M, F, K, nodes = 700, 5, 9, 3
    m = rng.integers(0, 2 ** 25 + 1, size=(2, M))
    bins = rng.integers(0, K, size=(F, M))
    node = rng.integers(-1, nodes, size=M)
    sums, counts = oracle.plain_histogram(m[0], m[1], bins, node, nodes, K)
    for f in range(F):
        sel = node >= 0
        key = node[sel] * K + bins[f][sel]
        for k in range(2):
            ref = np.bincount(key, weights=m[k][sel].astype(np.float64), minlength=nodes * K)
            got = np.array([sums[v][f][b][k] for v in range(nodes) for b in range(K)], dtype=np.float64)
            assert np.array_equal(got, ref)
        cref = np.bincount(key, minlength=nodes * K)
        assert [counts[v][f][b] for v in range(nodes) for b in range(K)] == cref.tolist()


def test_plain_histogram_np_equals_loop_definition():
    rng = synth.rng_misc(14)
    M, F, K, nodes = 2000, 4, 13, 5
    m = rng.integers(0, 2 ** 25 + 1, size=(2, M))
    bins = rng.integers(0, K, size=(F, M))
    node = rng.integers(-1, nodes, size=M)
    sums, counts = oracle.plain_histogram(m[0], m[1], bins, node, nodes, K)
    s2, c2 = oracle.plain_histogram_np(m[0], m[1], bins, node, nodes, K)
    assert s2.tolist() == sums and c2.tolist() == counts


def test_paper_operation_count():
    # Sec. III.C: one node, every bin non-empty -> (M - K) x 2 x J modular products
    rng = synth.rng_misc(12)
    M, J, K = 3000, 4, 16
    bins = np.stack([rng.permutation(np.arange(M) % K) for _ in range(J)])
    node = np.zeros(M, dtype=np.int64)
    _, counts = oracle.plain_histogram(np.zeros(M, int), np.zeros(M, int), bins, node, 1, K)
    ops = 2 * sum(max(c - 1, 0) for row in counts[0] for c in row)
    assert ops == (M - K) * 2 * J
    assert (200_000 - 256) * 2 * 30 == 11_984_640  # the paper's "approx 12m"


def test_encrypted_histogram_decrypts_to_plain():
    p, q = synth.gen_primes(256, 9)
    pub, priv = oracle.keypair(p, q)
    rng = synth.rng_misc(13)
    M, F, K, nodes = 120, 3, 5, 2
    m = rng.integers(0, 2 ** 25 + 1, size=(2, M))
    bins = rng.integers(0, K, size=(F, M))
    node = rng.integers(-1, nodes, size=M)
    rr = random.Random(3)
    c = [[oracle.encrypt(pub, int(m[k][i]), rr.randrange(1, pub.n)) for i in range(M)] for k in range(2)]
    H = oracle.encrypted_histogram(pub, c[0], c[1], bins, node, nodes, K)
    sums, counts = oracle.plain_histogram(m[0], m[1], bins, node, nodes, K)
    for v in range(nodes):
        for f in range(F):
            for b in range(K):
                for k in range(2):
                    assert oracle.decrypt(priv, H[v][f][b][k]) == sums[v][f][b][k] % pub.n
                    if counts[v][f][b] == 0:
                        assert H[v][f][b][k] == 1
                assert oracle.encrypted_histogram_cell(pub, c[0], bins, node, v, f, b) == H[v][f][b][0]
    # shuffling the samples leaves every cell unchanged (the product commutes)
    perm = np.array(rng.permutation(M))
    H2 = oracle.encrypted_histogram(pub, [c[0][i] for i in perm], [c[1][i] for i in perm],
                                    bins[:, perm], node[perm], nodes, K)
    assert H2 == H


def test_gh_packing_decrypts_to_both_plain_histograms():
    """One plaintext per sample, encode(g) + 2^B encode(h): the decrypted cell
    splits into the g and h sums of np.bincount (independent of the oracle's
    histogram code), for B just above the sums' width."""
    p, q = synth.gen_primes(256, 10)
    pub, priv = oracle.keypair(p, q)
    rng = synth.rng_misc(14)
    M, F, K = 90, 2, 4
    g = rng.uniform(-1, 1, size=M).astype(np.float32)
    h = rng.uniform(0, 0.25, size=M).astype(np.float32)
    bins = rng.integers(0, K, size=(F, M))
    node = np.zeros(M, dtype=int)
    B = 25 + int(np.ceil(np.log2(M))) + 1
    rr = random.Random(5)
    c = [oracle.encrypt(pub, oracle.encode_gh(g[i], h[i], B), rr.randrange(1, pub.n)) for i in range(M)]
    eg = np.array([oracle.encode(x) for x in g], dtype=np.int64)
    eh = np.array([oracle.encode(x) for x in h], dtype=np.int64)
    for f in range(F):
        want_g = np.bincount(bins[f], weights=eg, minlength=K).astype(np.int64)
        want_h = np.bincount(bins[f], weights=eh, minlength=K).astype(np.int64)
        for b in range(K):
            cell = oracle.encrypted_histogram_cell(pub, c, bins, node, 0, f, b)
            sg, sh = oracle.split_gh(oracle.decrypt(priv, cell), B)
            assert (sg, sh) == (int(want_g[b]), int(want_h[b]))
    with pytest.raises(ValueError):
        oracle.encode_gh(1.0, 0.0, 25)  # encode(1.0) = 2^25 needs 26 bits


def test_miller_rabin_known_values():
    for e in (521, 607, 1279):  # Mersenne primes
        assert oracle.is_probable_prime(2 ** e - 1)
    for x in (561, 1105, 41041, 2047, 3215031751, (2 ** 61 - 1) * (2 ** 89 - 1), 2 ** 512 + 1):
        assert not oracle.is_probable_prime(x)
    assert [x for x in range(60) if oracle.is_probable_prime(x)] == \
        [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59]


def test_check_key_rejects_bad_keys():
    p, q = synth.gen_primes(512, 4)
    oracle.check_key(p, q, 512)
    with pytest.raises(ValueError):
        oracle.check_key(p, p, 512)
    with pytest.raises(ValueError):
        oracle.check_key(p, q + 2 if not oracle.is_probable_prime(q + 2) else q + 4, 512)
    with pytest.raises(ValueError):
        oracle.check_key(p, q, 1024)


def test_mont_product_matches_redc():
    rng = random.Random(17)
    for _ in range(200):
        N = rng.randrange(3, 1 << 96) | 1
        R = 1 << 96
        a, b = rng.randrange(N), rng.randrange(N)
        # Montgomery's REDC, written out
        nprime = (-pow(N, -1, R)) % R
        t = a * b
        u = (t + ((t % R) * nprime % R) * N) // R
        if u >= N:
            u -= N
        assert oracle.mont_product(a, b, N, R) == u
