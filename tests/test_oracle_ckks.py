"""Pins for the CKKS oracle of the secure horizontal pattern."""

import numpy as np

from oracle import ckks
from paper_2504_03909_b300 import synth


def test_prime_is_ntt_friendly():
    for log_n in (4, 11, 13):
        q = synth.ckks_prime(log_n)
        assert q % (2 << log_n) == 1 and q < 2 ** 60 and q > 2 ** 59
        # a primitive 2N-th root of unity exists: g^((q-1)/2N) has order exactly 2N for some g
        N = 1 << log_n
        for g in range(2, 50):
            psi = pow(g, (q - 1) // (2 * N), q)
            if pow(psi, N, q) == q - 1:
                break
        else:
            raise AssertionError("no primitive 2N-th root")


def test_negacyclic_product_matches_definition_and_x_pow_n():
    q = synth.ckks_prime(5)
    N = 32
    rng = synth.rng_misc(41)
    for _ in range(4):
        a = [int(x) for x in rng.integers(0, q, size=N, dtype=np.uint64)]
        b = [int(x) for x in rng.integers(-3, 4, size=N)]
        assert ckks.poly_mul(a, b, q) == ckks.poly_mul_schoolbook(a, b, q)
    x_last = [0] * (N - 1) + [1]
    x = [0, 1] + [0] * (N - 2)
    assert ckks.poly_mul(x_last, x, q) == [q - 1] + [0] * (N - 1)  # X^(N-1) X = X^N = -1


def test_encoding_is_the_canonical_embedding():
    N, scale = 64, 2.0 ** 30
    rng = synth.rng_misc(42)
    z = rng.normal(size=N // 2) + 1j * rng.normal(size=N // 2)
    m = ckks.encode(z, N, scale)
    # evaluate m at the slot roots by Horner (independent of the encoder's sums)
    for j, r in enumerate(ckks.roots(N)):
        zeta = np.exp(1j * np.pi * r / N)
        val = 0j
        for c in m[::-1]:
            val = val * zeta + int(c)
        assert abs(val / scale - z[j]) < N / scale * 2  # rounding of N coefficients
    assert np.allclose(ckks.decode(m, N, scale), z, atol=N / scale)


def test_encrypt_decrypt_and_addition():
    N, scale, q = 256, 2.0 ** 30, synth.ckks_prime(8)
    s = synth.ckks_secret(N, 1)
    a = synth.ckks_uniform(N, q, 1)
    e = synth.ckks_gaussian(N, 1, 1)
    b = ckks.keygen(s, a, e, q)
    # b + a s = e exactly
    assert ckks.centre([(x + y) % q for x, y in zip(b, ckks.poly_mul(a, s, q))], q) == e.tolist()
    rng = synth.rng_misc(43)
    zs = [rng.normal(size=N // 2) * 100 + 1j * rng.normal(size=N // 2) for _ in range(3)]
    cts = []
    for i, z in enumerate(zs):
        m = ckks.encode(z, N, scale)
        v = synth.ckks_ternary(N, 2, 10 + i)
        e0 = synth.ckks_gaussian(N, 2, 20 + i)
        e1 = synth.ckks_gaussian(N, 2, 30 + i)
        c = ckks.encrypt(b, a, m, v, e0, e1, q)
        d = ckks.centre(ckks.decrypt(c, s, q), q)
        noise = np.array(d) - m
        # decrypt(encrypt(m)) - m = e v + e0 + e1 s: at most N * 19 + 19 + N * 19 in absolute value
        assert np.abs(noise).max() <= 19 * (2 * N + 1)
        cts.append(c)
    tot = cts[0]
    for c in cts[1:]:
        tot = ckks.add(tot, c, q)
    got = ckks.decode(ckks.centre(ckks.decrypt(tot, s, q), q), N, scale)
    assert np.allclose(got, sum(zs), atol=3 * (N * 0.5 + 19 * (2 * N + 1)) * N / scale)


def test_decoding_satisfies_parseval():
    """For a real polynomial m, the slot values are half of the evaluations at
    the primitive 2N-th roots (the other half are their conjugates), and the
    twisted DFT preserves energy: sum_j |m(zeta_j)|^2 = (N / 2) sum_k m_k^2.
    An identity of the mathematics, independent of the decoder's sums."""
    for N in (16, 256):
        rng = synth.rng_misc(44 + N)
        m = rng.integers(-1000, 1000, size=N)
        z = ckks.decode(m, N, 1.0)
        assert len(z) == N // 2
        lhs = float(np.sum(np.abs(z) ** 2))
        rhs = N / 2 * float(np.sum(m.astype(np.float64) ** 2))
        assert abs(lhs - rhs) <= 1e-9 * rhs
        # the slot roots are distinct primitive 2N-th roots, no two conjugate
        r = ckks.roots(N)
        assert len(set(r)) == N // 2 and all(x % 2 == 1 for x in r)
        assert not any((2 * N - x) in set(r) for x in r)
