"""CPU oracle for the secure horizontal pattern (test infrastructure only).

Sec. III.A of the paper: each client encrypts its local G/H histograms, the
server adds the ciphertexts, the clients decrypt the global histogram.
Sec. III.C: the scheme is CKKS (cited, not restated).  The formulas are the
textbook CKKS scheme (Cheon, Kim, Kim, Song, ASIACRYPT 2017) restricted to what
this pattern uses -- encoding, public-key encryption, addition, decryption,
decoding -- over R_q = Z_q[X] / (X^N + 1) with one prime q = 1 mod 2N:

    encode(z)     = round(scale * tau^-1(z)), tau(m) = (m(zeta_j))_j,
                    zeta_j = exp(i pi r_j / N), r_j = 5^j mod 2N, j < N/2
    keygen        b = -a s + e            (s ternary, a uniform, e Gaussian)
    encrypt(m)    = (b v + e0 + m, a v + e1)   (v ternary, e0, e1 Gaussian)
    add           component-wise mod q
    decrypt(c)    = c0 + c1 s mod q, centred in (-q/2, q/2]
    decode(m)     = tau(m) / scale

Products in R_q are the negacyclic convolution, computed exactly with
np.convolve on 21-bit pieces (a library primitive) and folded with X^N = -1.
Encoding and decoding are the direct O(N^2) sums in float64.  All randomness
(s, a, e, v, e0, e1) is an input.
"""

import numpy as np


def poly_mul(a, b, q: int):
    """Negacyclic product a b mod (X^N + 1, q) of integer coefficient vectors
    (any integers; the result is in [0, q))."""
    a = [int(x) % q for x in a]
    b = [int(x) % q for x in b]
    N = len(a)
    mask = (1 << 21) - 1
    pa = [np.array([(x >> (21 * u)) & mask for x in a], dtype=np.int64) for u in range(3)]
    pb = [np.array([(x >> (21 * u)) & mask for x in b], dtype=np.int64) for u in range(3)]
    full = [0] * (2 * N - 1)
    for u in range(3):
        for v in range(3):
            c = np.convolve(pa[u], pb[v])  # exact: terms < 2^42, N terms < 2^55
            sh = 21 * (u + v)
            for k in range(2 * N - 1):
                full[k] += int(c[k]) << sh
    return [(full[k] - (full[k + N] if k + N < 2 * N - 1 else 0)) % q for k in range(N)]


def poly_mul_schoolbook(a, b, q: int):
    """The same product by its definition (for small N)."""
    N = len(a)
    out = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                out[k] += int(a[i]) * int(b[j])
            else:
                out[k - N] -= int(a[i]) * int(b[j])
    return [x % q for x in out]


def roots(N: int):
    """r_j = 5^j mod 2N for the N/2 slots."""
    return [pow(5, j, 2 * N) for j in range(N // 2)]


def encode(z, N: int, scale: float):
    """Integer coefficients of round(scale * tau^-1(z)) for z in C^(N/2):
    m_k = (2 scale / N) Re(sum_j z_j exp(-i pi r_j k / N))."""
    z = np.asarray(z, dtype=np.complex128)
    r = np.array(roots(N), dtype=np.int64)
    k = np.arange(N, dtype=np.int64)
    ang = (np.outer(k, r) % (2 * N)) * (np.pi / N)
    s = (np.cos(ang) * z.real[None, :] + np.sin(ang) * z.imag[None, :]).sum(axis=1)
    return np.rint(s * (2.0 * scale / N)).astype(np.int64)


def decode(m_centred, N: int, scale: float):
    """z_j = sum_k m_k exp(i pi r_j k / N) / scale."""
    m = np.asarray(m_centred, dtype=np.float64)
    r = np.array(roots(N), dtype=np.int64)
    k = np.arange(N, dtype=np.int64)
    ang = (np.outer(r, k) % (2 * N)) * (np.pi / N)
    return (np.cos(ang) @ m + 1j * (np.sin(ang) @ m)) / scale


def keygen(s, a, e, q: int):
    """b = -a s + e mod q."""
    As = poly_mul(a, s, q)
    return [(-x + int(ei)) % q for x, ei in zip(As, e)]


def encrypt(b, a, m, v, e0, e1, q: int):
    bv = poly_mul(b, v, q)
    av = poly_mul(a, v, q)
    c0 = [(x + int(y) + int(mm)) % q for x, y, mm in zip(bv, e0, m)]
    c1 = [(x + int(y)) % q for x, y in zip(av, e1)]
    return c0, c1


def add(c, d, q: int):
    return [(x + y) % q for x, y in zip(c[0], d[0])], [(x + y) % q for x, y in zip(c[1], d[1])]


def decrypt(c, s, q: int):
    """c0 + c1 s mod q, in [0, q)."""
    c1s = poly_mul(c[1], s, q)
    return [(x + y) % q for x, y in zip(c[0], c1s)]


def centre(m, q: int):
    return [x - q if x > q // 2 else x for x in m]
