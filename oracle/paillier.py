"""Plain, slow, obviously-correct CPU oracle for the Paillier hot path.

TEST INFRASTRUCTURE ONLY (see the package docstring): nothing on the product
path imports this module.

What it computes, and where the paper states it:

* Sec. III.B (Secure Vertical): the active party encrypts every sample's
  gradient g and hessian h; each passive party accumulates the ciphertexts
  into the histogram slot (tree node, feature, bin) each sample falls in and
  returns the cumulative encrypted histograms; the active party decrypts them.
* Sec. III.C (HE scheme choice): one encryption per single number, M x 2 per
  boosting round; the encrypted "additions" number about (M - K) x 2 x J; the
  scheme is Paillier (cited, not restated, by the paper).

The Paillier formulas are the textbook scheme (P. Paillier, "Public-key
cryptosystems based on composite degree residuosity classes", EUROCRYPT 1999),
with the generator g = n + 1:

    encrypt(m, r) = g^m * r^n mod n^2 = (1 + m n) r^n mod n^2
    decrypt(c)    = L(c^lambda mod n^2) * mu mod n,  L(x) = (x - 1) / n,
                    lambda = lcm(p - 1, q - 1), mu = L(g^lambda mod n^2)^-1 mod n
    decrypt_crt   = the Chinese-remainder decryption of the same paper (its
                    Sec. 7), used here only as a cross-check of ``decrypt``.

Readings where the paper is silent (the same readings as the GPU path):
  * g = n + 1; the homomorphic "addition" is the product mod n^2;
  * fixed point: m = round_half_even(v * 2^24) + 2^24 (additive offset);
  * an empty histogram cell is the ciphertext 1 (the empty product);
  * samples whose node is -1 are in no histogram.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(brute force over toy primes, invariants, library routines, hand-derived
fixtures); nothing is "parity unpinned".
"""

from fractions import Fraction
from math import gcd

__all__ = [
    "SCALE_BITS", "OFFSET",
    "is_probable_prime", "check_key", "PublicKey", "PrivateKey", "keypair",
    "L", "encode", "decode", "encrypt", "decrypt", "decrypt_crt", "add",
    "plain_histogram", "encrypted_histogram_cell", "encrypted_histogram",
    "mont_product", "plain_histogram_np", "encode_gh", "split_gh",
]

SCALE_BITS = 24
OFFSET = 1 << SCALE_BITS

# Witnesses for the oracle's own primality check: the primes below 200.  The
# library's key generator uses a different (random) witness set, so the two
# checks are independent.
_WITNESSES = [x for x in range(2, 200) if all(x % d for d in range(2, int(x ** 0.5) + 1))]


def is_probable_prime(x: int) -> bool:
    """Miller-Rabin with the fixed witnesses above (error < 4^-46 for composites)."""
    if x < 2:
        return False
    for w in _WITNESSES:
        if x == w:
            return True
        if x % w == 0:
            return False
    d, s = x - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _WITNESSES:
        y = pow(a, d, x)
        if y == 1 or y == x - 1:
            continue
        for _ in range(s - 1):
            y = y * y % x
            if y == x - 1:
                break
        else:
            return False
    return True


def check_key(p: int, q: int, n_bits: int) -> None:
    """Raise ValueError unless (p, q) is a valid key of the reading adopted for
    key generation (the paper is silent): |p| = |q| = n_bits / 2 with the top
    two bits set, p != q, both prime, |n| = n_bits, gcd(n, (p-1)(q-1)) = 1."""
    half = n_bits // 2
    for name, x in (("p", p), ("q", q)):
        if x.bit_length() != half:
            raise ValueError(f"{name} has {x.bit_length()} bits, want {half}")
        if (x >> (half - 2)) != 3:
            raise ValueError(f"{name} does not have its top two bits set")
        if not is_probable_prime(x):
            raise ValueError(f"{name} is not prime")
    if p == q:
        raise ValueError("p == q")
    n = p * q
    if n.bit_length() != n_bits:
        raise ValueError("n has the wrong size")
    if gcd(n, (p - 1) * (q - 1)) != 1:
        raise ValueError("gcd(n, phi(n)) != 1")


def L(x: int, d: int) -> int:
    """Paillier's L function: (x - 1) / d, an exact division for the x it is
    applied to (x = 1 mod d)."""
    assert (x - 1) % d == 0, "L applied to x != 1 mod d"
    return (x - 1) // d


class PublicKey:
    def __init__(self, n: int):
        self.n = n
        self.n2 = n * n
        self.g = n + 1


class PrivateKey(PublicKey):
    def __init__(self, p: int, q: int):
        super().__init__(p * q)
        self.p, self.q = p, q
        self.lam = (p - 1) * (q - 1) // gcd(p - 1, q - 1)
        self.mu = pow(L(pow(self.g, self.lam, self.n2), self.n), -1, self.n)


def keypair(p: int, q: int):
    priv = PrivateKey(p, q)
    return PublicKey(priv.n), priv


def encode(v) -> int:
    """Fixed-point encoding of one g or h value: round_half_even(v * 2^24) + 2^24,
    in exact rational arithmetic (the float is converted exactly)."""
    x = Fraction(float(v)) * OFFSET
    fl = x.numerator // x.denominator
    rem = x - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return fl + OFFSET


def encode_gh(g, h, B: int) -> int:
    """g/h packing (a decrypt-count reduction; the paper encrypts g and h as two
    numbers): one plaintext encode(g) + 2^B encode(h)."""
    eg = encode(g)
    if eg >= 1 << B:
        raise ValueError("encode(g) must be below 2^B")
    return eg + (encode(h) << B)


def split_gh(s: int, B: int):
    """(S_g, S_h) of a decrypted g/h-packed sum S_g + 2^B S_h."""
    return s & ((1 << B) - 1), s >> B


def decode(s: int, count: int) -> Fraction:
    """Inverse of the encoding for a sum of ``count`` encoded values."""
    return Fraction(s - count * OFFSET, OFFSET)


def encrypt(pub: PublicKey, m: int, r: int) -> int:
    """Paillier encryption with g = n + 1 of plaintext m under randomness r."""
    n, n2 = pub.n, pub.n2
    if not 0 <= m < n:
        raise ValueError("plaintext out of range")
    if not (0 < r < n and gcd(r, n) == 1):
        raise ValueError("r must be a unit of Z_n")
    return pow(pub.g, m, n2) * pow(r, n, n2) % n2


def decrypt(priv: PrivateKey, c: int) -> int:
    """Textbook decryption L(c^lambda mod n^2) * mu mod n."""
    if not 0 < c < priv.n2 or gcd(c, priv.n) != 1:
        raise ValueError("ciphertext is not a unit of Z_{n^2}")
    return L(pow(c, priv.lam, priv.n2), priv.n) * priv.mu % priv.n


def decrypt_crt(priv: PrivateKey, c: int) -> int:
    """Chinese-remainder decryption (Paillier 1999, Sec. 7): decrypt mod p and
    mod q with the exponents p - 1 and q - 1, then recombine."""
    p, q = priv.p, priv.q
    p2, q2 = p * p, q * q
    hp = pow(L(pow(priv.g, p - 1, p2), p), -1, p)
    hq = pow(L(pow(priv.g, q - 1, q2), q), -1, q)
    mp = L(pow(c % p2, p - 1, p2), p) * hp % p
    mq = L(pow(c % q2, q - 1, q2), q) * hq % q
    return mq + q * ((mp - mq) * pow(q, -1, p) % p)


def add(pub: PublicKey, c1: int, c2: int) -> int:
    """Homomorphic addition of two plaintexts: the product of the ciphertexts mod n^2."""
    return c1 * c2 % pub.n2


def mont_product(a: int, b: int, N: int, R: int) -> int:
    """Montgomery product a * b * R^-1 mod N (definition, for kernel unit tests)."""
    return a * b * pow(R, -1, N) % N


def plain_histogram(m_g, m_h, bins, node, num_nodes: int, K: int):
    """Plaintext fixed-point histogram: for each (node v, feature f, bin b) the
    sums of m_g and m_h over samples i with node[i] = v and bins[f][i] = b, and
    the count of such samples.  Samples with node -1 are skipped.

    Returns (sums, counts): sums[v][f][b] = [G, H] (Python ints),
    counts[v][f][b] (int).  Plain loops: for small and sampled cases."""
    F = len(bins)
    M = len(node)
    sums = [[[[0, 0] for _ in range(K)] for _ in range(F)] for _ in range(num_nodes)]
    counts = [[[0] * K for _ in range(F)] for _ in range(num_nodes)]
    for i in range(M):
        v = int(node[i])
        if v < 0:
            continue
        for f in range(F):
            b = int(bins[f][i])
            cell = sums[v][f][b]
            cell[0] += int(m_g[i])
            cell[1] += int(m_h[i])
            counts[v][f][b] += 1
    return sums, counts


def plain_histogram_np(m_g, m_h, bins, node, num_nodes: int, K: int):
    """The same plaintext histogram as ``plain_histogram``, for large inputs:
    one np.bincount per feature over the key node * K + bin of the samples with
    node >= 0, in exact int64 arithmetic (sums < 2^63 for M < 2^38 samples of
    at most 2^25).  Returns (sums int64 [num_nodes][F][K][2], counts int64
    [num_nodes][F][K])."""
    import numpy as np
    node = np.asarray(node).astype(np.int64)
    sel = node >= 0
    F = len(bins)
    sums = np.zeros((num_nodes, F, K, 2), dtype=np.int64)
    counts = np.zeros((num_nodes, F, K), dtype=np.int64)
    mg = np.asarray(m_g).astype(np.int64)[sel]
    mh = np.asarray(m_h).astype(np.int64)[sel]
    for f in range(F):
        key = node[sel] * K + np.asarray(bins[f]).astype(np.int64)[sel]
        counts[:, f, :] = np.bincount(key, minlength=num_nodes * K).reshape(num_nodes, K)
        for k, mm in enumerate((mg, mh)):
            # split into 2^20-sized pieces so float64 weights stay exact
            lo = np.bincount(key, weights=(mm & 0xFFFFF).astype(np.float64), minlength=num_nodes * K)
            hi = np.bincount(key, weights=(mm >> 20).astype(np.float64), minlength=num_nodes * K)
            sums[:, f, :, k] = (lo.astype(np.int64) + (hi.astype(np.int64) << 20)).reshape(num_nodes, K)
    return sums, counts


def encrypted_histogram_cell(pub: PublicKey, cts, bins, node, v: int, f: int, b: int) -> int:
    """One cell of the encrypted histogram: the product mod n^2 of the
    ciphertexts of the samples with node v and bin b in feature f (1 if none)."""
    acc = 1
    col = bins[f]
    for i in range(len(node)):
        if int(node[i]) == v and int(col[i]) == b:
            acc = acc * cts[i] % pub.n2
    return acc


def encrypted_histogram(pub: PublicKey, c_g, c_h, bins, node, num_nodes: int, K: int):
    """Full encrypted histogram H[v][f][b] = [prod c_g, prod c_h] mod n^2 over
    the samples of each cell (the ciphertext 1 for an empty cell)."""
    F = len(bins)
    H = [[[[1, 1] for _ in range(K)] for _ in range(F)] for _ in range(num_nodes)]
    n2 = pub.n2
    for i in range(len(node)):
        v = int(node[i])
        if v < 0:
            continue
        for f in range(F):
            cell = H[v][f][int(bins[f][i])]
            cell[0] = cell[0] * c_g[i] % n2
            cell[1] = cell[1] * c_h[i] % n2
    return H
