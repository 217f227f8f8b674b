"""Seeded synthetic inputs for the Paillier hot path.

This module holds the input recipe shared by the tests, the bench and the
oracle-side checks.  It contains none of the method's arithmetic (no
encryption, no histogram, no modular exponentiation of the scheme): only random
draws, the data shapes of the paper's workloads, and limb packing.

Every stream is ``numpy.random.Generator(PCG64(SeedSequence([seed, tag])))``
with a fixed tag per purpose, so each input can be regenerated on its own.

Workload shapes (Sec. IV.B, Tables I-II; Sec. III.C's worked count M = 200K,
J = 30, K = 256): logistic-loss gradients of a binary label, features binned
to at most 256 bins, two passive parties splitting the features.
"""

from __future__ import annotations

import numpy as np

_TAG_PRIMES = 11
_TAG_GH = 21
_TAG_R = 31
_TAG_BINS = 41
_TAG_TREE = 51
_TAG_MISC = 61


def _rng(seed: int, tag: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(tag)])))


# ----------------------------------------------------------------------------
# limb packing (little-endian uint32 limbs, the library's exchange format)

def ints_to_limbs(values, limbs: int) -> np.ndarray:
    """Pack non-negative Python ints into a uint32 array [len(values)][limbs]."""
    nbytes = 4 * limbs
    buf = b"".join(int(v).to_bytes(nbytes, "little") for v in values)
    return np.frombuffer(buf, dtype="<u4").reshape(len(values), limbs).copy()


def limbs_to_ints(arr) -> list:
    """Unpack a uint32 array [..., limbs] into a flat list of Python ints."""
    a = np.ascontiguousarray(np.asarray(arr, dtype=np.uint32))
    limbs = a.shape[-1]
    flat = a.reshape(-1, limbs)
    raw = flat.astype("<u4").tobytes()
    nb = 4 * limbs
    return [int.from_bytes(raw[i * nb:(i + 1) * nb], "little") for i in range(flat.shape[0])]


def int_to_limbs(value: int, limbs: int) -> np.ndarray:
    return ints_to_limbs([value], limbs)[0]


# ----------------------------------------------------------------------------
# key material (inputs: the paper does not say how keys are made)

def _mr_round(x: int, a: int, d: int, s: int) -> bool:
    y = pow(a, d, x)
    if y == 1 or y == x - 1:
        return True
    for _ in range(s - 1):
        y = y * y % x
        if y == x - 1:
            return True
    return False


def _probable_prime(x: int, rng: np.random.Generator, rounds: int = 40) -> bool:
    for sp in (3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47):
        if x % sp == 0:
            return x == sp
    d, s = x - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for _ in range(rounds):
        a = 2 + int(rng.integers(0, 1 << 62)) % (x - 3)
        if not _mr_round(x, a, d, s):
            return False
    return True


def gen_primes(n_bits: int, seed: int):
    """Two distinct primes of n_bits/2 bits with the top two bits set (so that
    n = p q has exactly n_bits bits) and gcd(n, (p-1)(q-1)) = 1."""
    half = n_bits // 2
    rng = _rng(seed, _TAG_PRIMES)
    words = (half + 63) // 64

    def draw():
        while True:
            raw = rng.bit_generator.random_raw(words)
            x = int.from_bytes(np.asarray(raw, dtype="<u8").tobytes(), "little")
            x &= (1 << half) - 1
            x |= (3 << (half - 2)) | 1
            if _probable_prime(x, rng):
                return x

    from math import gcd
    while True:
        p = draw()
        q = draw()
        n = p * q
        if p != q and n.bit_length() == n_bits and gcd(n, (p - 1) * (q - 1)) == 1:
            return p, q


# ----------------------------------------------------------------------------
# per-sample data of the active party

def gen_gh(M: int, seed: int, pos_rate: float = 0.3):
    """Logistic-loss gradient and hessian in float32: labels y ~ Bernoulli(0.3),
    predictions p ~ U[0, 1) float32, g = p - y, h = p (1 - p).
    Returns a float32 array [2][M] (row 0 = g, row 1 = h)."""
    rng = _rng(seed, _TAG_GH)
    y = (rng.random(M) < pos_rate).astype(np.float32)
    p = rng.random(M, dtype=np.float32)
    g = (p - y).astype(np.float32)
    h = (p * (np.float32(1.0) - p)).astype(np.float32)
    return np.stack([g, h]).astype(np.float32)


def gen_r(n: int, n_bits: int, count: int, seed: int, p: int | None = None, q: int | None = None,
          tag: int = 0) -> np.ndarray:
    """Encryption randomness: ``count`` values uniform in Z_n^*.  Each candidate
    is ceil(n_bits/64) raw PCG64 words taken little-endian and masked to
    n_bits; candidates that are 0, >= n or share a factor with n are rejected
    in draw order.  With the factors p, q given the last test is done as
    p | r or q | r (the same test for r < n, only faster).
    Returns uint32 limbs [count][n_bits/32]."""
    rng = _rng(seed, _TAG_R * 1000 + tag)
    W = (n_bits + 63) // 64
    L = n_bits // 32
    top_mask = np.uint64((1 << (n_bits - 64 * (W - 1))) - 1) if n_bits % 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    n_words = np.frombuffer(n.to_bytes(8 * W, "little"), dtype="<u8")
    out = []
    got = 0
    while got < count:
        batch = max(64, int((count - got) * 1.8) + 16)
        raw = np.asarray(rng.bit_generator.random_raw(batch * W), dtype=np.uint64).reshape(batch, W)
        raw[:, W - 1] &= top_mask
        # lexicographic compare with n from the top word down
        ne = raw != n_words[None, :]
        any_ne = ne.any(axis=1)
        top_idx = W - 1 - np.argmax(ne[:, ::-1], axis=1)
        less = raw[np.arange(batch), top_idx] < n_words[top_idx]
        ok = any_ne & less & raw.any(axis=1)
        for row in np.nonzero(ok)[0]:
            v = int.from_bytes(raw[row].astype("<u8").tobytes(), "little")
            if p is not None and q is not None:
                if v % p == 0 or v % q == 0:
                    continue
            else:
                from math import gcd
                if gcd(v, n) != 1:
                    continue
            out.append(raw[row])
            got += 1
            if got == count:
                break
    words = np.stack(out).astype("<u8") if out else np.zeros((0, W), dtype="<u8")
    return np.frombuffer(words.tobytes(), dtype="<u4").reshape(count, 2 * W)[:, :L].copy()


# ----------------------------------------------------------------------------
# features of a passive party

def gen_bins_uniform(F: int, M: int, K: int, seed: int) -> np.ndarray:
    """Pre-binned features, bin ids uniform integers in [0, K): uint8 [F][M]."""
    rng = _rng(seed, _TAG_BINS)
    return rng.integers(0, K, size=(F, M), dtype=np.uint8 if K <= 256 else np.int32).astype(np.uint8)


def gen_bins_quantile(F: int, M: int, K: int, seed: int, dist: str = "normal") -> np.ndarray:
    """Float32 features (N(0,1) or log-normal(0,1)) quantile-binned to K bins:
    cut points are the empirical quantiles j/K, j = 1..K-1, and a value's bin is
    searchsorted(cuts, x, 'right') clipped to K - 1.  Returns uint8 [F][M]."""
    rng = _rng(seed, _TAG_BINS)
    out = np.empty((F, M), dtype=np.uint8)
    for f in range(F):
        if dist == "normal":
            x = rng.standard_normal(M, dtype=np.float32)
        elif dist == "lognormal":
            x = np.exp(rng.standard_normal(M).astype(np.float32)).astype(np.float32)
        else:
            raise ValueError(dist)
        cuts = np.quantile(x, np.arange(1, K) / K).astype(np.float32)
        out[f] = np.minimum(np.searchsorted(cuts, x, side="right"), K - 1).astype(np.uint8)
    return out


def gen_tree_levels(M: int, depth: int, seed: int):
    """Node membership per level of a full binary tree with skewed splits.

    At each split node the left fraction f ~ Beta(0.5, 0.5); sample i goes left
    iff u_i < f with u_i ~ U(0, 1) drawn fresh per level.  Level l has 2^l
    nodes numbered 0 .. 2^l - 1 (children of node v are 2v and 2v + 1).
    Returns a list of ``depth`` int32 arrays [M] (levels 0 .. depth-1)."""
    rng = _rng(seed, _TAG_TREE)
    node = np.zeros(M, dtype=np.int32)
    levels = [node.copy()]
    for lvl in range(1, depth):
        parents = 1 << (lvl - 1)
        frac = rng.beta(0.5, 0.5, size=parents)
        u = rng.random(M)
        left = u < frac[node]
        node = (2 * node + np.where(left, 0, 1)).astype(np.int32)
        levels.append(node.copy())
    return levels


def feature_split(F: int, parties: int = 2):
    """Contiguous feature ranges of the passive parties (15/15 for F = 30)."""
    per = F // parties
    return [(k * per, F if k == parties - 1 else (k + 1) * per) for k in range(parties)]


def rng_misc(seed: int) -> np.random.Generator:
    """A spare stream for tests that need extra seeded draws."""
    return _rng(seed, _TAG_MISC)


# ----------------------------------------------------------------------------
# the five workloads (Sec. III.C worked sizes; Sec. IV.B tree parameters)

CONFIGS = {
    # plain method, toy: 1,000 samples, 8 uniform pre-binned features x 16 bins, 1024-bit n, root node
    "toy": dict(M=1_000, F=8, K=16, n_bits=1024, seed=1, bins="uniform", depth=1),
    # plain method, one tree level: 250k samples, 30 N(0,1) features quantile-binned to 256, 2048-bit n
    "level": dict(M=250_000, F=30, K=256, n_bits=2048, seed=2, bins="normal", depth=1),
    # a small case of the level workload's kernels (same key size and shapes), for profiling
    "level_small": dict(M=8_192, F=30, K=256, n_bits=2048, seed=2, bins="normal", depth=1),
    # batched: the "level" data, a depth-6 tree with Beta(0.5, 0.5) splits
    "batched": dict(M=250_000, F=30, K=256, n_bits=2048, seed=3, data_seed=2, bins="normal", depth=6),
    # large: 1M samples x 64 log-normal features x 256 bins, 3072-bit n, depth 8
    "large": dict(M=1_000_000, F=64, K=256, n_bits=3072, seed=5, bins="lognormal", depth=8),
    # secure horizontal (CKKS): 5 clients, 200k samples split evenly, 30 features x 256 bins,
    # N = 8192 (4096 complex slots, G real / H imaginary), one 60-bit prime, scale 2^40
    "horizontal": dict(M=200_000, F=30, K=256, clients=5, log_n=13, scale_bits=40, seed=7),
}


def make_bins(cfg: dict) -> np.ndarray:
    seed = cfg.get("data_seed", cfg["seed"])
    if cfg["bins"] == "uniform":
        return gen_bins_uniform(cfg["F"], cfg["M"], cfg["K"], seed)
    return gen_bins_quantile(cfg["F"], cfg["M"], cfg["K"], seed, dist=cfg["bins"])


# ----------------------------------------------------------------------------
# secure horizontal pattern (Sec. III.A, III.C): CKKS inputs

_TAG_CKKS = 71


def ckks_prime(log_n: int, bits: int = 60) -> int:
    """The largest prime q < 2^bits with q = 1 mod 2N (N = 2^log_n): an
    NTT-friendly modulus.  Deterministic (Miller-Rabin with fixed bases that
    decide primality below 3.3e24)."""
    two_n = 1 << (log_n + 1)
    q = ((1 << bits) - 1) // two_n * two_n + 1
    bases = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41)
    while True:
        d, s = q - 1, 0
        while d % 2 == 0:
            d //= 2
            s += 1
        ok = True
        for a in bases:
            x = pow(a, d, q)
            if x in (1, q - 1):
                continue
            for _ in range(s - 1):
                x = x * x % q
                if x == q - 1:
                    break
            else:
                ok = False
                break
        if ok:
            return q
        q -= two_n


def ckks_secret(N: int, seed: int) -> np.ndarray:
    """Ternary secret key: coefficients uniform in {-1, 0, 1} (int8 [N])."""
    return _rng(seed, _TAG_CKKS).integers(-1, 2, size=N, dtype=np.int8)


def ckks_uniform(N: int, q: int, seed: int, tag: int = 0) -> np.ndarray:
    """Uniform polynomial mod q (uint64 [N]), by rejection from 64-bit draws."""
    rng = _rng(seed, _TAG_CKKS * 100 + tag)
    out = np.empty(0, dtype=np.uint64)
    limit = (1 << 64) - ((1 << 64) % q)
    while out.size < N:
        x = np.asarray(rng.bit_generator.random_raw(N), dtype=np.uint64)
        x = x[x < np.uint64(limit)] % np.uint64(q)
        out = np.concatenate([out, x])
    return out[:N]


def ckks_gaussian(shape, seed: int, tag: int, sigma: float = 3.2) -> np.ndarray:
    """Rounded Gaussian errors (int32), sigma 3.2, clipped at 6 sigma."""
    e = np.rint(_rng(seed, _TAG_CKKS * 100 + tag).normal(0.0, sigma, size=shape))
    return np.clip(e, -19, 19).astype(np.int32)


def ckks_ternary(shape, seed: int, tag: int) -> np.ndarray:
    return _rng(seed, _TAG_CKKS * 100 + tag).integers(-1, 2, size=shape, dtype=np.int8)


def horizontal_histograms(M: int, F: int, K: int, clients: int, seed: int):
    """Local G/H histograms of `clients` row partitions of one synthetic data
    set (Table III's even split): float64 [clients][F][K][2]."""
    gh = gen_gh(M, seed).astype(np.float64)
    bins = gen_bins_quantile(F, M, K, seed)
    bounds = np.linspace(0, M, clients + 1).astype(int)
    out = np.zeros((clients, F, K, 2))
    for c in range(clients):
        lo, hi = bounds[c], bounds[c + 1]
        for f in range(F):
            for k in range(2):
                out[c, f, :, k] = np.bincount(bins[f, lo:hi], weights=gh[k, lo:hi], minlength=K)
    return out
