"""The secure horizontal pattern on the GPU (Sec. III.A, CKKS per Sec. III.C)
against the CKKS oracle.

Integer stages (key generation, encryption, addition, decryption: products in
R_q by the negacyclic NTT) are compared bit for bit with the oracle's exact
products on the same inputs.  Encoding and decoding are float64 sums of N/2 and
N terms taken in different orders on the two sides; each side's rounding error
is at most gamma_n * sum |term| (gamma_n = n u / (1 - n u), u = 2^-53, plus two
ulps for the table's cos/sin and one for the product), so the two results differ
by at most twice that, plus one unit for a rounding boundary crossed on one side
only (encoding rounds to integers)."""

import numpy as np
import pytest
import torch

from oracle import ckks as ock
from paper_2504_03909_b300 import ckks as G, synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _gamma(n):
    return (n + 3) * U / (1 - (n + 3) * U)


def _inputs(N, q, batch, seed):
    s = synth.ckks_secret(N, seed)
    a = synth.ckks_uniform(N, q, seed)
    e = synth.ckks_gaussian(N, seed, 1)
    v = synth.ckks_ternary((batch, N), seed, 2)
    e0 = synth.ckks_gaussian((batch, N), seed, 3)
    e1 = synth.ckks_gaussian((batch, N), seed, 4)
    return s, a, e, v, e0, e1


def _u64(t: torch.Tensor):
    return [int(x) for x in t.cpu().numpy().view(np.uint64).reshape(-1)]


def _dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.view(dtype)
    return t.cuda()


@pytest.mark.parametrize("log_n", [4, 10, 13])
def test_keygen_bit_exact(log_n):
    N = 1 << log_n
    q = synth.ckks_prime(log_n)
    ctx = G.Context(log_n, q, 2.0 ** 30)
    s, a, e, *_ = _inputs(N, q, 1, 5 + log_n)
    b = ctx.keygen(_dev(s), _dev(a, torch.int64), _dev(e))
    assert _u64(b) == ock.keygen(s, a, e, q)


@pytest.mark.parametrize("log_n,batch", [(4, 3), (10, 3), (13, 2)])
def test_encrypt_sum_decrypt_bit_exact(log_n, batch):
    N = 1 << log_n
    q = synth.ckks_prime(log_n)
    ctx = G.Context(log_n, q, 2.0 ** 30)
    s, a, e, v, e0, e1 = _inputs(N, q, batch, 11 + log_n)
    b = ock.keygen(s, a, e, q)
    rng = synth.rng_misc(17 + log_n)
    m = rng.integers(-(2 ** 45), 2 ** 45, size=(batch, N), dtype=np.int64)
    b_d = _dev(np.array(b, dtype=np.uint64), torch.int64)
    a_d = _dev(a, torch.int64)
    c = ctx.encrypt(b_d, a_d, _dev(m), _dev(v), _dev(e0), _dev(e1))
    want = []
    for i in range(batch):
        c0, c1 = ock.encrypt(b, a, m[i], v[i], e0[i], e1[i], q)
        want.append((c0, c1))
        assert _u64(c[i, 0]) == c0 and _u64(c[i, 1]) == c1, f"ciphertext {i}"
    # the server's sum of three clients' arrays: the same ciphertexts in three orders
    c2 = ctx.encrypt(b_d, a_d, _dev(m[::-1].copy()), _dev(v), _dev(e0), _dev(e1))
    tot = ctx.sum([c, c2, c])
    dec = ctx.decrypt(tot, _dev(s))
    for i in range(batch):
        c0, c1 = ock.encrypt(b, a, m[batch - 1 - i], v[i], e0[i], e1[i], q)
        t = ock.add(ock.add(want[i], (c0, c1), q), want[i], q)
        assert _u64(tot[i, 0]) == t[0] and _u64(tot[i, 1]) == t[1], f"sum {i}"
        assert _u64(dec[i]) == ock.decrypt(t, s, q), f"decrypt {i}"


@pytest.mark.parametrize("log_n,batch,mag", [(4, 2, 1.0), (10, 3, 1e4), (12, 1, 1e5)])
def test_encode_within_float_bound(log_n, batch, mag):
    N, scale = 1 << log_n, 2.0 ** 40
    ctx = G.Context(log_n, synth.ckks_prime(log_n), scale)
    rng = synth.rng_misc(23 + log_n)
    re = rng.normal(size=(batch, N // 2)) * mag
    im = rng.normal(size=(batch, N // 2)) * mag
    got = ctx.encode(_dev(re), _dev(im)).cpu().numpy()
    for i in range(batch):
        want = ock.encode(re[i] + 1j * im[i], N, scale)
        terms = (np.abs(re[i]) + np.abs(im[i])).sum() * (2.0 * scale / N)
        tol = 1 + 2 * _gamma(N // 2) * terms
        assert np.abs(got[i] - want).max() <= tol
        # and the encoding decodes back to the slots (the embedding is the right one)
        back = ock.decode(got[i], N, scale)
        assert np.abs(back - (re[i] + 1j * im[i])).max() <= N * (0.5 + tol) / scale + 1e-9 * mag


@pytest.mark.parametrize("log_n,batch", [(4, 2), (10, 2), (12, 1)])
def test_decode_within_float_bound(log_n, batch):
    N, scale = 1 << log_n, 2.0 ** 40
    q = synth.ckks_prime(log_n)
    ctx = G.Context(log_n, q, scale)
    rng = synth.rng_misc(29 + log_n)
    mc = rng.integers(-(2 ** 50), 2 ** 50, size=(batch, N), dtype=np.int64)
    mq = np.array([[int(x) % q for x in row] for row in mc], dtype=np.uint64)
    re, im = ctx.decode(_dev(mq, torch.int64))
    for i in range(batch):
        want = ock.decode(ock.centre([int(x) for x in mq[i]], q), N, scale)
        tol = 2 * _gamma(N) * np.abs(mc[i]).astype(np.float64).sum() / scale
        assert np.abs(re.cpu().numpy()[i] - want.real).max() <= tol
        assert np.abs(im.cpu().numpy()[i] - want.imag).max() <= tol


def test_horizontal_round_full_size():
    """Five clients, N = 8192 (4096 complex slots), scale 2^40: each client
    encodes its local G (real part) and H (imaginary part) histograms of
    J x K = 30 x 256 = 7680 cells into two plaintexts, encrypts them under the
    shared public key, the server sums, a client decrypts and decodes.  The
    decoded sums equal the plain sums of the local histograms within the CKKS
    error bound: per slot at most ||sum of the clients' encoding rounding and
    noise||_1 / scale = clients * N * (0.5 + 19 (2N + 1)) / scale (plus float64
    error), 0.0116 here."""
    log_n, clients, F, K, M = 13, 5, 30, 256, 200_000
    N, scale = 1 << log_n, 2.0 ** 40
    q = synth.ckks_prime(log_n)
    ctx = G.Context(log_n, q, scale)
    hist = synth.horizontal_histograms(M, F, K, clients, 7)  # [clients][F][K][2]
    slots = N // 2
    cells = F * K
    msgs = -(-cells // slots)
    s, a, e, *_ = _inputs(N, q, 1, 31)
    b = ctx.keygen(_dev(s), _dev(a, torch.int64), _dev(e))
    a_d = _dev(a, torch.int64)
    cts = []
    for c in range(clients):
        flat = np.zeros((msgs, slots, 2))
        flat.reshape(-1, 2)[:cells] = hist[c].reshape(-1, 2)
        m = ctx.encode(_dev(flat[..., 0].copy()), _dev(flat[..., 1].copy()))
        v = synth.ckks_ternary((msgs, N), 40 + c, 2)
        e0 = synth.ckks_gaussian((msgs, N), 40 + c, 3)
        e1 = synth.ckks_gaussian((msgs, N), 40 + c, 4)
        cts.append(ctx.encrypt(b, a_d, m, _dev(v), _dev(e0), _dev(e1)))
    tot = ctx.sum(cts)
    re, im = ctx.decode(ctx.decrypt(tot, _dev(s)))
    got = np.stack([re.cpu().numpy(), im.cpu().numpy()], axis=-1).reshape(-1, 2)[:cells]
    want = hist.sum(axis=0).reshape(-1, 2)
    bound = clients * N * (0.5 + 19 * (2 * N + 1)) / scale + 1e-9 * np.abs(want).max()
    assert np.abs(got - want).max() <= bound
    # integer cross-check at full size: the GPU decryption equals the oracle's
    dec = ctx.decrypt(tot[:1], _dev(s))
    t = (_u64(tot[0, 0]), _u64(tot[0, 1]))
    assert _u64(dec[0]) == ock.decrypt(t, s, q)


def test_edges():
    log_n = 10
    N = 1 << log_n
    q = synth.ckks_prime(log_n)
    ctx = G.Context(log_n, q, 2.0 ** 30)
    assert ctx.slots == N // 2
    # empty batches are no-ops
    empty = torch.empty(0, N // 2, dtype=torch.float64, device="cuda")
    assert ctx.encode(empty, empty).shape == (0, N)
    # a modulus that is not 1 mod 2N, and a composite, are rejected
    from paper_2504_03909_b300.native import PaillierError
    with pytest.raises(PaillierError):
        G.Context(log_n, q + 2, 2.0 ** 30)
    with pytest.raises(PaillierError):
        G.Context(log_n, 12289 * 12289, 2.0 ** 30)  # 12289 = 6 * 2048 + 1 is prime, its square is not
    # zero ciphertext (all-zero randomness and message) decrypts to zero
    z8 = torch.zeros(1, N, dtype=torch.int8, device="cuda")
    z32 = torch.zeros(1, N, dtype=torch.int32, device="cuda")
    zero = torch.zeros(N, dtype=torch.int64, device="cuda")
    c = ctx.encrypt(zero, zero, torch.zeros(1, N, dtype=torch.int64, device="cuda"), z8, z32, z32)
    assert int(c.abs().sum()) == 0
    assert int(ctx.decrypt(c, z8[0]).abs().sum()) == 0
