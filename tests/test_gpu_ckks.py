"""The secure horizontal pattern on the GPU (Sec. III.A, CKKS per Sec. III.C)
against the CKKS oracle.

Integer stages (key generation, encryption, addition, decryption: products in
R_q by the negacyclic NTT) are compared bit for bit with the oracle's exact
products on the same inputs.

Encoding and decoding are float64 on both sides, computed differently: the
oracle sums the terms of the embedding directly, the kernels use a radix-2
FFT of length N/2 over the slot structure.  Each is compared with the exact value through its own error
bound, and the two bounds are added (plus one unit where the result is rounded
to an integer, since the two sides may fall on either side of a rounding
boundary):
  direct sum of n terms   |err| <= gamma_(n+3) * sum |term|
                          (gamma_k = k u / (1 - k u), u = 2^-53; three more
                          roundings for the table's cos/sin and the product)
  radix-2 FFT, length n   ||err||_2 <= ||y||_2 * L eta / (1 - L eta), L = log2 n,
                          eta = mu + gamma_4 (sqrt 2 + mu), mu = 2u the twiddle
                          error (Higham, Accuracy and Stability of Numerical
                          Algorithms, 2nd ed., Thm. 24.2), ||y||_2 = sqrt(n) ||x||_2;
                          the tests take L = log2 N and sqrt(N) (an upper bound);
                          the twist by omega^k and the final scaling add
                          gamma_5 sqrt 2 relative to the same norm."""

import numpy as np
import pytest
import torch

from oracle import ckks as ock
from paper_2504_03909_b300 import ckks as G, synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _gamma(n):
    return (n + 3) * U / (1 - (n + 3) * U)


def _g(k):
    return k * U / (1 - k * U)


def _fft_rel(N):
    """Relative 2-norm error of the kernels' FFT path (see the module text)."""
    L = N.bit_length() - 1
    mu = 2 * U
    eta = mu + _g(4) * (np.sqrt(2) + mu)
    return L * eta / (1 - L * eta) + _g(5) * np.sqrt(2)


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


@pytest.mark.parametrize("log_n,batch", [(4, 3), (10, 3), (11, 2), (12, 2), (13, 2)])
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


@pytest.mark.parametrize("log_n,batch", [(4, 3), (13, 3)])
def test_prepared_keys_bit_exact(log_n, batch):
    """encrypt/decrypt with keys prepared once equal the per-call forms and the oracle."""
    N = 1 << log_n
    q = synth.ckks_prime(log_n)
    ctx = G.Context(log_n, q, 2.0 ** 30)
    s, a, e, v, e0, e1 = _inputs(N, q, batch, 51 + log_n)
    b = ock.keygen(s, a, e, q)
    b_d = _dev(np.array(b, dtype=np.uint64), torch.int64)
    a_d, s_d = _dev(a, torch.int64), _dev(s)
    m = synth.rng_misc(53).integers(-(2 ** 40), 2 ** 40, size=(batch, N), dtype=np.int64)
    args = (_dev(m), _dev(v), _dev(e0), _dev(e1))
    with pytest.raises(Exception):
        ctx.encrypt_prepared(*args)  # nothing prepared yet
    ctx.prepare_public_key(b_d, a_d)
    ctx.prepare_secret_key(s_d)
    c1 = ctx.encrypt_prepared(*args)
    c2 = ctx.encrypt(b_d, a_d, *args)
    assert torch.equal(c1, c2)
    d1 = ctx.decrypt_prepared(c1)
    assert torch.equal(d1, ctx.decrypt(c1, s_d))
    i = batch - 1
    c0o, c1o = ock.encrypt(b, a, m[i], v[i], e0[i], e1[i], q)
    assert _u64(c1[i, 0]) == c0o and _u64(c1[i, 1]) == c1o
    assert _u64(d1[i]) == ock.decrypt((c0o, c1o), s, q)


def test_large_batch_path_bit_exact():
    """A batch above 64 polynomials runs one CTA per polynomial (smaller batches
    spread each polynomial over a cluster of CTAs): both give the oracle's bits."""
    log_n, batch = 10, 66
    N = 1 << log_n
    q = synth.ckks_prime(log_n)
    ctx = G.Context(log_n, q, 2.0 ** 40)
    s, a, e, v, e0, e1 = _inputs(N, q, batch, 61)
    b = ock.keygen(s, a, e, q)
    b_d = _dev(np.array(b, dtype=np.uint64), torch.int64)
    a_d, s_d = _dev(a, torch.int64), _dev(s)
    m = synth.rng_misc(62).integers(-(2 ** 40), 2 ** 40, size=(batch, N), dtype=np.int64)
    args = (_dev(m), _dev(v), _dev(e0), _dev(e1))
    c_all = ctx.encrypt(b_d, a_d, *args)  # one CTA per polynomial
    c_few = ctx.encrypt(b_d, a_d, *(t[:3] for t in args))  # clusters
    assert torch.equal(c_all[:3], c_few)
    d_all = ctx.decrypt(c_all, s_d)
    assert torch.equal(d_all[:3], ctx.decrypt(c_few, s_d))
    ctx.set_cluster_limit(1 << 20)  # the whole batch in clusters
    assert torch.equal(ctx.encrypt(b_d, a_d, *args), c_all)
    assert torch.equal(ctx.decrypt(c_all, s_d), d_all)
    ctx.set_cluster_limit(0)  # small batches without clusters
    assert torch.equal(ctx.encrypt(b_d, a_d, *(t[:3] for t in args)), c_few)
    ctx.set_cluster_limit(64)
    for i in (0, batch - 1):
        c0, c1 = ock.encrypt(b, a, m[i], v[i], e0[i], e1[i], q)
        assert _u64(c_all[i, 0]) == c0 and _u64(c_all[i, 1]) == c1
        assert _u64(d_all[i]) == ock.decrypt((c0, c1), s, q)
    # the embedding: both paths agree to the last bit on the same inputs? (not
    # required: different stage orders) -- each within its bound of the oracle
    rng = synth.rng_misc(63)
    re, im = rng.normal(size=(batch, N // 2)) * 1e3, rng.normal(size=(batch, N // 2)) * 1e3
    m_all = ctx.encode(_dev(re), _dev(im)).cpu().numpy()
    m_few = ctx.encode(_dev(re[:3].copy()), _dev(im[:3].copy())).cpu().numpy()
    f = 2.0 * 2.0 ** 40 / N
    for i in (0, 2, batch - 1):
        want = ock.encode(re[i] + 1j * im[i], N, 2.0 ** 40)
        terms = (np.abs(re[i]) + np.abs(im[i])).sum() * f
        z2 = np.sqrt((re[i] ** 2 + im[i] ** 2).sum())
        tol = 1 + _gamma(N // 2) * terms + f * np.sqrt(N) * z2 * _fft_rel(N) + U * np.abs(want).max()
        assert np.abs(m_all[i] - want).max() <= tol
        if i < 3:
            assert np.abs(m_few[i] - want).max() <= tol
    zr_all, zi_all = ctx.decode(d_all)
    zr_few, zi_few = ctx.decode(d_all[:3].contiguous())
    for i in (0, 2):
        assert np.allclose(zr_all[i].cpu().numpy(), zr_few[i].cpu().numpy(), rtol=0, atol=1e-6)
        assert np.allclose(zi_all[i].cpu().numpy(), zi_few[i].cpu().numpy(), rtol=0, atol=1e-6)


@pytest.mark.parametrize("log_n,batch,mag", [(4, 2, 1.0), (10, 3, 1e4), (12, 1, 1e5), (13, 1, 1e4)])
def test_encode_within_float_bound(log_n, batch, mag):
    N, scale = 1 << log_n, 2.0 ** 40
    ctx = G.Context(log_n, synth.ckks_prime(log_n), scale)
    rng = synth.rng_misc(23 + log_n)
    re = rng.normal(size=(batch, N // 2)) * mag
    im = rng.normal(size=(batch, N // 2)) * mag
    got = ctx.encode(_dev(re), _dev(im)).cpu().numpy()
    for i in range(batch):
        want = ock.encode(re[i] + 1j * im[i], N, scale)
        f = 2.0 * scale / N
        terms = (np.abs(re[i]) + np.abs(im[i])).sum() * f
        z2 = np.sqrt((re[i] ** 2 + im[i] ** 2).sum())
        tol = 1 + _gamma(N // 2) * terms + f * np.sqrt(N) * z2 * _fft_rel(N) + U * np.abs(want).max()
        assert np.abs(got[i] - want).max() <= tol
        # and the encoding decodes back to the slots (the embedding is the right one)
        back = ock.decode(got[i], N, scale)
        assert np.abs(back - (re[i] + 1j * im[i])).max() <= N * (0.5 + tol) / scale + 1e-9 * mag


@pytest.mark.parametrize("log_n,batch", [(4, 2), (10, 2), (12, 1), (13, 1)])
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
        mf = mc[i].astype(np.float64)
        tol = (_gamma(N) * np.abs(mf).sum() + np.sqrt(N) * np.sqrt((mf ** 2).sum()) * _fft_rel(N)) / scale
        tol += U * np.abs(want).max()
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
    with pytest.raises(PaillierError):
        G.Context(14, synth.ckks_prime(14), 2.0 ** 30)  # N = 16384 does not fit one CTA's shared memory
    # zero ciphertext (all-zero randomness and message) decrypts to zero
    z8 = torch.zeros(1, N, dtype=torch.int8, device="cuda")
    z32 = torch.zeros(1, N, dtype=torch.int32, device="cuda")
    zero = torch.zeros(N, dtype=torch.int64, device="cuda")
    c = ctx.encrypt(zero, zero, torch.zeros(1, N, dtype=torch.int64, device="cuda"), z8, z32, z32)
    assert int(c.abs().sum()) == 0
    assert int(ctx.decrypt(c, z8[0]).abs().sum()) == 0
