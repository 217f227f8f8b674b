"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerance is zero everywhere: ciphertexts, plaintexts, histogram cells and
counts must be bit-identical (integer arithmetic; several orders of the
product are equally correct and give the same residue).
"""

import random

import numpy as np
import pytest
import torch

import oracle
from paper_2504_03909_b300 import native, paillier as P, synth

from helpers import oracle_decrypt_many, oracle_encrypt_many

pytestmark = pytest.mark.gpu

LANES = [(32, 2), (32, 4), (64, 2), (64, 4), (64, 8), (96, 4), (96, 8), (128, 4), (128, 8), (192, 8), (192, 16)]


def _dev(a):
    return P.to_limb_tensor(a)


def _mont_gpu(limbs, lanes, N, A, B):
    a = _dev(synth.ints_to_limbs(A, limbs))
    b = _dev(synth.ints_to_limbs(B, limbs))
    out = torch.empty_like(a)
    Nl = synth.int_to_limbs(N, limbs)
    native.call("paillier_test_mont_mul", limbs, lanes, Nl.ctypes.data, a.data_ptr(), b.data_ptr(), len(A),
                out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return synth.limbs_to_ints(P.from_limb_tensor(out))


@pytest.mark.parametrize("limbs,lanes", LANES)
def test_mont_mul_random_and_edges(limbs, lanes):
    rng = random.Random(limbs * 100 + lanes)
    R = 1 << (32 * limbs)
    moduli = [
        rng.randrange(R // 2, R) | 1,                 # top bit set
        R - 1,                                         # all-ones limbs
        rng.randrange(1 << (32 * limbs - 31), 1 << (32 * limbs - 30)) | 1,  # top limb = 1 or 2
    ]
    # a composite modulus p q, to reach products = 0 mod N (pre-reduction value exactly N)
    p = rng.randrange(1 << (16 * limbs - 2), 1 << (16 * limbs - 1)) | 1
    q = rng.randrange(1 << (16 * limbs), 1 << (16 * limbs + 1)) | 1
    moduli.append(p * q)
    for N in moduli:
        A, B = [], []
        edge = [0, 1, 2, N - 1, N - 2, N // 2, (1 << 32) - 1, R // 2 % N, (R - 1) % N, (N - 1) // 3]
        for x in edge:
            for y in edge:
                A.append(x % N)
                B.append(y % N)
        if N == p * q:
            for _ in range(64):
                A.append(p * rng.randrange(1, q))
                B.append(q * rng.randrange(1, p))
        for _ in range(1500):
            A.append(rng.randrange(N))
            B.append(rng.randrange(N))
        # long carry chains: values whose low limbs are all ones
        for s in (1, limbs // 2, limbs - 1):
            A.append(((1 << (32 * s)) - 1) % N)
            B.append(N - 1)
        got = _mont_gpu(limbs, lanes, N, A, B)
        Rinv = pow(R, -1, N)
        want = [a * b * Rinv % N for a, b in zip(A, B)]
        bad = [i for i in range(len(A)) if got[i] != want[i]]
        assert not bad, f"N={N:#x} first bad index {bad[0]}: a={A[bad[0]]:#x} b={B[bad[0]]:#x}"


SOS_LANES = [(32, 2), (32, 4), (64, 4), (64, 8), (96, 4), (96, 8)]


def _sos_gpu(limbs, lanes, N, A, B=None):
    a = _dev(synth.ints_to_limbs(A, limbs))
    b = _dev(synth.ints_to_limbs(B, limbs)) if B is not None else None
    out = torch.empty_like(a)
    Nl = synth.int_to_limbs(N, limbs)
    native.call("paillier_test_mont_sos", limbs, lanes, Nl.ctypes.data, a.data_ptr(),
                b.data_ptr() if b is not None else None, len(A), out.data_ptr(),
                torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return synth.limbs_to_ints(P.from_limb_tensor(out))


@pytest.mark.parametrize("limbs,lanes", SOS_LANES)
def test_mont_sos_products_and_squares(limbs, lanes):
    """The separated-form Montgomery body of the exponentiations (chunk-pair
    rounds over the lanes, products and squares in one routine) equals
    a b R^-1 mod N and a^2 R^-1 mod N on the moduli and edge inputs of the
    product test: all-ones limbs (N = R - 1, so (P + M N) / R reaches its 2N
    bound), top limb 1 or 2, a composite N with results = 0 mod N, long carry
    chains, and values with one lane's chunk all ones or zero (every lane's
    share of the chunk products at its extremes)."""
    rng = random.Random(limbs * 1000 + lanes)
    R = 1 << (32 * limbs)
    S = limbs // lanes
    p = rng.randrange(1 << (16 * limbs - 2), 1 << (16 * limbs - 1)) | 1
    q = rng.randrange(1 << (16 * limbs), 1 << (16 * limbs + 1)) | 1
    moduli = [rng.randrange(R // 2, R) | 1, R - 1, rng.randrange(1 << (32 * limbs - 31), 1 << (32 * limbs - 30)) | 1,
              p * q]
    for N in moduli:
        A = [0, 1, 2, N - 1, N - 2, N // 2, (1 << 32) - 1, R // 2 % N, (R - 1) % N, (N - 1) // 3]
        if N == p * q:
            # multiples of q and of p: results sharing a factor with N (0 mod N for the products p x q)
            A += [q * rng.randrange(1, p) for _ in range(32)]
            A += [N - p * rng.randrange(1, q) for _ in range(32)]
        # one lane's chunk all ones, the others zero (and the complement)
        for k in range(lanes):
            chunk = ((1 << (32 * S)) - 1) << (32 * S * k)
            A += [chunk % N, (R - 1 - chunk) % N]
        for s in (1, limbs // 2, limbs - 1):
            A.append(((1 << (32 * s)) - 1) % N)
        A += [rng.randrange(N) for _ in range(1500)]
        B = [A[(i * 7 + 3) % len(A)] for i in range(len(A))]  # every edge against many partners
        if N == p * q:
            B[10:42] = [p * rng.randrange(1, q) for _ in range(32)]  # q-multiples x p-multiples = 0 mod N
        Rinv = pow(R, -1, N)
        got = _sos_gpu(limbs, lanes, N, A, B)
        want = [a * b * Rinv % N for a, b in zip(A, B)]
        bad = [i for i in range(len(A)) if got[i] != want[i]]
        assert not bad, f"product N={N:#x} first bad index {bad[0]}: a={A[bad[0]]:#x} b={B[bad[0]]:#x}"
        got = _sos_gpu(limbs, lanes, N, A)
        want = [a * a * Rinv % N for a in A]
        bad = [i for i in range(len(A)) if got[i] != want[i]]
        assert not bad, f"square N={N:#x} first bad index {bad[0]}: a={A[bad[0]]:#x}"


# ---------------------------------------------------------------------------
# toy workload (1,000 samples, 8 features x 16 bins, 1024-bit n): full parity

@pytest.fixture(scope="module")
def toy():
    cfg = synth.CONFIGS["toy"]
    p, q = synth.gen_primes(cfg["n_bits"], cfg["seed"])
    oracle.check_key(p, q, cfg["n_bits"])
    n = p * q
    key = P.Key.from_primes(cfg["n_bits"], p, q)
    gh = synth.gen_gh(cfg["M"], cfg["seed"])
    r = synth.gen_r(n, cfg["n_bits"], 2 * cfg["M"], cfg["seed"], p, q)
    bins = synth.make_bins(cfg)
    return dict(cfg=cfg, p=p, q=q, n=n, key=key, gh=gh, r=r, bins=bins)


def test_toy_encode(toy):
    v = torch.from_numpy(toy["gh"].reshape(-1)).cuda()
    m = P.encode(v)
    P.sync()
    got = m.cpu().numpy().view(np.uint64)
    want = np.array([oracle.encode(x) for x in toy["gh"].reshape(-1)], dtype=np.uint64)
    assert np.array_equal(got, want)


@pytest.fixture(scope="module")
def toy_ct(toy):
    M = toy["cfg"]["M"]
    v = torch.from_numpy(toy["gh"].reshape(-1)).cuda()
    m = P.encode(v)
    r = _dev(toy["r"])
    ct = P.encrypt(toy["key"], m, r)
    P.sync()
    ms = [oracle.encode(x) for x in toy["gh"].reshape(-1)]
    return dict(m=ms, ct=ct, ct_int=synth.limbs_to_ints(P.from_limb_tensor(ct)))


def test_toy_encrypt_bit_exact(toy, toy_ct):
    rs = synth.limbs_to_ints(toy["r"])
    want = oracle_encrypt_many(toy["n"], toy_ct["m"], rs)
    got = toy_ct["ct_int"]
    bad = [i for i in range(len(want)) if got[i] != want[i]]
    assert not bad, f"{len(bad)} ciphertexts differ, first at {bad[0]}"


def test_toy_decrypt_bit_exact(toy, toy_ct):
    key = toy["key"]
    pt = P.decrypt(key, toy_ct["ct"])
    u64 = P.decrypt_u64(key, toy_ct["ct"])
    P.sync()
    got = synth.limbs_to_ints(P.from_limb_tensor(pt))
    assert got == toy_ct["m"]
    assert u64.cpu().numpy().view(np.uint64).tolist() == toy_ct["m"]
    # random units mod n^2 (not produced by encrypt): against the lambda-form oracle
    rng = random.Random(4)
    n, n2 = toy["n"], toy["n"] ** 2
    cs = []
    while len(cs) < 96:
        c = rng.randrange(1, n2)
        if c % toy["p"] and c % toy["q"]:
            cs.append(c)
    ct = _dev(synth.ints_to_limbs(cs, 2 * key.L))
    pt = P.decrypt(key, ct)
    P.sync()
    assert synth.limbs_to_ints(P.from_limb_tensor(pt)) == oracle_decrypt_many(toy["p"], toy["q"], cs)


def _toy_hist_inputs(toy, toy_ct):
    M = toy["cfg"]["M"]
    ct = toy_ct["ct"].view(2, M, -1)
    key = toy["key"]
    ctm = P.ct_prepare(key, ct)
    bins = torch.from_numpy(toy["bins"]).cuda()
    return key, ct, ctm, bins


def test_toy_ct_prepare(toy, toy_ct):
    key, ct, ctm, _ = _toy_hist_inputs(toy, toy_ct)
    P.sync()
    n2 = toy["n"] ** 2
    R = 1 << (64 * key.L)
    got = synth.limbs_to_ints(P.from_limb_tensor(ctm.reshape(-1, 2 * key.L)))
    want = [c * R % n2 for c in toy_ct["ct_int"]]
    assert got == want


def test_toy_root_histogram_bit_exact(toy, toy_ct):
    key, ct, ctm, bins = _toy_hist_inputs(toy, toy_ct)
    cfg = toy["cfg"]
    M, F, K = cfg["M"], cfg["F"], cfg["K"]
    node = torch.zeros(M, dtype=torch.int32, device="cuda")
    hist, cnt = P.hist_aggregate(key, ctm, bins, node, 1, K)
    P.sync()
    pub = oracle.PublicKey(toy["n"])
    cg, chh = toy_ct["ct_int"][:M], toy_ct["ct_int"][M:]
    H = oracle.encrypted_histogram(pub, cg, chh, toy["bins"], np.zeros(M, dtype=np.int64), 1, K)
    got = synth.limbs_to_ints(P.from_limb_tensor(hist.reshape(-1, 2 * key.L)))
    want = [H[0][f][b][k] for f in range(F) for b in range(K) for k in range(2)]
    assert got == want
    sums, counts = oracle.plain_histogram(toy_ct["m"][:M], toy_ct["m"][M:], toy["bins"], np.zeros(M, int), 1, K)
    assert cnt.cpu().numpy().reshape(-1).tolist() == [counts[0][f][b] for f in range(F) for b in range(K)]
    # decrypted cells equal the plaintext fixed-point sums (Sec. IV: same trees as without encryption)
    dec = P.decrypt_u64(key, hist.reshape(-1, 2 * key.L))
    P.sync()
    assert dec.cpu().numpy().view(np.uint64).tolist() == [sums[0][f][b][k] for f in range(F) for b in range(K)
                                                          for k in range(2)]


@pytest.mark.parametrize("num_nodes,tile_note", [(3, "ragged"), (7, "sparse")])
def test_toy_multi_node_batched_equals_per_node_and_oracle(toy, toy_ct, num_nodes, tile_note):
    key, ct, ctm, bins = _toy_hist_inputs(toy, toy_ct)
    cfg = toy["cfg"]
    M, F, K = cfg["M"], cfg["F"], cfg["K"]
    rng = synth.rng_misc(num_nodes)
    node_np = rng.integers(-1, num_nodes, size=M).astype(np.int32)
    if num_nodes == 7:
        node_np[node_np == 3] = -1  # an empty node
    node = torch.from_numpy(node_np).cuda()
    h1, c1 = P.hist_aggregate(key, ctm, bins, node, num_nodes, K)
    h2, c2 = P.hist_aggregate(key, ctm, bins, node, num_nodes, K, per_node=True)
    P.sync()
    assert torch.equal(h1, h2) and torch.equal(c1, c2)
    pub = oracle.PublicKey(toy["n"])
    H = oracle.encrypted_histogram(pub, toy_ct["ct_int"][:M], toy_ct["ct_int"][M:], toy["bins"], node_np,
                                   num_nodes, K)
    got = synth.limbs_to_ints(P.from_limb_tensor(h1.reshape(-1, 2 * key.L)))
    want = [H[v][f][b][k] for v in range(num_nodes) for f in range(F) for b in range(K) for k in range(2)]
    assert got == want


def test_empty_and_degenerate_histograms(toy, toy_ct):
    key, ct, ctm, bins = _toy_hist_inputs(toy, toy_ct)
    K = toy["cfg"]["K"]
    M = toy["cfg"]["M"]
    # every sample excluded: all cells are the ciphertext 1, counts 0
    node = torch.full((M,), -1, dtype=torch.int32, device="cuda")
    h, c = P.hist_aggregate(key, ctm, bins, node, 2, K)
    P.sync()
    hv = P.from_limb_tensor(h.reshape(-1, 2 * key.L))
    assert (hv[:, 0] == 1).all() and (hv[:, 1:] == 0).all() and int(c.sum()) == 0
    # one sample, K = 1
    one = ctm[:, :1].contiguous()
    b1 = torch.zeros((3, 1), dtype=torch.uint8, device="cuda")
    n1 = torch.zeros(1, dtype=torch.int32, device="cuda")
    h, c = P.hist_aggregate(key, one, b1, n1, 1, 1)
    P.sync()
    got = synth.limbs_to_ints(P.from_limb_tensor(h.reshape(-1, 2 * key.L)))
    assert got == [toy_ct["ct_int"][0], toy_ct["ct_int"][M]] * 3
    assert c.cpu().numpy().reshape(-1).tolist() == [1, 1, 1]


def test_bad_bin_reports_device_error(toy, toy_ct):
    key, ct, ctm, bins = _toy_hist_inputs(toy, toy_ct)
    M = toy["cfg"]["M"]
    node = torch.zeros(M, dtype=torch.int32, device="cuda")
    bad = bins.clone()
    bad[0, 5] = 200  # >= K
    P.hist_aggregate(key, ctm, bad, node, 1, toy["cfg"]["K"])
    with pytest.raises(native.PaillierError) as e:
        P.sync()
    assert e.value.code == native.PL_EDEVICE
    P.sync()  # the word was cleared
