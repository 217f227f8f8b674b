"""Packing of histogram cells (fewer decryptions): pack + one decryption per
packed ciphertext returns exactly the per-cell plaintexts, for several slot
widths, ragged last groups and every key size; an overflowing slot is reported."""

import numpy as np
import pytest
import torch

import oracle
from paper_2504_03909_b300 import native, paillier as P, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[1024, 2048, 3072])
def cells(request):
    n_bits = request.param
    p, q = synth.gen_primes(n_bits, 6)
    key = P.Key.from_primes(n_bits, p, q)
    count = 700 if n_bits < 3072 else 200
    rng = synth.rng_misc(n_bits)
    m = rng.integers(0, 1 << 45, size=count, dtype=np.int64)
    m[:5] = [0, 1, (1 << 45) - 1, 7, 0]
    r = synth.gen_r(p * q, n_bits, count, 6, p, q)
    ct = P.encrypt(key, torch.from_numpy(m).cuda(), P.to_limb_tensor(r))
    P.sync()
    return dict(key=key, m=m, ct=ct, p=p, q=q, count=count)


@pytest.mark.parametrize("B", [45, 48, 64])
def test_packed_decrypt_equals_per_cell(cells, B):
    key, count = cells["key"], cells["count"]
    slots = P.pack_slots(key, B)
    assert slots == (key.n_bits - 2) // B
    for c in (count, count - 1, slots + 1, 1):   # ragged last groups
        packed = P.pack(key, cells["ct"][:c], B)
        got = P.decrypt_packed_u64(key, packed, c, B)
        P.sync()
        assert packed.shape[0] == (c + slots - 1) // slots
        assert got.cpu().numpy().tolist() == cells["m"][:c].tolist()


@pytest.mark.parametrize("slots", [1, 2, 7])
def test_fewer_slots_give_the_same_plaintexts(cells, slots):
    """pack_n / decrypt_packed_u64_n with fewer cells per packed ciphertext
    (shorter Horner chains): the same per-cell plaintexts, and a packed
    ciphertext that decrypts to the Horner sum of its `slots` cells."""
    key, B, count = cells["key"], 46, cells["count"]
    for c in (count, slots + 1, 1):
        packed = P.pack(key, cells["ct"][:c], B, slots=slots)
        got = P.decrypt_packed_u64(key, packed, c, B, slots=slots)
        P.sync()
        assert packed.shape[0] == -(-c // slots)
        assert got.cpu().numpy().tolist() == cells["m"][:c].tolist()
    pt = P.decrypt(key, P.pack(key, cells["ct"][:slots], B, slots=slots))
    P.sync()
    assert synth.limbs_to_ints(P.from_limb_tensor(pt))[0] == sum(int(cells["m"][j]) << (B * j) for j in range(slots))


def test_slots_out_of_range_are_refused(cells):
    key, B = cells["key"], 46
    most = P.pack_slots(key, B)
    for bad in (-1, most + 1):
        with pytest.raises(ValueError):
            P.pack(key, cells["ct"][:4], B, slots=bad)
        # and by the library itself, before any launch
        with pytest.raises(native.PaillierError):
            native.call("paillier_pack_n", key.handle, cells["ct"].data_ptr(), 4, B, bad,
                        cells["ct"].data_ptr(), None)
    assert P.pack(key, cells["ct"][:4], B, slots=most).shape[0] == 1


def test_packed_plaintext_is_the_horner_sum(cells):
    # the packed ciphertext decrypts (full width) to sum_j m_j 2^(B j)
    key, B = cells["key"], 48
    slots = P.pack_slots(key, B)
    packed = P.pack(key, cells["ct"][:slots], B)
    pt = P.decrypt(key, packed)
    P.sync()
    want = sum(int(cells["m"][j]) << (B * j) for j in range(slots))
    assert synth.limbs_to_ints(P.from_limb_tensor(pt))[0] == want
    # and the oracle agrees on the packed ciphertext itself
    priv = oracle.PrivateKey(cells["p"], cells["q"])
    assert oracle.decrypt_crt(priv, synth.limbs_to_ints(P.from_limb_tensor(packed))[0]) == want


def test_overflowing_slot_is_reported(cells):
    key, B = cells["key"], 30
    slots = P.pack_slots(key, B)
    packed = P.pack(key, cells["ct"][5:5 + slots], B)   # values up to 2^45 do not fit 30 bits
    P.decrypt_packed_u64(key, packed, slots, B)
    with pytest.raises(native.PaillierError) as e:
        P.sync()
    assert e.value.code == native.PL_ERANGE


# ---- g/h packing: one plaintext per sample -----------------------------------

@pytest.fixture(scope="module", params=[1024, 2048, 3072])
def gh_case(request):
    n_bits = request.param
    p, q = synth.gen_primes(n_bits, 7)
    key = P.Key.from_primes(n_bits, p, q)
    M, F, K, nodes = (3000 if n_bits < 3072 else 800), 5, 16, 3
    gh = synth.gen_gh(M, 7)
    bins = synth.gen_bins_uniform(F, M, K, 7)
    node = synth.rng_misc(70).integers(-1, nodes, size=M).astype(np.int32)
    r = synth.gen_r(p * q, n_bits, M, 7, p, q)
    B = 25 + int(np.ceil(np.log2(M))) + 1
    g_d, h_d = torch.from_numpy(gh[0].copy()).cuda(), torch.from_numpy(gh[1].copy()).cuda()
    m2 = P.encode_gh(g_d, h_d, B)
    ct = P.encrypt_gh(key, m2, P.to_limb_tensor(r))
    ctm = P.ct_prepare(key, ct)
    hist, cnt = P.hist_aggregate_gh(key, ctm, torch.from_numpy(bins).cuda(), torch.from_numpy(node).cuda(), nodes, K)
    P.sync()
    return dict(key=key, p=p, q=q, M=M, F=F, K=K, nodes=nodes, gh=gh, bins=bins, node=node, r=r, B=B, m2=m2,
                ct=ct, hist=hist, cnt=cnt)


def test_gh_encode_and_encrypt_bit_exact(gh_case):
    c = gh_case
    g, h, B = c["gh"][0], c["gh"][1], c["B"]
    words = c["m2"].cpu().numpy().view(np.uint64)
    got = [int(lo) + (int(hi) << 64) for lo, hi in words]
    want = [oracle.encode_gh(g[i], h[i], B) for i in range(c["M"])]
    assert got == want
    pub = oracle.PublicKey(c["p"] * c["q"])
    cts = synth.limbs_to_ints(P.from_limb_tensor(c["ct"]))
    rs = synth.limbs_to_ints(c["r"])
    for i in [0, 1, c["M"] - 1] + list(synth.rng_misc(71).integers(0, c["M"], size=20)):
        assert cts[i] == oracle.encrypt(pub, want[i], rs[i]), i


def test_gh_histogram_cells_and_sums(gh_case):
    c = gh_case
    key, B, K, F, nodes = c["key"], c["B"], c["K"], c["F"], c["nodes"]
    pub = oracle.PublicKey(c["p"] * c["q"])
    cts = synth.limbs_to_ints(P.from_limb_tensor(c["ct"]))
    cells = synth.limbs_to_ints(P.from_limb_tensor(c["hist"].reshape(-1, 2 * key.L)))
    for v, f, b in [(0, 0, 0), (nodes - 1, F - 1, K - 1), (1, 2, 7)]:
        assert cells[(v * F + f) * K + b] == oracle.encrypted_histogram_cell(pub, cts, c["bins"], c["node"], v, f, b)
    eg = np.array([oracle.encode(x) for x in c["gh"][0]], dtype=np.int64)
    eh = np.array([oracle.encode(x) for x in c["gh"][1]], dtype=np.int64)
    want, counts = oracle.plain_histogram_np(eg, eh, c["bins"], c["node"], nodes, K)
    assert c["cnt"].cpu().numpy().tolist() == counts.tolist()
    flat = c["hist"].reshape(-1, 2 * key.L)
    sums = P.decrypt_gh(key, flat, B)
    P.sync()
    assert sums.cpu().numpy().reshape(want.shape).tolist() == want.tolist()
    # with ciphertext packing on top: slots of 2B bits, split at B
    for cnum in (flat.shape[0], flat.shape[0] - 5):
        packed = P.pack(key, flat[:cnum], 2 * B)
        s2 = P.decrypt_packed_gh(key, packed, cnum, B)
        P.sync()
        assert packed.shape[0] == -(-cnum // P.pack_slots(key, 2 * B))
        assert s2.cpu().numpy().tolist() == want.reshape(-1, 2)[:cnum].tolist()
        # fewer cells per packed ciphertext
        packed = P.pack(key, flat[:cnum], 2 * B, slots=3)
        s3 = P.decrypt_packed_gh(key, packed, cnum, B, slots=3)
        P.sync()
        assert packed.shape[0] == -(-cnum // 3)
        assert s3.cpu().numpy().tolist() == want.reshape(-1, 2)[:cnum].tolist()


def test_gh_ranges(gh_case):
    key = gh_case["key"]
    g = torch.full((4,), 4.0, dtype=torch.float32, device="cuda")  # enc(4.0) = 5 2^24 needs 27 bits
    h = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(native.PaillierError):
        P.encode_gh(g, h, 25)  # B below 26
    P.encode_gh(g, h, 26)
    with pytest.raises(native.PaillierError) as e:
        P.sync()
    assert e.value.code == native.PL_ERANGE
    # a cell above 2B bits is reported on decryption
    big = P.encrypt(key, torch.tensor([1 << 62], dtype=torch.int64, device="cuda"),
                    P.to_limb_tensor(gh_case["r"][:1]))
    P.decrypt_gh(key, big, 30)
    with pytest.raises(native.PaillierError) as e:
        P.sync()
    assert e.value.code == native.PL_ERANGE
