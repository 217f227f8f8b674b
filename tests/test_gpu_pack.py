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
