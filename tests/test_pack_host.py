"""Argument checks of the packing entry points with a chosen slot count
(include/paillier_pack.h: paillier_pack_n, paillier_decrypt_packed_u64_n,
paillier_decrypt_packed_gh_n), which the library makes before any launch, so
they run without a GPU."""
import pytest

from paper_2504_03909_b300 import native, paillier as P, synth


@pytest.fixture(scope="module")
def key():
    p, q = synth.gen_primes(2048, 41)
    return P.Key.from_primes(2048, p, q)


def test_slot_counts(key):
    assert P.pack_slots(key, 46) == (2048 - 2) // 46 == 44
    assert P.pack_slots(key, 90) == 22
    assert P.pack_slots(key, 129) == 0


@pytest.mark.parametrize("fn, bits", [("paillier_pack_n", 46), ("paillier_decrypt_packed_u64_n", 46),
                                      ("paillier_decrypt_packed_gh_n", 45)])
def test_slots_range(key, fn, bits):
    most = P.pack_slots(key, 2 * bits if fn.endswith("gh_n") else bits)
    for bad in (-1, most + 1, 1 << 30):
        with pytest.raises(native.PaillierError) as e:
            native.call(fn, key.handle, None, 0, bits, bad, None, None)
        assert e.value.code == native.PL_EINVAL
    for ok in (0, 1, most):  # an empty call with a valid count is a no-op
        native.call(fn, key.handle, None, 0, bits, ok, None, None)


def test_widths(key):
    with pytest.raises(native.PaillierError):
        native.call("paillier_decrypt_packed_u64_n", key.handle, None, 0, 65, 0, None, None)
    with pytest.raises(native.PaillierError):
        native.call("paillier_decrypt_packed_gh_n", key.handle, None, 0, 25, 0, None, None)
    with pytest.raises(native.PaillierError):
        native.call("paillier_pack_n", key.handle, None, 0, 129, 0, None, None)


def test_python_wrapper_refuses_before_the_call(key):
    with pytest.raises(ValueError):
        P._slots(key, 46, 45)
    assert P._slots(key, 46, 0) == 44 and P._slots(key, 46, 3) == 3
