"""Host-side checks of the C ABI (no GPU): the library loads, exports every
function the headers declare, and its host-only key set-up is right."""

import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2504_03909_b300 import native, paillier as P, synth


def test_library_exports_every_declared_function():
    lib = native.lib()
    names = native.header_functions()
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # every declared function has a ctypes signature (an undeclared one would
    # pass 64-bit pointers as C ints)
    assert set(native.SIGNATURES) == set(names)


def test_checked_library_exports_the_same_functions():
    """The bounds-checked build (build.py --checked) has the same ABI."""
    import os
    path = os.path.join(native.HERE, "libpaillier_b300_checked.so")
    if not os.path.exists(path):
        pytest.skip("checked library not built")
    lib = C.CDLL(path)
    missing = [n for n in native.header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_refuses_host_tensors_before_any_call():
    """The Python layer checks every tensor before its pointer crosses the ABI
    (the kernels trust them): a host tensor never reaches the library."""
    import torch
    from paper_2504_03909_b300 import ckks
    key = P.Key.generate(1024, 3)
    m = torch.zeros(4, dtype=torch.int64)
    r = torch.zeros((4, key.L), dtype=torch.int32)
    with pytest.raises(ValueError, match="CUDA"):
        P.encrypt(key, m, r)
    with pytest.raises(ValueError, match="CUDA"):
        P.decrypt_u64(key, torch.zeros((2, 2 * key.L), dtype=torch.int32))
    with pytest.raises(ValueError, match="CUDA"):
        P.split_find(torch.zeros((1, 2, 4, 2), dtype=torch.int64), torch.zeros((1, 2, 4), dtype=torch.int32))
    with pytest.raises(ValueError):
        P.decrypt(key, torch.zeros((2, 2 * key.L + 1), dtype=torch.int32))
    with pytest.raises(TypeError):
        P._ptr(np.zeros(3), "x")
    with pytest.raises(ValueError, match="CUDA"):
        ckks.Context._poly(type("C", (), {"N": 8})(), torch.zeros(8, dtype=torch.int8), "s", torch.int8)


@pytest.mark.parametrize("n_bits", [1024, 2048])
def test_keygen_is_valid_and_deterministic(n_bits):
    k1 = P.Key.generate(n_bits, 11)
    k2 = P.Key.generate(n_bits, 11)
    n, p, q = k1.export()
    oracle.check_key(p, q, n_bits)
    assert n == p * q and k2.export() == (n, p, q)
    assert P.Key.generate(n_bits, 12).export()[0] != n
    assert k1.is_private and k1.n_bits == n_bits and k1.L == n_bits // 32


def test_import_roundtrip_and_public_key():
    p, q = synth.gen_primes(1024, 1)
    k = P.Key.from_primes(1024, p, q)
    assert k.export() == (p * q, p, q)
    pub = P.Key.public(1024, p * q)
    assert not pub.is_private and pub.export() == (p * q, None, None)


def test_import_rejects_bad_keys():
    p, q = synth.gen_primes(1024, 1)
    with pytest.raises(native.PaillierError) as e:
        P.Key.from_primes(1024, p, p)
    assert e.value.code == native.PL_EINVAL
    with pytest.raises(native.PaillierError):
        P.Key.from_primes(1024, p >> 1, q)  # too short
    arr = np.zeros(48, dtype=np.uint32)
    out = C.c_void_p()
    assert native.lib().paillier_key_import(1000, arr.ctypes.data, arr.ctypes.data, C.byref(out)) == native.PL_EINVAL
    with pytest.raises(native.PaillierError):
        P.Key.public(2048, (p * q) | 1)  # 1024-bit n as a 2048-bit key
    assert "n_bits" in native.last_error() or "n must" in native.last_error()


def test_null_arguments_fail_before_any_launch():
    lib = native.lib()
    out = C.c_void_p()
    assert lib.paillier_keygen(2048, 1, None) == native.PL_EINVAL
    assert lib.paillier_encrypt(None, None, None, 1, None, None) == native.PL_EINVAL
    assert lib.paillier_decrypt(None, None, 1, None, None) == native.PL_EINVAL
    p, q = synth.gen_primes(1024, 1)
    k = P.Key.public(1024, p * q)
    # a public key cannot decrypt or encrypt
    assert lib.paillier_decrypt(k.handle, C.c_void_p(16), 1, C.c_void_p(16), None) == native.PL_EINVAL
    assert lib.paillier_encrypt(k.handle, C.c_void_p(16), C.c_void_p(16), 1, C.c_void_p(16), None) == native.PL_EINVAL
    assert lib.paillier_hist_aggregate(k.handle, None, 0, None, 0, 16, None, 1, C.c_void_p(16), None, None) \
        == native.PL_EINVAL  # F = 0
    assert lib.paillier_key_bits(None) == 0
    del out
