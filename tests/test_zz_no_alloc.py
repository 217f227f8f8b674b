"""The allocation-free decryption entry point against the regular one.

paillier_decrypt_u64_noalloc serves callers that may not call cudaMalloc (a
process whose device memory belongs to another allocator, a loop that cannot
afford cudaMalloc's device synchronisation, an embedder that forbids
allocation after start-up).  Its scratch is one fixed array inside the
library.  This file is collected last so that a stop-at-first-failure run has
already run every other test; it also passes on its own in a fresh process.
"""

import ctypes as C

import numpy as np
import pytest
import torch

from paper_2504_03909_b300 import native, paillier as P, synth

pytestmark = pytest.mark.gpu


def _ciphertexts(key, n, count, seed, p, q):
    rng = synth.rng_misc(seed)
    m = torch.from_numpy(rng.integers(0, 1 << 45, size=count, dtype=np.int64)).cuda()
    r = P.to_limb_tensor(synth.gen_r(n, key.n_bits, count, seed, p, q))
    return m, P.encrypt(key, m, r)


def _noalloc(key, ct):
    out = torch.empty(ct.shape[0], dtype=torch.int64, device="cuda")
    native.call("paillier_decrypt_u64_noalloc", key.handle, ct.data_ptr(), ct.shape[0], out.data_ptr(),
                torch.cuda.current_stream().cuda_stream)
    return out


@pytest.mark.parametrize("n_bits,seed", [(1024, 1), (2048, 2), (3072, 5)])
def test_noalloc_decrypt_equals_regular_on_two_calls(n_bits, seed):
    p, q = synth.gen_primes(n_bits, seed)
    key = P.Key.from_primes(n_bits, p, q)
    # two calls in a row with different inputs and sizes (one ragged, one at the maximum)
    for count, s in ((3001, 101), (8192, 102)):
        m, ct = _ciphertexts(key, p * q, count, s, p, q)
        got = _noalloc(key, ct)
        want = P.decrypt_u64(key, ct)
        P.sync()
        assert torch.equal(got, want)
        assert torch.equal(got, m)  # and both equal the plaintexts that were encrypted


def test_noalloc_rejects_oversized_call():
    p, q = synth.gen_primes(1024, 1)
    key = P.Key.from_primes(1024, p, q)
    ct = torch.zeros((8193, 2 * key.L), dtype=torch.int32, device="cuda")
    out = torch.empty(8193, dtype=torch.int64, device="cuda")
    rc = native.lib().paillier_decrypt_u64_noalloc(key.handle, ct.data_ptr(), 8193, out.data_ptr(), None)
    assert rc == native.PL_EINVAL and "8192" in native.last_error()
