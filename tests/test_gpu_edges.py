"""Edge cases through the C ABI: a passive party holding only the public key,
empty calls, values outside the encodable range, randomness that is not a unit
of Z_n, plaintexts >= 2^64, graph replays with fewer nodes, the largest bin
count."""

from math import gcd

import numpy as np
import pytest
import torch

import oracle
from paper_2504_03909_b300 import native, paillier as P, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    p, q = synth.gen_primes(1024, 1)
    key = P.Key.from_primes(1024, p, q)
    pub = P.Key.public(1024, p * q)
    M = 600
    gh = synth.gen_gh(M, 3)
    r = synth.gen_r(p * q, 1024, 2 * M, 3, p, q)
    m = P.encode(torch.from_numpy(gh.reshape(-1)).cuda())
    ct = P.encrypt(key, m, P.to_limb_tensor(r))
    P.sync()
    return dict(key=key, pub=pub, p=p, q=q, M=M, ct=ct, m=m)


def test_public_key_party_aggregates_like_the_key_holder(env):
    M, K = env["M"], 256
    bins = torch.from_numpy(synth.gen_bins_uniform(3, M, K, 4)).cuda()
    node = torch.from_numpy(synth.rng_misc(5).integers(-1, 2, size=M).astype(np.int32)).cuda()
    ctm_pub = P.ct_prepare(env["pub"], env["ct"].view(2, M, -1))
    ctm_priv = P.ct_prepare(env["key"], env["ct"].view(2, M, -1))
    h1, c1 = P.hist_aggregate(env["pub"], ctm_pub, bins, node, 2, K)
    h2, c2 = P.hist_aggregate(env["key"], ctm_priv, bins, node, 2, K)
    P.sync()
    assert torch.equal(ctm_pub, ctm_priv) and torch.equal(h1, h2) and torch.equal(c1, c2)
    # a public key cannot decrypt
    with pytest.raises(native.PaillierError):
        P.decrypt(env["pub"], h1.reshape(-1, 2 * env["key"].L))


def test_empty_calls_are_no_ops(env):
    key = env["key"]
    z64 = torch.empty(0, dtype=torch.int64, device="cuda")
    zl = torch.empty((0, key.L), dtype=torch.int32, device="cuda")
    assert P.encrypt(key, z64, zl).shape == (0, 2 * key.L)
    assert P.decrypt(key, torch.empty((0, 2 * key.L), dtype=torch.int32, device="cuda")).shape == (0, key.L)
    assert P.encode(torch.empty(0, dtype=torch.float32, device="cuda")).numel() == 0
    P.sync()


def test_encode_rejects_values_outside_range():
    v = torch.tensor([0.5, -1.0, 32768.0, -1.5, float("nan"), 40000.0], dtype=torch.float32, device="cuda")
    m = P.encode(v)
    with pytest.raises(native.PaillierError) as e:
        P.sync()
    assert e.value.code == native.PL_EDEVICE
    got = m.cpu().numpy().view(np.uint64).tolist()
    assert got[:3] == [oracle.encode(0.5), oracle.encode(-1.0), oracle.encode(32768.0)]
    assert got[3:] == [0, 0, 0]


def test_encrypt_flags_randomness_that_is_not_a_unit(env):
    key, p, q = env["key"], env["p"], env["q"]
    n = p * q
    # r = 0, a multiple of p, a multiple of q; then units, one given as r + n
    rs = [0, p, 3 * q, 5, 5 + n, 7]
    ms = [11, 12, 13, 14, 15, 16]
    assert 5 + n < 1 << 1024
    ct = P.encrypt(key, torch.tensor(ms, dtype=torch.int64, device="cuda"),
                   P.to_limb_tensor(synth.ints_to_limbs(rs, key.L)))
    with pytest.raises(native.PaillierError) as e:
        P.sync()
    assert e.value.code == native.PL_EDEVICE and "factor with n" in str(e.value)
    got = synth.limbs_to_ints(P.from_limb_tensor(ct))
    pub = oracle.PublicKey(n)
    # r^n mod n^2 depends on r mod n only, so r + n encrypts as r
    assert got[3:] == [oracle.encrypt(pub, 14, 5), oracle.encrypt(pub, 15, 5), oracle.encrypt(pub, 16, 7)]
    assert all(gcd(c, n) != 1 for c in got[:3])
    P.sync()  # the word was cleared by the report
    # units only: no report
    P.encrypt(key, torch.tensor(ms[3:], dtype=torch.int64, device="cuda"),
              P.to_limb_tensor(synth.ints_to_limbs(rs[3:], key.L)))
    P.sync()


def test_decrypt_u64_reports_wide_plaintexts(env):
    key, n = env["key"], env["p"] * env["q"]
    rng = synth.rng_misc(9)
    # a random unit mod n^2 decrypts to a full-width plaintext
    c = int(rng.integers(2, 1 << 62)) ** 16 % (n * n)
    ct = P.to_limb_tensor(synth.ints_to_limbs([c], 2 * key.L))
    out = P.decrypt_u64(key, ct)
    with pytest.raises(native.PaillierError) as e:
        P.sync()
    assert e.value.code == native.PL_ERANGE
    assert out.cpu().numpy().view(np.uint64)[0] == np.uint64(2 ** 64 - 1)
    full = P.decrypt(key, ct)
    P.sync()
    assert synth.limbs_to_ints(P.from_limb_tensor(full))[0] == oracle.decrypt_crt(
        oracle.PrivateKey(env["p"], env["q"]), c)


def test_graph_replay_with_fewer_nodes_after_more(env):
    key, M, K = env["key"], env["M"], 16
    ctm = P.ct_prepare(key, env["ct"].view(2, M, -1))
    bins = torch.from_numpy(synth.gen_bins_uniform(2, M, K, 6)).cuda()
    plan = P.LevelPlan(key, M, 2, K, 8)
    node = torch.empty(M, dtype=torch.int32, device="cuda")
    hist = torch.empty((8, 2, K, 2, 2 * key.L), dtype=torch.int32, device="cuda")
    cnt = torch.empty((8, 2, K), dtype=torch.int32, device="cuda")
    for nn in (8, 2, 5, 1):
        node.copy_(torch.from_numpy(synth.rng_misc(nn).integers(-1, nn, size=M).astype(np.int32)))
        plan.run(ctm, bins, node, nn, hist=hist, count=cnt)
        h, c = P.hist_aggregate(key, ctm, bins, node, nn, K)
        P.sync()
        assert torch.equal(hist[:nn], h) and torch.equal(cnt[:nn], c)
    assert plan.stats()["captures"] == 1
