"""Edge cases through the C ABI: a passive party holding only the public key,
empty calls, values outside the encodable range, randomness that is not a unit
of Z_n, plaintexts >= 2^64, graph replays with fewer nodes, the largest bin
count, bad tensor arguments (refused before any launch) and out-of-range ids
in the tree kernels (bounded on the device and reported)."""

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


def test_binding_checks_arguments_before_any_launch(env):
    key, M = env["key"], env["M"]
    m = env["m"][:8]
    r = P.to_limb_tensor(synth.ints_to_limbs([5] * 8, key.L))
    ctm = P.ct_prepare(key, env["ct"].view(2, M, -1))
    bins = torch.from_numpy(synth.gen_bins_uniform(2, M, 16, 8)).cuda()
    node = torch.zeros(M, dtype=torch.int32, device="cuda")
    P.sync()
    bad = [
        lambda: P.encrypt(key, m.to(torch.int32), r),  # dtype
        lambda: P.encrypt(key, m, r[:, :-1]),  # shape
        lambda: P.encrypt(key, m, r.t().contiguous().t()),  # not contiguous
        lambda: P.encrypt(key, m, r, out=torch.empty((7, 2 * key.L), dtype=torch.int32, device="cuda")),  # short out
        lambda: P.decrypt(key, env["ct"][:, :-1].contiguous()),  # row width
        lambda: P.decrypt_u64(key, env["ct"][:4], out=torch.empty(3, dtype=torch.int64, device="cuda")),
        lambda: P.hist_aggregate(key, ctm, bins.to(torch.int32), node, 1, 16),
        lambda: P.hist_aggregate(key, ctm[:, :-1].contiguous(), bins, node, 1, 16),
        lambda: P.hist_aggregate(key, ctm, bins, node, 1, 16,
                                 hist=torch.empty((1, 2, 16, 2, key.L), dtype=torch.int32, device="cuda")),
        lambda: P.decrypt_packed_u64(key, env["ct"][:1], 10_000, 40),  # fewer packed rows than cells need
        lambda: P.split_apply(bins, node, torch.zeros(2, dtype=torch.int32, device="cuda"),
                              torch.zeros(1, dtype=torch.int32, device="cuda")),
    ]
    for i, f in enumerate(bad):
        with pytest.raises(ValueError):
            f()
    assert P.sync() == 0  # nothing reached the device


def test_tree_kernels_bound_device_read_ids():
    M, F, K = 64, 3, 8
    bins = torch.from_numpy(synth.gen_bins_uniform(F, M, K, 7)).cuda()
    b_np = bins.cpu().numpy()
    node = torch.zeros(M, dtype=torch.int32, device="cuda")
    node[5], node[6], node[7] = 2, 1, -1  # two nodes exist: id 2 is out of range; node 1 splits on feature 7 >= F
    bf = torch.tensor([1, 7], dtype=torch.int32, device="cuda")
    bb = torch.tensor([3, 3], dtype=torch.int32, device="cuda")
    nxt = P.split_apply(bins, node, bf, bb)
    with pytest.raises(native.PaillierError) as e:
        P.sync()
    assert e.value.code == native.PL_EDEVICE
    assert "node >= num_nodes" in str(e.value) and "split feature >= F" in str(e.value)
    got = nxt.cpu().tolist()
    assert got[5] == got[6] == got[7] == -1
    assert all(got[i] == (1 if b_np[1, i] > 3 else 0) for i in range(M) if i not in (5, 6, 7))

    # child ids beyond 2 nodes are skipped and reported
    counts = torch.ones((2, F, K), dtype=torch.int32, device="cuda")
    zero2 = torch.zeros(2, dtype=torch.int32, device="cuda")
    ids = torch.tensor([0, 1, 2, 3, 9, -1], dtype=torch.int32, device="cuda")
    sr, sn = P.child_select(ids, counts, zero2, torch.full((2,), 3, dtype=torch.int32, device="cuda"))
    with pytest.raises(native.PaillierError) as e:
        P.sync()
    assert "node >= num_nodes" in str(e.value)
    assert sr.cpu().tolist() == [0, 0] and sn.cpu().tolist() == [0, -1, 1, -1, -1, -1]

    # any non-zero "small is right" flag means right
    rng = synth.rng_misc(12)
    ps = torch.from_numpy(rng.integers(1 << 40, 1 << 41, size=(2, F, K, 2)).astype(np.int64)).cuda()
    pc = torch.from_numpy(rng.integers(100, 200, size=(2, F, K)).astype(np.int32)).cuda()
    ss = torch.from_numpy(rng.integers(0, 1 << 40, size=(2, F, K, 2)).astype(np.int64)).cuda()
    sc = torch.from_numpy(rng.integers(0, 100, size=(2, F, K)).astype(np.int32)).cuda()
    a = P.child_subtract(ps, pc, ss, sc, torch.tensor([1, 0], dtype=torch.int32, device="cuda"))
    b = P.child_subtract(ps, pc, ss, sc, torch.tensor([7, 0], dtype=torch.int32, device="cuda"))
    P.sync()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert torch.equal(a[0][1], ss[0]) and torch.equal(a[0][0], ps[0] - ss[0])

    # any non-zero decision byte means right
    depth = 3
    tf = torch.tensor([0, 1, 2, -1, -1, -1, -1], dtype=torch.int32, device="cuda")
    ones = torch.ones((7, M), dtype=torch.uint8, device="cuda")
    leaf1 = P.tree_route(ones, tf, depth)
    leaf255 = P.tree_route(torch.full((7, M), 255, dtype=torch.uint8, device="cuda"), tf, depth)
    P.sync()
    assert leaf1.cpu().tolist() == leaf255.cpu().tolist() == [6] * M
