"""GPU tests of the batched level path (graph capture + replay), the
launch configurations and the autotuner.  Results must be bit-identical for
every configuration: tuning changes speed, never bits."""

import os

import numpy as np
import pytest
import torch

import oracle
from paper_2504_03909_b300 import native, paillier as P, synth

from helpers import oracle_encrypt_many

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tree():
    """Toy-scale data (1024-bit key) with a depth-4 skewed tree."""
    n_bits, M, F, K = 1024, 1500, 5, 16
    p, q = synth.gen_primes(n_bits, 1)
    key = P.Key.from_primes(n_bits, p, q)
    gh = synth.gen_gh(M, 7)
    r = synth.gen_r(p * q, n_bits, 2 * M, 7, p, q)
    m = P.encode(torch.from_numpy(gh.reshape(-1)).cuda())
    ct = P.encrypt(key, m, P.to_limb_tensor(r))
    ctm = P.ct_prepare(key, ct.view(2, M, -1))
    bins_np = synth.gen_bins_uniform(F, M, K, 7)
    levels = synth.gen_tree_levels(M, 4, 7)
    P.sync()
    return dict(key=key, p=p, q=q, M=M, F=F, K=K, ct=ct, ctm=ctm, bins_np=bins_np,
                bins=torch.from_numpy(bins_np).cuda(), levels=levels,
                ct_int=synth.limbs_to_ints(P.from_limb_tensor(ct)),
                m=m.cpu().numpy().view(np.uint64).tolist())


def test_level_graph_replay_matches_plain_per_node_and_oracle(tree):
    key, M, F, K = tree["key"], tree["M"], tree["F"], tree["K"]
    plan = P.LevelPlan(key, M, F, K, max_nodes=8)
    node_buf = torch.empty(M, dtype=torch.int32, device="cuda")
    hist_buf = torch.empty((8, F, K, 2, 2 * key.L), dtype=torch.int32, device="cuda")
    cnt_buf = torch.empty((8, F, K), dtype=torch.int32, device="cuda")
    pub = oracle.PublicKey(tree["p"] * tree["q"])
    for lvl, node_np in enumerate(tree["levels"]):
        nn = 1 << lvl
        node_buf.copy_(torch.from_numpy(node_np))
        plan.run(tree["ctm"], tree["bins"], node_buf, nn, hist=hist_buf, count=cnt_buf)
        h_plain, c_plain = P.hist_aggregate(key, tree["ctm"], tree["bins"], node_buf, nn, K)
        h_node, c_node = P.hist_aggregate(key, tree["ctm"], tree["bins"], node_buf, nn, K, per_node=True)
        P.sync()
        hg = hist_buf[:nn].reshape(nn, F, K, 2, -1)
        assert torch.equal(hg, h_plain) and torch.equal(hg, h_node)
        assert torch.equal(cnt_buf[:nn], c_plain) and torch.equal(cnt_buf[:nn], c_node)
        H = oracle.encrypted_histogram(pub, tree["ct_int"][:M], tree["ct_int"][M:], tree["bins_np"], node_np, nn, K)
        got = synth.limbs_to_ints(P.from_limb_tensor(hg.reshape(-1, 2 * key.L)))
        assert got == [H[v][f][b][k] for v in range(nn) for f in range(F) for b in range(K) for k in range(2)]
    st = plan.stats()
    assert st["captures"] == 1 and st["replays"] == len(tree["levels"]) and st["kernels"] >= 6


def test_gh_level_plan_matches_direct_and_oracle(tree):
    """The plan over one g/h-packed array per sample: one capture, every level
    equal to paillier_hist_aggregate_gh and, cell by cell, to the oracle's
    product of the packed ciphertexts."""
    key, M, F, K = tree["key"], tree["M"], tree["F"], tree["K"]
    B = 37
    gh = synth.gen_gh(M, 7)
    r = synth.gen_r(tree["p"] * tree["q"], key.n_bits, M, 8, tree["p"], tree["q"])
    g_d, h_d = torch.from_numpy(gh[0].copy()).cuda(), torch.from_numpy(gh[1].copy()).cuda()
    ct1 = P.encrypt_gh(key, P.encode_gh(g_d, h_d, B), P.to_limb_tensor(r))
    ctm1 = P.ct_prepare(key, ct1)
    plan = P.LevelPlan(key, M, F, K, max_nodes=8, gh=True)
    node_buf = torch.empty(M, dtype=torch.int32, device="cuda")
    hist_buf = torch.empty((8, F, K, 2 * key.L), dtype=torch.int32, device="cuda")
    cnt_buf = torch.empty((8, F, K), dtype=torch.int32, device="cuda")
    pub = oracle.PublicKey(tree["p"] * tree["q"])
    cts = synth.limbs_to_ints(P.from_limb_tensor(ct1))
    for lvl, node_np in enumerate(tree["levels"]):
        nn = 1 << lvl
        node_buf.copy_(torch.from_numpy(node_np))
        plan.run(ctm1, tree["bins"], node_buf, nn, hist=hist_buf, count=cnt_buf)
        h_d, c_d = P.hist_aggregate_gh(key, ctm1, tree["bins"], node_buf, nn, K)
        P.sync()
        assert torch.equal(hist_buf[:nn], h_d) and torch.equal(cnt_buf[:nn], c_d), lvl
        got = synth.limbs_to_ints(P.from_limb_tensor(hist_buf[:nn].reshape(-1, 2 * key.L)))
        for v, f, b in [(0, 0, 0), (nn - 1, F - 1, K - 1), (nn // 2, 2, 5)]:
            want = oracle.encrypted_histogram_cell(pub, cts, tree["bins_np"], node_np, v, f, b)
            assert got[(v * F + f) * K + b] == want, (lvl, v, f, b)
    st = plan.stats()
    assert st["captures"] == 1 and st["replays"] == len(tree["levels"])


def test_level_plan_recaptures_on_new_buffers(tree):
    key, M, F, K = tree["key"], tree["M"], tree["F"], tree["K"]
    plan = P.LevelPlan(key, M, F, K, max_nodes=2)
    node = torch.from_numpy(tree["levels"][1]).cuda()
    h1, c1 = plan.run(tree["ctm"], tree["bins"], node, 2)
    h2, c2 = plan.run(tree["ctm"], tree["bins"], node, 2)  # new output tensors -> new capture
    P.sync()
    assert torch.equal(h1, h2) and torch.equal(c1, c2)
    assert plan.stats()["captures"] == 2
    with pytest.raises(native.PaillierError):
        plan.run(tree["ctm"], tree["bins"], node, 3)  # more nodes than planned


@pytest.mark.parametrize("lanes,tile", [(4, 1), (4, 7), (4, 64), (8, 16), (8, 256), (8, 4096)])
def test_hist_configs_are_bit_identical(tree, lanes, tile):
    key, K = tree["key"], tree["K"]
    node = torch.from_numpy(tree["levels"][2]).cuda()
    ref, cref = P.hist_aggregate(key, tree["ctm"], tree["bins"], node, 4, K)
    old = P.get_config(key, native.OP_HIST)
    try:
        P.set_config(key, native.OP_HIST, lanes, tile)
        h, c = P.hist_aggregate(key, tree["ctm"], tree["bins"], node, 4, K)
        ctm2 = P.ct_prepare(key, tree["ct"])
        P.sync()
    finally:
        P.set_config(key, native.OP_HIST, *old)
    assert torch.equal(h, ref) and torch.equal(c, cref)
    assert torch.equal(ctm2.view(2, tree["M"], -1), tree["ctm"])


@pytest.mark.parametrize("op", [native.OP_ENCRYPT, native.OP_DECRYPT])
@pytest.mark.parametrize("lanes,w", [(2, 2), (2, 4), (4, 3), (4, 6), (4, 7)])
def test_modexp_configs_are_bit_identical(tree, op, lanes, w):
    key = tree["key"]
    sel = slice(0, 64)
    m = torch.from_numpy(np.array(tree["m"][:64], dtype=np.uint64).view(np.int64)).cuda()
    old = P.get_config(key, op)
    try:
        P.set_config(key, op, lanes, w)
        if op == native.OP_ENCRYPT:
            r = synth.gen_r(tree["p"] * tree["q"], 1024, 64, 7, tree["p"], tree["q"])
            ct = P.encrypt(key, m, P.to_limb_tensor(r))
            P.sync()
            assert torch.equal(ct, tree["ct"][sel])
        else:
            pt = P.decrypt_u64(key, tree["ct"][sel])
            P.sync()
            assert pt.cpu().numpy().view(np.uint64).tolist() == tree["m"][:64]
    finally:
        P.set_config(key, op, *old)


def test_2048bit_modexp_configs_bit_exact_vs_oracle():
    p, q = synth.gen_primes(2048, 2)
    n = p * q
    key = P.Key.from_primes(2048, p, q)
    count = 40
    rng = synth.rng_misc(5)
    ms = rng.integers(0, 1 << 40, size=count).astype(np.uint64)
    r = synth.gen_r(n, 2048, count, 5, p, q)
    want = oracle_encrypt_many(n, ms.tolist(), synth.limbs_to_ints(r))
    m = torch.from_numpy(ms.view(np.int64)).cuda()
    for lanes in (2, 4, 8):
        for w in (4, 5, 6):
            P.set_config(key, native.OP_ENCRYPT, lanes, w)
            P.set_config(key, native.OP_DECRYPT, lanes, w)
            ct = P.encrypt(key, m, P.to_limb_tensor(r))
            pt = P.decrypt_u64(key, ct)
            P.sync()
            assert synth.limbs_to_ints(P.from_limb_tensor(ct)) == want, (lanes, w)
            assert pt.cpu().numpy().view(np.uint64).tolist() == ms.tolist(), (lanes, w)


def test_autotune_installs_a_valid_config_and_caches(tree, tmp_path):
    key = tree["key"]
    cache = str(tmp_path / "tune.jsonl")
    for op in (native.OP_ENCRYPT, native.OP_DECRYPT, native.OP_HIST):
        la, pa = P.autotune(key, op, cache)
        assert (la, pa) == P.get_config(key, op)
        assert P.autotune(key, op, cache) == (la, pa)  # served from the cache
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 3 and all('"sms"' in ln for ln in lines)
    # tuned configuration still bit-exact
    node = torch.from_numpy(tree["levels"][1]).cuda()
    h, _ = P.hist_aggregate(key, tree["ctm"], tree["bins"], node, 2, tree["K"])
    pt = P.decrypt_u64(key, tree["ct"][:32])
    P.sync()
    assert pt.cpu().numpy().view(np.uint64).tolist() == tree["m"][:32]
    pub = oracle.PublicKey(tree["p"] * tree["q"])
    M = tree["M"]
    H = oracle.encrypted_histogram(pub, tree["ct_int"][:M], tree["ct_int"][M:], tree["bins_np"], tree["levels"][1],
                                   2, tree["K"])
    got = synth.limbs_to_ints(P.from_limb_tensor(h.reshape(-1, 2 * key.L)))
    assert got == [H[v][f][b][k] for v in range(2) for f in range(tree["F"]) for b in range(tree["K"])
                   for k in range(2)]
