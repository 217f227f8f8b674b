"""Secure vertical inference with partially-saved models (Sec. IV.A): two
parties each keep only the splits on their own features; the joint inference
reaches the same node for every sample as the centralized model (the oracle's
routing with the full tree), and so gives the same prediction."""

import numpy as np
import pytest
import torch

import oracle
from oracle import tree as otree
from paper_2504_03909_b300 import paillier as P, synth

pytestmark = pytest.mark.gpu


def test_partially_saved_models_predict_like_the_full_model():
    n_bits, M, F, K, depth, seed = 1024, 3000, 8, 32, 4, 12
    p, q = synth.gen_primes(n_bits, seed)
    key = P.Key.from_primes(n_bits, p, q)
    gh = synth.gen_gh(M, seed)
    r = synth.gen_r(p * q, n_bits, 2 * M, seed, p, q)
    bins = synth.gen_bins_quantile(F, M, K, seed)
    m = P.encode(torch.from_numpy(gh.reshape(-1)).cuda())
    ct = P.encrypt(key, m, P.to_limb_tensor(r))
    ctm = P.ct_prepare(key, ct.view(2, M, -1))
    bins_d = torch.from_numpy(bins).cuda()
    plan = P.LevelPlan(key, M, F, K, 1 << (depth - 1))
    node = torch.zeros(M, dtype=torch.int32, device="cuda")
    tree_f, tree_b, weights = [], [], []
    for lvl in range(depth):
        nn = 1 << lvl
        hist, cnt = plan.run(ctm, bins_d, node, nn)
        sums = P.decrypt_u64(key, hist.reshape(-1, 2 * key.L)).view(nn, F, K, 2)
        w = P.leaf_weights(sums, cnt, 1.0)
        if lvl + 1 < depth:
            bf, bb, _ = P.split_find(sums, cnt, 1.0, 0.0, 1.0)
            node = P.split_apply(bins_d, node, bf, bb)
        else:
            bf = torch.full((nn,), -1, dtype=torch.int32, device="cuda")
            bb = bf.clone()
        P.sync()
        # leaf weights against the oracle's formula on the decrypted sums
        s_np, c_np = sums.cpu().numpy().view(np.uint64), cnt.cpu().numpy()
        for v in range(nn):
            want = otree.leaf_weight(int(s_np[v, 0, :, 0].sum()), int(s_np[v, 0, :, 1].sum()), int(c_np[v, 0].sum()),
                                     1.0)
            if c_np[v, 0].sum() > 0:
                assert w[v].item() == want
        tree_f += bf.cpu().tolist()
        tree_b += bb.cpu().tolist()
        weights += w.cpu().tolist()
    tf = torch.tensor(tree_f, dtype=torch.int32, device="cuda")
    tb = torch.tensor(tree_b, dtype=torch.int32, device="cuda")
    nodes = len(tree_f)
    # two parties: features [0, 4) and [4, 8); each evaluates only its own splits
    go = torch.full((nodes, M), 255, dtype=torch.uint8, device="cuda")
    for lo, hi in synth.feature_split(F, 2):
        P.tree_decide(bins_d[lo:hi].contiguous(), lo, tf, tb, go)
    leaf = P.tree_route(go, tf, depth)
    P.sync()
    want = otree.predict_leaf(bins, tree_f, tree_b, depth)
    assert leaf.cpu().tolist() == want
    # every split node's decisions were written by exactly its owning party
    gnp = go.cpu().numpy()
    for t, f in enumerate(tree_f):
        assert (gnp[t] != 255).all() == (f >= 0)
    # predictions of the joint model = the full model's leaf weights
    pred = np.array(weights)[leaf.cpu().numpy()]
    assert np.array_equal(pred, np.array(weights)[np.array(want)])
    assert sum(1 for f in tree_f if f >= 0) >= 3
