"""The full secure tree loop on the GPU (encrypt -> per-level encrypted
histograms -> CRT decrypt -> split finding -> node update) equals the tree the
oracle builds from the plaintext histograms: the same split (feature, bin,
float64 gain, bit for bit) at every node and the same node of every sample at
every level (Sec. IV: secure vertical trees have the same structure as the
non-secure ones)."""

import numpy as np
import pytest
import torch

import oracle
from oracle import tree as otree
from paper_2504_03909_b300 import paillier as P, synth

pytestmark = pytest.mark.gpu


def _secure_vs_plain(n_bits, M, F, K, depth, seed, lam=1.0, gamma=0.0, mcw=1.0, subtract=False, pack_bits=0,
                     gh_bits=0):
    """gh_bits > 0: g/h packed, one ciphertext per sample (enc(g) + 2^B enc(h));
    pack_bits is then ignored in favour of slots of 2 gh_bits bits."""
    p, q = synth.gen_primes(n_bits, seed)
    key = P.Key.from_primes(n_bits, p, q)
    gh = synth.gen_gh(M, seed)
    r = synth.gen_r(p * q, n_bits, 2 * M, seed, p, q)
    bins = synth.gen_bins_quantile(F, M, K, seed)
    bins_d = torch.from_numpy(bins).cuda()
    if gh_bits:
        g_d, h_d = torch.from_numpy(gh[0].copy()).cuda(), torch.from_numpy(gh[1].copy()).cuda()
        ctm = P.ct_prepare(key, P.encrypt_gh(key, P.encode_gh(g_d, h_d, gh_bits), P.to_limb_tensor(r[:M])))

        class _Plan:  # the g/h-packed histogram of one level
            def run(self, ctm, bins_d, node, nn):
                return P.hist_aggregate_gh(key, ctm, bins_d, node, nn, K)
        plan = _Plan()
    else:
        m = P.encode(torch.from_numpy(gh.reshape(-1)).cuda())
        ct = P.encrypt(key, m, P.to_limb_tensor(r))
        ctm = P.ct_prepare(key, ct.view(2, M, -1))
        plan = P.LevelPlan(key, M, F, K, 1 << (depth - 1))
    node = torch.zeros(M, dtype=torch.int32, device="cuda")
    ms = [oracle.encode(x) for x in gh.reshape(-1)]
    onode = [0] * M
    prev = None  # (sums, counts, best_f, best_b) of the parent level
    for lvl in range(depth):
        nn = 1 << lvl

        def decrypt(h):
            cells = h.reshape(-1, 2 * key.L)
            if gh_bits and pack_bits:
                return P.decrypt_packed_gh(key, P.pack(key, cells, 2 * gh_bits), cells.shape[0], gh_bits)
            if gh_bits:
                return P.decrypt_gh(key, cells, gh_bits)
            if pack_bits:
                return P.decrypt_packed_u64(key, P.pack(key, cells, pack_bits), cells.shape[0], pack_bits)
            return P.decrypt_u64(key, cells)

        if subtract and prev is not None:
            psums, pcnt, pf, pb = prev
            small_right, small_node = P.child_select(node, pcnt, pf, pb)
            hist, scnt = plan.run(ctm, bins_d, small_node, nn // 2)
            ssums = decrypt(hist).view(nn // 2, F, K, 2)
            sums, cnt = P.child_subtract(psums, pcnt, ssums, scnt, small_right)
        else:
            hist, cnt = plan.run(ctm, bins_d, node, nn)
            sums = decrypt(hist).view(nn, F, K, 2)
        bf, bb, bg = P.split_find(sums, cnt, lam, gamma, mcw)
        prev = (sums.clone(), cnt.clone(), bf, bb)
        nxt = P.split_apply(bins_d, node, bf, bb)
        P.sync()
        # oracle: plaintext histogram of the same node assignment, same split rule
        psums, pcnt = oracle.plain_histogram(ms[:M], ms[M:], bins, onode, nn, K)
        of, ob, og = otree.split_find(psums, pcnt, lam, gamma, mcw)
        assert bf.cpu().tolist() == of and bb.cpu().tolist() == ob, lvl
        assert bg.cpu().tolist() == og, lvl                 # float64 gains bit for bit
        onode = otree.split_apply(bins, onode, of, ob)
        assert nxt.cpu().tolist() == onode, lvl
        node = nxt
    return sum(1 for f in of if f >= 0)


def test_secure_tree_equals_plaintext_tree_1024():
    assert _secure_vs_plain(1024, 1500, 5, 16, 4, seed=8) > 0


def test_secure_tree_equals_plaintext_tree_2048():
    assert _secure_vs_plain(2048, 6000, 8, 64, 5, seed=9, lam=0.5, gamma=0.01, mcw=2.0) > 0


def test_secure_tree_with_subtraction_and_packing_equals_plaintext_tree():
    assert _secure_vs_plain(2048, 6000, 8, 64, 5, seed=9, lam=0.5, gamma=0.01, mcw=2.0, subtract=True,
                            pack_bits=40) > 0
    assert _secure_vs_plain(1024, 1500, 5, 16, 4, seed=8, subtract=True) > 0


def test_gh_packed_secure_tree_equals_plaintext_tree():
    """One ciphertext per sample carrying g and h: the same splits, gains and
    node assignments as the plaintext tree (with and without ciphertext packing
    and subtraction)."""
    assert _secure_vs_plain(2048, 6000, 8, 64, 5, seed=9, lam=0.5, gamma=0.01, mcw=2.0, subtract=True,
                            pack_bits=1, gh_bits=40) > 0
    assert _secure_vs_plain(1024, 1500, 5, 16, 4, seed=8, gh_bits=38) > 0
