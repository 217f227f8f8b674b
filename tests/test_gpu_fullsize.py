"""Parity at the workloads' full sizes, in the launch configuration bench.py
times (default key configuration), on outputs the oracle can compute one by
one, plus properties that hold at any size:

* level workload (250,000 samples x 30 features x 256 bins, 2048-bit n):
  a seeded sample of 4,096 ciphertexts bit-exact vs the oracle; EVERY decrypted
  histogram cell equal to the plaintext fixed-point histogram (so every
  ciphertext is consistent through the homomorphism); EVERY root cell (15,360
  products of about 1,000 ciphertexts each) bit-exact vs the oracle's product;
  8 sampled decryptions vs the lambda form; every decoded float64 cell equal
  to the oracle's exact decode.
* batched workload (same data, depth-6 Beta(0.5, 0.5) tree): every level
  through the captured graph, every decrypted cell of every level equal to the
  plaintext histogram; 4,096 distinct sampled cells of every level below the
  root (the root is the level workload's) bit-exact vs the oracle's product;
  batched == plain per-node at the deepest level.
* large workload's kernel shapes (3072-bit n, 64 log-normal features, 256
  bins) on 20,000 samples and a depth-3 tree; 257 sampled ciphertexts (the
  last one included) bit-exact vs the oracle.
Tolerance: none (bit-exact integers).
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2504_03909_b300 import paillier as P, synth

from helpers import oracle_cells_many, oracle_decrypt_many, oracle_encrypt_many, sample_cells

pytestmark = pytest.mark.gpu


def _setup(cfg, M=None, F=None, depth=None):
    cfg = dict(cfg)
    if M:
        cfg["M"] = M
    if F:
        cfg["F"] = F
    M, F, K, n_bits = cfg["M"], cfg["F"], cfg["K"], cfg["n_bits"]
    seed = cfg.get("data_seed", cfg["seed"])
    p, q = synth.gen_primes(n_bits, seed)
    key = P.Key.from_primes(n_bits, p, q)
    gh = synth.gen_gh(M, seed)
    r = synth.gen_r(p * q, n_bits, 2 * M, seed, p, q)
    bins = synth.make_bins(dict(cfg, seed=seed))
    m = P.encode(torch.from_numpy(gh.reshape(-1)).cuda())
    ct = P.encrypt(key, m, P.to_limb_tensor(r))
    ctm = P.ct_prepare(key, ct.view(2, M, -1))
    P.sync()
    ms = [oracle.encode(x) for x in gh.reshape(-1)]
    assert m.cpu().numpy().view(np.uint64).tolist() == ms  # every plaintext encoded as the oracle does
    return dict(cfg=cfg, p=p, q=q, n=p * q, key=key, gh=gh, r=r, bins=bins, m=np.array(ms, dtype=np.int64),
                ct=ct, ctm=ctm, bins_d=torch.from_numpy(bins).cuda())


@pytest.fixture(scope="module")
def level():
    return _setup(synth.CONFIGS["level"])


def test_level_sampled_ciphertexts_bit_exact(level):
    M = level["cfg"]["M"]
    idx = sorted(synth.rng_misc(21).choice(2 * M, size=4096, replace=False).tolist())
    rs = synth.limbs_to_ints(level["r"][idx])
    want = oracle_encrypt_many(level["n"], [int(level["m"][i]) for i in idx], rs)
    got = synth.limbs_to_ints(P.from_limb_tensor(level["ct"][idx]))
    assert got == want


def test_level_root_histogram_every_cell_and_sampled_products(level, tmp_path):
    cfg, key = level["cfg"], level["key"]
    M, F, K = cfg["M"], cfg["F"], cfg["K"]
    node = torch.zeros(M, dtype=torch.int32, device="cuda")
    hist, cnt = P.hist_aggregate(key, level["ctm"], level["bins_d"], node, 1, K)
    sums = P.decrypt_u64(key, hist.reshape(-1, 2 * key.L))
    P.sync()
    ps, pc = oracle.plain_histogram_np(level["m"][:M], level["m"][M:], level["bins"], np.zeros(M, np.int64), 1, K)
    assert np.array_equal(sums.cpu().numpy().reshape(1, F, K, 2), ps)
    assert np.array_equal(cnt.cpu().numpy(), pc)
    # A9: every decoded cell (g and h) equals the oracle's exact decode, rounded once to float64
    cnt2 = cnt.reshape(1, F, K, 1).expand(1, F, K, 2).contiguous()
    dec = P.decode(sums.reshape(-1), cnt2.reshape(-1))
    P.sync()
    want_dec = [float(oracle.decode(int(s_), int(c_)))
                for s_, c_ in zip(ps.reshape(-1).tolist(), cnt2.reshape(-1).cpu().tolist())]
    assert dec.cpu().numpy().tolist() == want_dec
    # every cell (g and h) of the root: the oracle's product of the cell's ciphertexts
    rng = synth.rng_misc(22)
    cells = sample_cells(rng, [0], F, K, F * K * 2)
    want = oracle_cells_many(str(tmp_path), level["n"], P.from_limb_tensor(level["ct"]), level["bins"],
                             np.zeros((1, M), np.int32), cells)
    got = P.from_limb_tensor(hist[0])
    assert [synth.limbs_to_ints(got[f, b, k][None])[0] for _, _, f, b, k in cells] == want
    # sampled decryptions against the textbook lambda form
    flat = P.from_limb_tensor(hist.reshape(-1, 2 * key.L))
    pick = rng.choice(flat.shape[0], size=8, replace=False)
    want = oracle_decrypt_many(level["p"], level["q"], synth.limbs_to_ints(flat[pick]))
    assert sums.reshape(-1).cpu().numpy()[pick].tolist() == want


def test_batched_depth6_every_level_every_cell(level, tmp_path):
    cfg, key = level["cfg"], level["key"]
    M, F, K = cfg["M"], cfg["F"], cfg["K"]
    bcfg = synth.CONFIGS["batched"]
    levels = synth.gen_tree_levels(M, bcfg["depth"], bcfg["seed"])
    maxn = 1 << (bcfg["depth"] - 1)
    plan = P.LevelPlan(key, M, F, K, maxn)
    node_buf = torch.empty(M, dtype=torch.int32, device="cuda")
    hist = torch.empty((maxn, F, K, 2, 2 * key.L), dtype=torch.int32, device="cuda")
    cnt = torch.empty((maxn, F, K), dtype=torch.int32, device="cuda")
    rng = synth.rng_misc(23)
    cells = sample_cells(rng, range(1, len(levels)), F, K, 4096)
    got_cells = {}
    for lvl, node_np in enumerate(levels):
        nn = 1 << lvl
        node_buf.copy_(torch.from_numpy(node_np))
        plan.run(level["ctm"], level["bins_d"], node_buf, nn, hist=hist, count=cnt)
        sums = P.decrypt_u64(key, hist[:nn].reshape(-1, 2 * key.L))
        P.sync()
        ps, pc = oracle.plain_histogram_np(level["m"][:M], level["m"][M:], level["bins"], node_np, nn, K)
        assert np.array_equal(sums.cpu().numpy().reshape(nn, F, K, 2), ps), lvl
        assert np.array_equal(cnt[:nn].cpu().numpy(), pc), lvl
        got = P.from_limb_tensor(hist[:nn])
        for c in cells:
            if c[0] == lvl:
                got_cells[c] = synth.limbs_to_ints(got[c[1], c[2], c[3], c[4]][None])[0]
        if lvl == len(levels) - 1:
            h2, c2 = P.hist_aggregate(key, level["ctm"], level["bins_d"], node_buf, nn, K, per_node=True)
            P.sync()
            assert torch.equal(h2, hist[:nn]) and torch.equal(c2, cnt[:nn])
    assert plan.stats()["captures"] == 1
    # 4,096 sampled cells of every level below the root vs the oracle's product
    want = oracle_cells_many(str(tmp_path), level["n"], P.from_limb_tensor(level["ct"]), level["bins"],
                             np.stack(levels).astype(np.int32), cells)
    assert [got_cells[c] for c in cells] == want


def test_large_shapes_3072bit():
    d = _setup(synth.CONFIGS["large"], M=20_000)
    cfg, key = d["cfg"], d["key"]
    M, F, K = cfg["M"], cfg["F"], cfg["K"]
    idx = sorted(set(synth.rng_misc(23).choice(2 * M, size=256, replace=False).tolist()) | {2 * M - 1})
    want = oracle_encrypt_many(d["n"], [int(d["m"][i]) for i in idx], synth.limbs_to_ints(d["r"][idx]))
    assert synth.limbs_to_ints(P.from_limb_tensor(d["ct"][idx])) == want
    levels = synth.gen_tree_levels(M, 3, cfg["seed"])
    plan = P.LevelPlan(key, M, F, K, 4)
    node_buf = torch.empty(M, dtype=torch.int32, device="cuda")
    pub = oracle.PublicKey(d["n"])
    cts_h = synth.limbs_to_ints(P.from_limb_tensor(d["ct"][M:]))
    for lvl, node_np in enumerate(levels):
        nn = 1 << lvl
        node_buf.copy_(torch.from_numpy(node_np))
        hist, cnt = plan.run(d["ctm"], d["bins_d"], node_buf, nn)
        sums = P.decrypt_u64(key, hist.reshape(-1, 2 * key.L))
        P.sync()
        ps, pc = oracle.plain_histogram_np(d["m"][:M], d["m"][M:], d["bins"], node_np, nn, K)
        assert np.array_equal(sums.cpu().numpy().reshape(nn, F, K, 2), ps), lvl
        assert np.array_equal(cnt.cpu().numpy(), pc), lvl
    # sampled cells of the deepest level, h ciphertexts
    rng = synth.rng_misc(24)
    got = P.from_limb_tensor(hist[:, :, :, 1])
    for _ in range(6):
        v, f, b = int(rng.integers(nn)), int(rng.integers(F)), int(rng.integers(K))
        want = oracle.encrypted_histogram_cell(pub, cts_h, d["bins"], levels[-1], v, f, b)
        assert synth.limbs_to_ints(got[v, f, b][None])[0] == want
