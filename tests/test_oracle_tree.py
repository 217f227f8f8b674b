"""Pins for the tree-building oracle: a hand-derived gain table, a planted
threshold the best split must find, sample-order invariance, and the leaf and
tie rules."""

import numpy as np

import oracle
from oracle import tree
from paper_2504_03909_b300 import synth

OFF = oracle.OFFSET


def _cells(gh):
    """[(G, H, count)] per bin -> fixed-point sums with one sample per unit of count."""
    return [[(g + c) * OFF, (h + c) * OFF] for g, h, c in gh], [c for _, _, c in gh]


def test_hand_derived_gains():
    # feature 0: bins with (G, H) = (-2,1), (-1,1), (1,1), (2,1); lambda = 1, gamma = 0.
    #   split after bin 0: 0.5 * (4/2 + 4/4 - 0/5) = 1.5
    #   split after bin 1: 0.5 * (9/3 + 9/3 - 0)   = 3.0   <- best
    #   split after bin 2: 1.5
    # feature 1: every bin (0, 1): gain 0 everywhere.
    s0, c0 = _cells([(-2, 1, 1), (-1, 1, 1), (1, 1, 1), (2, 1, 1)])
    s1, c1 = _cells([(0, 1, 1)] * 4)
    bf, bb, bg = tree.split_find([[s0, s1]], [[c0, c1]], 1.0, 0.0, 0.0)
    assert (bf, bb, bg) == ([0], [1], [3.0])
    # gamma larger than every gain -> leaf
    assert tree.split_find([[s0, s1]], [[c0, c1]], 1.0, 3.5, 0.0)[0] == [-1]
    # min_child_weight 2.5 forbids every split of 4 unit-weight bins except none -> leaf
    assert tree.split_find([[s0, s1]], [[c0, c1]], 1.0, 0.0, 2.5)[0] == [-1]


def test_ties_go_to_lowest_feature_then_bin():
    s, c = _cells([(-1, 1, 1), (1, 1, 1), (-1, 1, 1), (1, 1, 1)])
    bf, bb, _ = tree.split_find([[s, s]], [[c, c]], 1.0, 0.0, 0.0)
    # both features identical: feature 0; within it bins 0 and 2 tie -> bin 0
    assert bf == [0] and bb == [0]


def test_planted_threshold_is_found():
    rng = synth.rng_misc(31)
    M, F, K = 4000, 6, 16
    bins = rng.integers(0, K, size=(F, M))
    y = (bins[3] > 9).astype(np.float64)        # label decided by feature 3, threshold after bin 9
    g = 0.5 - y                                  # logistic gradient at p = 0.5
    h = np.full(M, 0.25)
    mg = [oracle.encode(x) for x in g]
    mh = [oracle.encode(x) for x in h]
    sums, counts = oracle.plain_histogram(mg, mh, bins, np.zeros(M, int), 1, K)
    bf, bb, bg = tree.split_find(sums, counts, 1.0, 0.0, 0.0)
    assert (bf[0], bb[0]) == (3, 9) and bg[0] > 0
    nxt = tree.split_apply(bins, np.zeros(M, int), bf, bb)
    assert nxt == [int(b > 9) for b in bins[3]]
    # the same data in another sample order gives the same split
    perm = rng.permutation(M)
    s2, c2 = oracle.plain_histogram([mg[i] for i in perm], [mh[i] for i in perm], bins[:, perm],
                                    np.zeros(M, int), 1, K)
    assert tree.split_find(s2, c2, 1.0, 0.0, 0.0) == (bf, bb, bg)


def test_split_apply_leaves_and_excluded():
    bins = np.array([[0, 5, 9, 3]])
    node = np.array([0, 0, -1, 1])
    assert tree.split_apply(bins, node, [0, -1], [4, -1]) == [0, 1, -1, -1]


def test_predict_leaf_and_leaf_weight():
    # depth-2 tree: root splits on feature 1 at bin 3; left child is a leaf; right child splits feature 0 at bin 0
    tree_f = [1, -1, 0]
    tree_b = [3, -1, 0]
    bins = [[0, 1, 0, 5], [2, 4, 9, 3]]
    # sample 0: f1=2 <= 3 -> left (node 1, leaf); sample 1: f1=4 > 3 -> node 2, f0=1 > 0 -> right -> level 2 node 3 -> index 6
    # sample 2: f1=9 -> node 2, f0=0 <= 0 -> index 5; sample 3: f1=3 -> left -> index 1
    assert tree.predict_leaf(bins, tree_f + [-1] * 4, tree_b + [-1] * 4, 3) == [1, 6, 5, 1]
    # weight: G = -1.5, H = 0.5, lambda = 1 -> 1.0 ; encoded sums of 3 samples
    S_g = int((-1.5 + 3) * OFF)
    S_h = int((0.5 + 3) * OFF)
    assert tree.leaf_weight(S_g, S_h, 3, 1.0) == 1.0
