"""Oracle for tree building on the decrypted histograms (test infrastructure).

Sec. III.B of the paper: the active party decrypts the cumulative histograms
and uses them for tree building; Sec. IV: the secure vertical trees have the
same structure as the non-secure ones.  The split criterion is XGBoost's exact
histogram gain (T. Chen, C. Guestrin, "XGBoost: A Scalable Tree Boosting
System", KDD 2016):

    score(G, H) = G^2 / (H + lambda)
    gain = 0.5 * (score(G_L, H_L) + score(G_R, H_R) - score(G, H)) - gamma

for the split "bin <= b goes left", b = 0 .. K-2, with H_L, H_R >=
min_child_weight.  G and H are the decoded fixed-point sums (exact rationals
with denominator 2^24, exactly representable as floats here); the gain is
evaluated with Python floats (IEEE double, one rounding per operation, in the
order written).  The best split is the first maximum with gain > 0 in
(feature, bin) order; a node without one is a leaf (feature -1).

Plain loops; pinned by tests/test_oracle_tree.py.
"""

from .paillier import OFFSET


def _dec(s: int, c: int) -> float:
    return float(s - c * OFFSET) / OFFSET


def split_find(sums, counts, lam: float, gamma: float, min_child_weight: float):
    """sums[v][f][b] = [S_g, S_h] (fixed-point integer sums), counts[v][f][b].
    Returns lists best_f, best_b, best_gain over nodes v."""
    best_f, best_b, best_gain = [], [], []
    for v in range(len(sums)):
        bf, bb, bg = -1, -1, 0.0
        for f in range(len(sums[v])):
            cells = sums[v][f]
            cnt = counts[v][f]
            K = len(cells)
            Sg = sum(int(c[0]) for c in cells)
            Sh = sum(int(c[1]) for c in cells)
            C = sum(int(x) for x in cnt)
            G, H = _dec(Sg, C), _dec(Sh, C)
            parent = G * G / (H + lam)
            Lg = Lh = Lc = 0
            for b in range(K - 1):
                Lg += int(cells[b][0])
                Lh += int(cells[b][1])
                Lc += int(cnt[b])
                GL, HL = _dec(Lg, Lc), _dec(Lh, Lc)
                GR, HR = _dec(Sg - Lg, C - Lc), _dec(Sh - Lh, C - Lc)
                if not (HL >= min_child_weight and HR >= min_child_weight):
                    continue
                gain = 0.5 * ((GL * GL / (HL + lam) + GR * GR / (HR + lam)) - parent) - gamma
                if gain > bg:
                    bf, bb, bg = f, b, gain
        best_f.append(bf)
        best_b.append(bb)
        best_gain.append(bg if bf >= 0 else 0.0)
    return best_f, best_b, best_gain


def split_apply(bins, node, best_f, best_b):
    """Next-level node of every sample: 2 v + (bin > b) under its node's split,
    -1 for samples outside any node or in a leaf."""
    out = []
    for i in range(len(node)):
        v = int(node[i])
        if v < 0 or best_f[v] < 0:
            out.append(-1)
        else:
            out.append(2 * v + (1 if int(bins[best_f[v]][i]) > best_b[v] else 0))
    return out


def predict_leaf(bins, tree_f, tree_b, depth):
    """Centralized inference (the full model): level-order index of the node each
    sample reaches, following "bin <= b goes left" until a leaf or the last level."""
    out = []
    for i in range(len(bins[0])):
        v, first = 0, 0
        for lvl in range(depth):
            t = first + v
            if tree_f[t] < 0 or lvl == depth - 1:
                break
            v = 2 * v + (1 if int(bins[tree_f[t]][i]) > tree_b[t] else 0)
            first = 2 * first + 1
        out.append(first + v)
    return out


def leaf_weight(S_g: int, S_h: int, count: int, lam: float) -> float:
    """XGBoost's optimal leaf weight -G / (H + lambda) from fixed-point sums."""
    G, H = _dec(S_g, count), _dec(S_h, count)
    return -G / (H + lam)
