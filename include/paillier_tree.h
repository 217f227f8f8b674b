/*
 * paillier_tree.h -- tree building on the decrypted histograms (Sec. III.B:
 * the active party decrypts the cumulative histograms and uses them "for tree
 * building"; Sec. IV: the secure vertical trees equal the non-secure ones).
 *
 * Split finding is XGBoost's exact histogram gain (Chen & Guestrin, KDD 2016):
 *   score(G, H) = G^2 / (H + lambda)
 *   gain = 0.5 * (score(G_L, H_L) + score(G_R, H_R) - score(G, H)) - gamma
 * for the split "bin <= b goes left", over every feature f and bin b < K - 1,
 * subject to H_L >= min_child_weight and H_R >= min_child_weight.  G, H are the
 * decoded fixed-point sums: G = (S_g - count * 2^24) / 2^24, exact in float64
 * (prefix sums are taken on the exact integers first).  The gain is evaluated
 * in IEEE float64 with one rounding per operation in the order written above
 * (no fused multiply-add), so the result is reproducible bit for bit.  The
 * best split of a node is the largest gain > 0; ties go to the lowest feature,
 * then the lowest bin.  A node without a positive-gain split is a leaf.
 */
#ifndef PAILLIER_B300_TREE_H
#define PAILLIER_B300_TREE_H

#include <stddef.h>
#include <stdint.h>

#include "paillier.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Best split per node from decrypted histogram sums.
 *   d_sums   : [nodes][F][K][2] uint64 fixed-point sums (g, h) (decrypted cells)
 *   d_counts : [nodes][F][K] int32 sample counts
 *   d_best_f, d_best_b : [nodes] out: feature and bin of the best split, -1 for a leaf
 *   d_best_gain        : [nodes] out (may be NULL): its gain (0 for a leaf) */
pl_status paillier_split_find(const uint64_t* d_sums, const int32_t* d_counts, int nodes, int F, int K,
                              double lambda, double gamma, double min_child_weight,
                              int32_t* d_best_f, int32_t* d_best_b, double* d_best_gain, void* stream);

/* Node membership of the next level: for sample i in node v = d_node[i] >= 0
 * with split (f, b) = (d_best_f[v], d_best_b[v]), f >= 0:
 * d_next[i] = 2 v + (d_bins[f * M + i] > b); d_next[i] = -1 if d_node[i] < 0 or
 * node v is a leaf.  (In the vertical setting the party owning feature f
 * applies its own split; here the parties are simulated on one device.)
 *   d_bins [F][M]; d_node [M]; d_best_f, d_best_b [nodes]; d_next [M] out.
 * A node id >= nodes or a split feature >= F writes -1 for that sample and
 * sets PL_EDEVICE in the status word. */
pl_status paillier_split_apply(const uint8_t* d_bins, size_t M, int F, const int32_t* d_node, int nodes,
                               const int32_t* d_best_f, const int32_t* d_best_b, int32_t* d_next, void* stream);

/* Histogram subtraction (XGBoost's trick; the paper does not use it): at a
 * level below the root only the smaller child of every split node needs an
 * encrypted histogram; the sibling's decrypted sums are the parent's minus the
 * child's, exact integer arithmetic on the fixed-point sums and counts.
 *
 * paillier_child_select: from the children's node ids d_next [M] (2 v and
 * 2 v + 1, -1 outside) and the parents' decrypted counts, picks the smaller
 * child of each parent node v (fewer samples; ties -> the left child) and
 * writes d_small_node [M] = v for the samples of that child, -1 for all
 * others: a node array of parents.  nodes = number of parents.  d_small_right
 * [nodes] (out) = 1 if the smaller child is the right one.  The parent's split
 * (d_best_f, d_best_b) gives the child sizes from d_counts [nodes][F][K].
 * A child id >= 2 nodes or a split feature >= F is skipped (-1, left) and
 * sets PL_EDEVICE in the status word. */
pl_status paillier_child_select(const int32_t* d_next, size_t M, const int32_t* d_counts, int nodes, int F, int K,
                                const int32_t* d_best_f, const int32_t* d_best_b, int32_t* d_small_right,
                                int32_t* d_small_node, void* stream);

/* Full child level from the parents' and the smaller children's decrypted
 * histograms: for parent v, child (2 v + s) with s = d_small_right[v] gets
 * d_small_sums[v] and the other child gets d_parent_sums[v] - d_small_sums[v]
 * (and the same for counts).  Layouts [nodes][F][K][2] (sums, uint64) and
 * [nodes][F][K] (counts) for parents and small children; [2 nodes][F][K][2]
 * and [2 nodes][F][K] out.  Any non-zero d_small_right[v] means "right". */
pl_status paillier_child_subtract(const uint64_t* d_parent_sums, const int32_t* d_parent_counts,
                                  const uint64_t* d_small_sums, const int32_t* d_small_counts,
                                  const int32_t* d_small_right, int nodes, int F, int K, uint64_t* d_child_sums,
                                  int32_t* d_child_counts, void* stream);

/* ------------------------------------------------ inference (Sec. IV.A) --
 * A partially-saved model: every party keeps the splits of the nodes whose
 * feature it owns and "nan" for the others.  Inference runs the model jointly:
 * each party evaluates its own splits on its own features, and the decisions
 * are combined by walking the tree; the prediction equals the centralized
 * model's.  Trees here are complete binary trees in level order: node v of
 * level l is index (2^l - 1) + v, its children 2v and 2v + 1 of level l + 1. */

/* One party's decisions: for every tree node t (level order, `nodes` in all)
 * whose feature d_tree_f[t] lies in [f_lo, f_lo + F_party), and every sample
 * i: d_go_right[t * M + i] = (d_bins_party[(f - f_lo) * M + i] > d_tree_b[t]).
 * Entries of nodes owned by other parties or leaves (d_tree_f[t] < 0) are not
 * written. */
pl_status paillier_tree_decide(const uint8_t* d_bins_party, int F_party, int f_lo, size_t M, const int32_t* d_tree_f,
                               const int32_t* d_tree_b, int nodes, uint8_t* d_go_right, void* stream);

/* Routing with the combined decisions: from the root, follow d_go_right of
 * each split node until a leaf (d_tree_f < 0) or `depth` levels; d_leaf[i] is
 * the level-order index of the node reached.  d_tree_f holds at least
 * 2^depth - 1 nodes and d_go_right [2^depth - 1][M] (only the entries of
 * split nodes are read; any non-zero byte means "right"). */
pl_status paillier_tree_route(const uint8_t* d_go_right, size_t M, const int32_t* d_tree_f, int depth,
                              int32_t* d_leaf, void* stream);

/* XGBoost leaf weights w = -G / (H + lambda) of `nodes` nodes from their
 * decrypted sums [nodes][F][K][2] and counts [nodes][F][K] (feature 0's bins
 * hold every sample of the node). */
pl_status paillier_leaf_weights(const uint64_t* d_sums, const int32_t* d_counts, int nodes, int F, int K,
                                double lambda, double* d_w, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PAILLIER_B300_TREE_H */
