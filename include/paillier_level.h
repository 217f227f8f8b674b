/*
 * paillier_level.h -- the batched tree-level path and the launch autotuner.
 *
 * Batching (Sec. III.B at every level of a tree; Sec. IV.B trains trees of
 * depth 5 with 256 bins): every node of a tree level is aggregated in ONE pass
 * -- one set of launches whose segmented-product kernel is persistent over a
 * device-side work list of fixed-size chunks, so nodes of very different sizes
 * balance inside one launch.  The level's launch set is captured once into a
 * CUDA graph and the graph is replayed for every later level: the node count
 * of the level is written to device memory before each replay, and the kernels
 * read it from there.
 */
#ifndef PAILLIER_B300_LEVEL_H
#define PAILLIER_B300_LEVEL_H

#include <stddef.h>
#include <stdint.h>

#include "paillier.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pl_level_plan pl_level_plan;

/* A plan for M samples, F features, K <= 256 bins and levels of up to
 * max_nodes nodes.  It owns its scratch (allocated here, on the current
 * device: sample ids, offsets, work list, partial products), a capture stream
 * and the graph.  The key must outlive the plan; the launch configuration of
 * the key (lanes, tile) is frozen into the plan at creation. */
pl_status paillier_level_plan_create(const pl_key* key, size_t M, int F, int K, int max_nodes,
                                     pl_level_plan** out);

/* The same for ONE g/h-packed ciphertext array per sample (see paillier_pack.h):
 * paillier_level_run then takes d_ctm [M][2L] and writes
 * d_hist [num_nodes][F][K][2L], as paillier_hist_aggregate_gh. */
pl_status paillier_level_plan_create_gh(const pl_key* key, size_t M, int F, int K, int max_nodes,
                                        pl_level_plan** out);

/* The encrypted histogram of one level, same layouts and results as
 * paillier_hist_aggregate:  d_ctm [2][M][2L], d_bins [F][M], d_node [M]
 * (values -1 .. num_nodes-1), d_hist [num_nodes][F][K][2][2L] out,
 * d_count [num_nodes][F][K] out (may be NULL), 1 <= num_nodes <= max_nodes.
 * The first call captures the launch set into a CUDA graph; later calls with
 * the same buffers replay it (new node contents and node counts are fine).
 * Calls with other buffers re-capture.  Asynchronous on `stream` (not the
 * legacy default stream: the graph is launched on it). */
pl_status paillier_level_run(pl_level_plan* plan, const uint32_t* d_ctm, const uint8_t* d_bins,
                             const int32_t* d_node, int num_nodes, uint32_t* d_hist, int32_t* d_count,
                             void* stream);

/* Counters of a plan: graph captures, graph replays, kernel nodes per graph. */
pl_status paillier_level_plan_stats(const pl_level_plan* plan, int* captures, int* replays, int* kernels);

/* Frees the plan (synchronises its device first). */
void paillier_level_plan_free(pl_level_plan* plan);

/* ---------------------------------------------------------- autotuner -- */

#define PL_OP_ENCRYPT 0  /* exponentiation of encryption: lanes x window */
#define PL_OP_DECRYPT 1  /* exponentiation of decryption: lanes x window */
#define PL_OP_HIST    2  /* histogram products mod n^2: lanes x tile */

/* The configured lanes serve large calls.  A call too small to keep the
 * GPU's multiply-add pipes busy (at most about 1.5 warps per SM
 * sub-partition at the configured lanes: about 3,000 encryptions or
 * decryptions, or 2,000 packed ciphertexts, at 2048-bit) runs with twice
 * the lanes per instance where that kernel exists: fewer, faster instances,
 * shorter latency; the results are the same bits. */

/* Current configuration of an op on this key: lanes per instance (limbs per
 * lane = limbs / lanes) and the window width (ops 0, 1) or tile (op 2).
 * Encryption with 4 lanes at 2048-bit or 8 at 3072-bit runs as two launches:
 * the first exponentiation (mod p and mod q, half the limbs) at half the
 * lanes, then the second (mod p^2 and mod q^2) at the configured lanes, so
 * that both keep the same limbs per lane; other settings run one launch. */
pl_status paillier_get_config(const pl_key* key, int op, int* lanes, int* param);

/* Sets a configuration (checked against the compiled kernel shapes:
 * windows 2..7, tiles 1..4096).  Results do not depend on it, only speed. */
pl_status paillier_set_config(pl_key* key, int op, int lanes, int param);

/* Times every compiled candidate of `op` on synthetic data on the current
 * device (CUDA events on `stream`), installs the fastest in the key and
 * returns it in *lanes, *param (may be NULL).  cache_path (may be NULL) names
 * a JSON-lines file of results keyed by (op, n_bits, SM count): a matching
 * line is used without measuring, a new result is appended.  Allocates and
 * frees its own device buffers; synchronises the stream. */
pl_status paillier_autotune(pl_key* key, int op, const char* cache_path, void* stream, int* lanes, int* param);

#ifdef __cplusplus
}
#endif

#endif /* PAILLIER_B300_LEVEL_H */
