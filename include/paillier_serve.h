/*
 * paillier_serve.h -- a continuous-batching request loop for histogram +
 * decryption jobs (the paper's secure vertical round, Sec. III.B: a passive
 * party's encrypted histogram followed by the active party's decryption; the
 * processor interface of Sec. III.D hands such buffers between parties).
 *
 * A server owns `slots` CUDA streams.  Submitted requests wait in a FIFO queue;
 * a scheduler thread admits the head of the queue when a slot is free AND the
 * request's device memory (outputs + scratch, allocated stream-ordered from
 * the device's memory pool) fits under the HBM budget next to the requests
 * already running.  Admitted requests run concurrently on their slots' streams
 * and overlap on the GPU; a request's result is bit-identical whether it runs
 * alone or in a mix.  Latency is measured from submit to the completion of the
 * request's last copy (host clock, polled every few tens of microseconds).
 *
 * Ciphertexts stay resident on the device: a request points at Montgomery-form
 * ciphertexts ([.., 2L], from paillier_ct_prepare) and bins already there.
 */
#ifndef PAILLIER_B300_SERVE_H
#define PAILLIER_B300_SERVE_H

#include <stddef.h>
#include <stdint.h>

#include "paillier.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pl_server pl_server;

typedef struct pl_request {
  /* Private key: the request covers the passive party's aggregation and the
   * active party's decryption, both simulated in this process. */
  const pl_key* key;
  /* g rows at d_ctm[i * 2L], h rows at d_ctm[(gh_stride + i) * 2L], i < M
   * (gh_stride >= M rows: a request may use the first M samples of a larger
   * resident array). */
  const uint32_t* d_ctm;
  size_t gh_stride;
  size_t M;
  int F, K;                 /* 1 <= K <= 256 */
  const uint8_t* d_bins;    /* bin of sample i in feature f at d_bins[f * bins_stride + i] */
  size_t bins_stride;       /* >= M */
  const int32_t* d_node;    /* [M] node ids (-1 skips), or NULL: every sample in node 0 */
  int num_nodes;            /* >= 1 (1 when d_node is NULL) */
  /* Host outputs (page-locked memory keeps the copies asynchronous):
   * decrypted fixed-point sums [num_nodes][F][K][2] and counts [num_nodes][F][K]. */
  uint64_t* h_sums;
  int32_t* h_counts;
  /* 0: decrypt every cell; B in [1, 64]: pack the cells into B-bit slots
   * before decrypting (see paillier_pack.h; every cell sum must be < 2^B). */
  int pack_bits;
  /* 0: d_ctm holds separate g and h arrays as above.  G in [26, 64]: d_ctm
   * holds ONE g/h-packed array [M][2L] (paillier_encrypt_gh with B = G, then
   * paillier_ct_prepare; gh_stride is not used); the cells split into
   * (S_g, S_h) at bit G, and a nonzero pack_bits packs them in 2G-bit slots. */
  int gh_bits;
  /* Cells per packed ciphertext when pack_bits > 0.  N > 0: at most N (the
   * most that fit when N is larger).  0: chosen from the request -- the most
   * that fit for a request whose histogram alone is modelled at 3e12
   * multiply-adds or more (the default large_imad of pl_server_set_policy),
   * else few enough to leave at least 1,024 packed ciphertexts.  Each packed ciphertext is a chain of
   * (slots - 1) (B + 1) products mod n^2 run one after another, so for a
   * request with few cells that chain, not the GPU's throughput, bounds the
   * packing time; shorter chains cost more decryptions.  A choice of one
   * cell per ciphertext decrypts the cells directly.  The sums do not depend
   * on it. */
  int pack_slots;
} pl_request;

#define PL_REQ_QUEUED    0
#define PL_REQ_RUNNING   1
#define PL_REQ_DONE      2
#define PL_REQ_FAILED    3
#define PL_REQ_CANCELLED 4

/* Creates a server on the current device: `slots` >= 1 concurrent requests,
 * at most hbm_budget bytes of request memory in flight.  Request memory is
 * stream-ordered (cudaMallocAsync from the device's default memory pool); the
 * server sets that pool's release threshold to its maximum, so freed request
 * memory stays cached in the pool for the next request.  The setting belongs
 * to the process's default pool of this device and outlives the server;
 * memory cached there is returned by cudaMemPoolTrimTo or at process exit. */
pl_status pl_server_create(int slots, size_t hbm_budget, pl_server** out);

/* Queues a request (arguments are checked here; PL_EBUSY if it can never fit
 * the budget).  *ticket identifies it.  The request's device inputs and host
 * outputs must stay valid until it completes. */
pl_status pl_server_submit(pl_server* srv, const pl_request* req, uint64_t* ticket);

/* State of a request (PL_REQ_*), its latency in ms once done (else -1) and,
 * for a failed request, its error code in *error (may be NULL). */
pl_status pl_server_poll(pl_server* srv, uint64_t ticket, int* state, double* latency_ms, int* error);

/* Waits until the request is no longer queued or running, at most timeout_ms
 * (PL_ETIMEDOUT if it still is).  *state and *latency_ms as in poll (may be NULL). */
pl_status pl_server_wait(pl_server* srv, uint64_t ticket, int timeout_ms, int* state, double* latency_ms);

/* Device memory the server reserves against its budget while the request
 * runs (outputs and scratch), for sizing budgets. */
pl_status pl_server_request_bytes(const pl_request* req, size_t* bytes);

/* The server's plan for a request, without a server: *slots = cells per
 * packed ciphertext (0: the cells are decrypted directly) and *work_imad =
 * the modelled multiply-adds that classify it (see pl_server_set_policy).
 * Either output may be NULL. */
pl_status pl_server_request_plan(const pl_request* req, int* slots, double* work_imad);

/* Cancels a request that is still queued (PL_EINVAL if it was admitted). */
pl_status pl_server_cancel(pl_server* srv, uint64_t ticket);

/* Device scheduling and admission policy of the server (this project's
 * serving design; the paper has no serving loop).
 *   * Launches of bounded work.  The exponentiation and histogram kernels are
 *     persistent, so one launch of a large request holds every SM until it
 *     ends.  A request's work is issued as launches of at most chunk_imad
 *     modelled 32-bit multiply-add halves each: the histogram of a request
 *     without a node array by groups of features, packing and decryption by
 *     ranges of ciphertexts (a decryption launch takes at least 2,048).
 *   * Size classes.  A request whose whole modelled work is below small_imad
 *     is small, above large_imad large, else medium.  Each class runs on a
 *     stream of its own priority (small highest), so at every launch boundary
 *     the device schedules the smaller classes' pending blocks first.
 *   * Admission.  FIFO within each class: a request that cannot start (no
 *     budget, or no slot for its class) holds back only the later requests of
 *     its class.  Medium and large requests together hold at most
 *     slots - reserved_slots slots, so small requests find a slot in time.
 * Results do not depend on the policy (every launch forms the same cells).
 * Defaults: chunk_imad = small_imad = 3e11 and large_imad = 3e12 (about 25 ms
 * and 250 ms of work on a B300), reserved_slots = max(1, slots / 4) (0 for one
 * slot).  Applies to requests submitted after the call.  PL_EINVAL unless
 * chunk_imad > 0, 0 <= small_imad <= large_imad and 0 <= reserved_slots < slots. */
pl_status pl_server_set_policy(pl_server* srv, double chunk_imad, double small_imad, double large_imad,
                               int reserved_slots);

/* Aging: a large request that has run for promote_ms milliseconds issues its
 * remaining launch groups at the medium priority (ordered after its earlier
 * groups by an event), so that it stops yielding to every medium request.
 * promote_ms <= 0 turns aging off.  Default 250.  Results do not depend on it.
 * Applies to launch groups issued after the call. */
pl_status pl_server_set_aging(pl_server* srv, double promote_ms);

/* Policy counters: per_class[3] requests admitted per size class (small,
 * medium, large; may be NULL), launch groups issued (histogram feature groups,
 * packing and decryption ranges), the peak number of medium and large
 * requests running at once, and the requests promoted by aging.  Every output
 * pointer may be NULL. */
pl_status pl_server_policy_stats(pl_server* srv, long long* per_class, long long* launch_groups,
                                 int* peak_nonsmall, long long* promoted);

/* Counters: submitted, completed, failed, cancelled, peak concurrently
 * running requests, peak bytes in flight. */
pl_status pl_server_stats(pl_server* srv, long long* submitted, long long* completed, long long* failed,
                          long long* cancelled, int* peak_running, size_t* peak_bytes);

/* Waits for running requests, cancels queued ones and frees the server. */
void pl_server_destroy(pl_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* PAILLIER_B300_SERVE_H */
