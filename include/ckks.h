/*
 * ckks.h -- the secure horizontal pattern (Sec. III.A of the paper): every
 * client encrypts its local G/H histograms, the aggregating server adds the
 * ciphertexts, the clients decrypt the global histograms.  Sec. III.C picks
 * CKKS for this vector workload (one J x K histogram per encryption) and cites
 * it without restating it.  Textbook CKKS (Cheon, Kim, Kim, Song 2017)
 * restricted to encoding, public-key encryption, addition, decryption and
 * decoding, over R_q = Z_q[X]/(X^N + 1) with one prime q < 2^62, q = 1 mod 2N:
 *
 *   encode(z)  = round(scale * tau^-1(z)),  tau(m) = (m(zeta_j)) over the N/2
 *                slots, zeta_j = exp(i pi r_j / N), r_j = 5^j mod 2N
 *   keygen     b = -a s + e mod q
 *   encrypt(m) = (b v + e0 + m, a v + e1) mod q
 *   add        component-wise mod q
 *   decrypt(c) = c0 + c1 s mod q
 *   decode(m)  = tau(centred m) / scale
 *
 * Products in R_q use a negacyclic number-theoretic transform on the device.
 * All randomness (s ternary, a uniform, e/e0/e1 small, v ternary) is given by
 * the caller.  Polynomials are [.. ][N] arrays of coefficients; ciphertexts
 * are [batch][2][N] uint64 (c0 then c1).  Device pointers, asynchronous on
 * `stream`; errors as in paillier.h.  A context keeps one scratch area for its
 * calls: calls on one context run on one stream (or one at a time); use one
 * context per stream for concurrent work.
 */
#ifndef PAILLIER_B300_CKKS_H
#define PAILLIER_B300_CKKS_H

#include <stddef.h>
#include <stdint.h>

#include "paillier.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ckks_ctx ckks_ctx;

/* N = 2^log_n (log_n in 4..13), q an odd prime < 2^62 with q = 1 mod 2N
 * (checked), scale > 0.  Allocates the transform and embedding tables on the
 * current device. */
pl_status ckks_create(int log_n, uint64_t q, double scale, ckks_ctx** out);
void ckks_free(ckks_ctx* ctx);

/* Launch shape (results are identical either way): a call on at most
 * max_batch polynomials spreads each polynomial over a cluster of 8 CTAs that
 * exchange data through distributed shared memory (for N >= 1024); a larger
 * call keeps one polynomial per CTA.  Default 64; 0 never uses clusters. */
pl_status ckks_set_cluster_limit(ckks_ctx* ctx, size_t max_batch);

/* Slots per polynomial (N/2). */
int ckks_slots(const ckks_ctx* ctx);

/* d_re, d_im [batch][N/2] (float64) -> d_m [batch][N] signed coefficients. */
pl_status ckks_encode(ckks_ctx* ctx, const double* d_re, const double* d_im, size_t batch, int64_t* d_m,
                      void* stream);

/* d_m [batch][N] in [0, q) (centred internally) -> d_re, d_im [batch][N/2]. */
pl_status ckks_decode(ckks_ctx* ctx, const uint64_t* d_m, size_t batch, double* d_re, double* d_im, void* stream);

/* Public key half b [N] = -a s + e mod q from s [N] (int8, |s| <= 1), a [N]
 * (< q) and e [N] (int32). */
pl_status ckks_keygen(ckks_ctx* ctx, const int8_t* d_s, const uint64_t* d_a, const int32_t* d_e, uint64_t* d_b,
                      void* stream);

/* Encrypts `batch` plaintexts d_m [batch][N] under (d_b, d_a) with
 * d_v [batch][N] (int8) and d_e0, d_e1 [batch][N] (int32) into
 * d_c [batch][2][N]. */
pl_status ckks_encrypt(ckks_ctx* ctx, const uint64_t* d_b, const uint64_t* d_a, const int64_t* d_m,
                       const int8_t* d_v, const int32_t* d_e0, const int32_t* d_e1, size_t batch, uint64_t* d_c,
                       void* stream);

/* d_out [batch][2][N] = sum over the `count` ciphertext arrays d_cts[k]
 * [batch][2][N] (the server's aggregation; d_cts is a host array of device
 * pointers). */
pl_status ckks_sum(ckks_ctx* ctx, const uint64_t* const* d_cts, int count, size_t batch, uint64_t* d_out,
                   void* stream);

/* d_m [batch][N] = c0 + c1 s mod q for ciphertexts d_c [batch][2][N]. */
pl_status ckks_decrypt(ckks_ctx* ctx, const uint64_t* d_c, const int8_t* d_s, size_t batch, uint64_t* d_m,
                       void* stream);

/* Prepared keys: a client's keys do not change between rounds, so their
 * transforms can be taken once.  ckks_prepare_public_key stores (b, a) and
 * ckks_prepare_secret_key stores s in the transform domain inside ctx (device
 * memory owned by ctx, replaced by the next call; the stored key is ready for
 * work later on the same stream).  ckks_encrypt_prepared and
 * ckks_decrypt_prepared then equal ckks_encrypt / ckks_decrypt with that key,
 * bit for bit; they return PL_EINVAL if no key was prepared. */
pl_status ckks_prepare_public_key(ckks_ctx* ctx, const uint64_t* d_b, const uint64_t* d_a, void* stream);
pl_status ckks_prepare_secret_key(ckks_ctx* ctx, const int8_t* d_s, void* stream);
pl_status ckks_encrypt_prepared(ckks_ctx* ctx, const int64_t* d_m, const int8_t* d_v, const int32_t* d_e0,
                                const int32_t* d_e1, size_t batch, uint64_t* d_c, void* stream);
pl_status ckks_decrypt_prepared(ckks_ctx* ctx, const uint64_t* d_c, size_t batch, uint64_t* d_m, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PAILLIER_B300_CKKS_H */
