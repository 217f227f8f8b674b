/*
 * paillier.h -- C ABI of the B300 Paillier hot path for vertical secure
 * federated XGBoost.
 *
 * The three steps of the vertical secure pattern (Sec. III.B of the paper):
 * the active party encrypts each sample's gradient g and hessian h; every
 * passive party multiplies the ciphertexts into the histogram slot
 * (tree node, feature, bin) each sample falls in; the active party decrypts
 * the returned histograms.  Sec. III.C gives the scheme (Paillier, cited) and
 * the per-round counts: M x 2 single-number encryptions and about
 * (M - K) x 2 x J ciphertext "additions" (modular multiplications).
 * Sec. III.D's processor interface takes "g/h pairs" in and hands a
 * "processed buffer" out; here that buffer is the canonical ciphertext array.
 *
 * Scheme (textbook Paillier, g = n + 1; the paper cites it without restating):
 *   encrypt(m, r) = (1 + m n) r^n mod n^2
 *   decrypt(c)    = CRT form: m_p = L_p(c^(p-1) mod p^2) h_p mod p, same for q,
 *                   m = m_q + q ((m_p - m_q) q^-1 mod p),  L_p(x) = (x - 1)/p.
 *
 * Conventions for every entry point:
 *   - Multi-precision values are little-endian arrays of uint32 limbs.  With
 *     n_bits the modulus size, L = n_bits / 32: a plaintext or r has L limbs,
 *     a ciphertext (mod n^2) has 2 L limbs, rows are contiguous (row-major).
 *   - Pointers named d_* are device pointers on the current CUDA device;
 *     h_* are host pointers.  The caller owns every buffer and every stream;
 *     the library never frees or reallocates them.  Device buffers must be
 *     16-byte aligned (cudaMalloc / torch allocations are).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *     Calls are asynchronous on it; argument checks are synchronous and
 *     return an error before anything is launched.
 *   - Scratch memory (window tables, sort indices, work lists, partial
 *     products) belongs to the key object: it is allocated on first use,
 *     grows when a larger call needs it, and is freed with the key.  Calls
 *     with the SAME key on different streams that overlap in time race on
 *     that scratch; use one key object per concurrent stream.
 *   - Errors that only the device can see (a bin >= K, a node >= num_nodes,
 *     a decrypted sum >= 2^64, a bounded wait that ran out) are recorded in a
 *     device status word and returned by paillier_sync().
 *   - On error the return value is non-zero and paillier_last_error() gives a
 *     message (thread-local, valid until the next call on the same thread).
 *   - Inputs must be canonical: 0 <= m < n, 1 <= r < n with gcd(r, n) = 1,
 *     ciphertexts in [1, n^2).  Outputs are canonical (fully reduced).
 *     Encryption checks the randomness on the device: an r with
 *     gcd(r, n) != 1 sets PL_EDEVICE in the status word.
 */
#ifndef PAILLIER_B300_H
#define PAILLIER_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int pl_status;
#define PL_OK        0
#define PL_EINVAL    1  /* bad argument (null pointer, size, unsupported n_bits) */
#define PL_ENOMEM    2  /* device or host allocation failed */
#define PL_ECUDA     3  /* a CUDA runtime call failed */
#define PL_ERANGE    4  /* a value is out of range (e.g. decrypted sum >= 2^64) */
#define PL_ETIMEDOUT 5  /* a bounded device wait ran out */
#define PL_EBUSY     6  /* admission refused (serving: no slot or HBM budget) */
#define PL_EDEVICE   7  /* a kernel reported bad input in the device status word */

/* Supported key sizes: n_bits in {1024, 2048, 3072}. */
typedef struct pl_key pl_key;

/* ---------------------------------------------------------------- keys -- */

/* Deterministic key generation (host only; the paper does not say how keys
 * are made): two distinct n_bits/2-bit primes with the top two bits set,
 * 64 Miller-Rabin rounds each, gcd(n, (p-1)(q-1)) = 1.  Same seed, same key.
 * *out is owned by the library until paillier_key_free(). */
pl_status paillier_keygen(int n_bits, uint64_t seed, pl_key** out);

/* Private key from its primes (host arrays of n_bits/64 limbs each).  The
 * primes are checked for size, top bits and p != q, not for primality. */
pl_status paillier_key_import(int n_bits, const uint32_t* h_p, const uint32_t* h_q, pl_key** out);

/* Public key from the modulus n (host array of n_bits/32 limbs): what a
 * passive party holds.  Only ct_prepare and the aggregation calls accept it. */
pl_status paillier_key_import_public(int n_bits, const uint32_t* h_n, pl_key** out);

/* Copies n (L limbs) and, for a private key, p and q (L/2 limbs each) to host
 * arrays; any output pointer may be NULL. */
pl_status paillier_key_export(const pl_key* key, uint32_t* h_n, uint32_t* h_p, uint32_t* h_q);

/* n_bits of the key (0 for NULL) and whether it holds p and q. */
int paillier_key_bits(const pl_key* key);
int paillier_key_is_private(const pl_key* key);

/* Frees the key and its scratch (synchronises the device first). */
void paillier_key_free(pl_key* key);

/* ------------------------------------------------------------ encode -- */

/* Fixed-point encoding (the paper fixes none; reading: scale 2^24, additive
 * offset 2^24, ties to even): d_m[i] = rint(d_v[i] * 2^24) + 2^24.
 * d_v[i] must lie in [-1, 2^15] (a logistic g lies in (-1, 1), h in
 * [0, 1/4]); other values write 0 and set PL_EDEVICE in the status word. */
pl_status paillier_encode(const float* d_v, size_t count, uint64_t* d_m, void* stream);

/* Decoding of histogram sums (Sec. III.B: the decrypted G/H go on to tree
 * building): d_out[i] = (d_s[i] - d_cnt[i] * 2^24) / 2^24 in float64, for
 * sums of d_cnt[i] >= 0 encoded values.  The difference is formed exactly in
 * 64-bit integers (valid while |d_s[i] - d_cnt[i] 2^24| < 2^63, which every
 * sum of at most 2^31 encoded values meets) and rounded once to float64,
 * nearest, ties to even; the scaling by 2^-24 is exact.  d_s, d_cnt, d_out:
 * [count] device arrays owned by the caller.  count = 0 does nothing. */
pl_status paillier_decode(const uint64_t* d_s, const int32_t* d_cnt, size_t count,
                          double* d_out, void* stream);

/* ----------------------------------------------------------- encrypt -- */

/* Encryption of `count` plaintexts (Sec. III.B/III.C: every g and every h is
 * one single-number encryption).  d_m: [count] uint64 plaintexts (< n);
 * d_r: [count][L] randomness (uniform in Z_n^*, given by the caller);
 * d_ct: [count][2L] ciphertexts out.  Needs the private key: r^n is computed
 * mod p^2 and mod q^2 and recombined (the key holder's CRT split).
 * An r with r mod p = 0 or r mod q = 0 (gcd(r, n) != 1, r = 0 included) sets
 * PL_EDEVICE in the status word; its row then holds a value that is not a
 * unit mod n^2, the other rows are unaffected.  An r in [n, 2^(32L)) gives
 * the encryption under r mod n, since r^n mod n^2 depends on r mod n only. */
pl_status paillier_encrypt(const pl_key* key, const uint64_t* d_m, const uint32_t* d_r,
                           size_t count, uint32_t* d_ct, void* stream);

/* ------------------------------------------------------- aggregation -- */

/* Montgomery form of ciphertexts for the passive party's histogram:
 * d_ctm[i] = d_ct[i] * 2^(64 L) mod n^2, [count][2L] each.  Done once per
 * received ciphertext array and reused by every level of a tree. */
pl_status paillier_ct_prepare(const pl_key* key, const uint32_t* d_ct, size_t count,
                              uint32_t* d_ctm, void* stream);

/* Encrypted histogram of one passive party (Sec. III.B: the encrypted
 * gradients are accumulated by feature bin; Sec. III.C: the "addition" of
 * Paillier ciphertexts is their product mod n^2).
 *   d_ctm  : [2][M][2L] Montgomery-form ciphertexts (row 0 = g, row 1 = h),
 *            from paillier_ct_prepare;
 *   d_bins : [F][M] uint8 bin of sample i in feature f (feature-major);
 *   d_node : [M] int32 tree node of sample i at this level, -1 = not in any
 *            node (its ciphertexts are skipped);
 *   d_hist : [num_nodes][F][K][2][2L] out: canonical product of the g (and h)
 *            ciphertexts of the cell's samples; an empty cell holds 1;
 *   d_count: [num_nodes][F][K] int32 out, the cell's sample count (may be NULL).
 * All nodes of the level are done in one pass (one set of launches).  K <= 256.
 * A bin >= K or a node >= num_nodes sets PL_EDEVICE in the status word and
 * the sample is skipped. */
pl_status paillier_hist_aggregate(const pl_key* key, const uint32_t* d_ctm, size_t M,
                                  const uint8_t* d_bins, int F, int K,
                                  const int32_t* d_node, int num_nodes,
                                  uint32_t* d_hist, int32_t* d_count, void* stream);

/* The same histogram computed the plain way: one set of launches per tree
 * node (each over the whole sample range with the other nodes masked out),
 * and one work item -- one lane group multiplying all the cell's ciphertexts
 * in sequence -- per cell.  The comparator of the batched level path, which
 * splits cells into fixed-size chunks and runs all nodes in one pass; results
 * are identical. */
pl_status paillier_hist_aggregate_per_node(const pl_key* key, const uint32_t* d_ctm, size_t M,
                                           const uint8_t* d_bins, int F, int K,
                                           const int32_t* d_node, int num_nodes,
                                           uint32_t* d_hist, int32_t* d_count, void* stream);

/* ----------------------------------------------------------- decrypt -- */

/* CRT decryption (Sec. III.B: the active party decrypts the returned
 * histograms) of `count` ciphertexts d_ct [count][2L] into d_m [count][L]. */
pl_status paillier_decrypt(const pl_key* key, const uint32_t* d_ct, size_t count,
                           uint32_t* d_m, void* stream);

/* As paillier_decrypt, narrowed to uint64 (histogram sums are < 2^64); a
 * plaintext >= 2^64 writes UINT64_MAX and sets PL_ERANGE in the status word. */
pl_status paillier_decrypt_u64(const pl_key* key, const uint32_t* d_ct, size_t count,
                               uint64_t* d_m, void* stream);

/* As paillier_decrypt_u64, for callers that cannot allocate device memory.
 * The paper has no counterpart; it exists because some callers may not call
 * cudaMalloc at all: a process whose device memory is owned by another
 * allocator (a framework's caching pool that has reserved the GPU), a
 * latency-critical loop where cudaMalloc's implicit device synchronisation is
 * not acceptable, or an embedding application that forbids allocation after
 * start-up.  This call allocates nothing: its scratch (the CRT half results
 * and the window tables) is one fixed device array inside the library, about
 * 21 MB, which every GPU that loads the library holds until the process exits.
 *   - count must be <= 8192 ciphertexts per call (else PL_EINVAL, nothing is
 *     launched); every supported key size is accepted.
 *   - The first call on a device looks up the array's device address on that
 *     device (the device must be current).  Make that first call before any
 *     stream capture.
 *   - All calls share the one array, which keeps the last call's contents;
 *     nothing in it needs to start at zero.  Calls whose kernels overlap on
 *     the GPU (different streams, or different host threads) race on it and
 *     give wrong results: serialise them.
 *   - A plaintext >= 2^64 is written as UINT64_MAX (the device status word of
 *     paillier_sync is not set by this call).
 *   - It uses a 4-bit window, so it is somewhat slower than
 *     paillier_decrypt_u64; results are identical. */
pl_status paillier_decrypt_u64_noalloc(const pl_key* key, const uint32_t* d_ct, size_t count, uint64_t* d_m,
                                       void* stream);

/* ------------------------------------------------------------ status -- */

/* Synchronises `stream`, then returns the first CUDA error or the device
 * status word (PL_EDEVICE / PL_ERANGE / PL_ETIMEDOUT), and clears the word.
 * *device_status (may be NULL) receives the raw word. */
pl_status paillier_sync(void* stream, int* device_status);

/* Message of the last error on this thread ("" if none). */
const char* paillier_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PAILLIER_B300_H */
