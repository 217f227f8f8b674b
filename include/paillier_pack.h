/*
 * paillier_pack.h -- fewer decryptions for the same histogram.
 *
 * The paper counts encryptions and ciphertext additions (Sec. III.C) but not
 * decryptions, which at deep levels cost as much as the encryptions (every
 * cell of every node of a level is decrypted).  Packing, done by the passive
 * party with the public key, folds `slots` cells into one ciphertext by
 * Horner's rule on the plaintexts:
 *     packed = (...((c_{s-1})^(2^B) c_{s-2})^(2^B) ... )^(2^B) c_0   mod n^2
 * which encrypts sum_j m_j 2^(B j): one decryption then yields `slots` sums of
 * B bits each.  It is exact as long as every cell's plaintext is below 2^B
 * (histogram sums of fixed-point values are: M samples of at most 2^25 each
 * need B >= 25 + log2(M)); slots = floor((n_bits - 2) / B) keeps the packed
 * plaintext below n.  Cost per cell: B squarings and two products mod n^2
 * plus 1/slots of a decryption, against one full decryption.
 */
#ifndef PAILLIER_B300_PACK_H
#define PAILLIER_B300_PACK_H

#include <stddef.h>
#include <stdint.h>

#include "paillier.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Cells per packed ciphertext for a key and a slot width B (1 <= B <= 128;
 * widths above 64 serve g/h-packed cells, below). */
int paillier_pack_slots(const pl_key* key, int slot_bits);

/* Packs d_ct [count][2L] (canonical ciphertexts, e.g. histogram cells) into
 * d_packed [ceil(count / slots)][2L]; packed ciphertext i holds cells
 * i*slots .. i*slots + slots - 1 (slot 0 = lowest bits).  Public key enough. */
pl_status paillier_pack(const pl_key* key, const uint32_t* d_ct, size_t count, int slot_bits, uint32_t* d_packed,
                        void* stream);

/* Decrypts packed ciphertexts and writes the `count` original plaintexts as
 * uint64: d_m[i] = slot (i mod slots) of packed ciphertext i / slots
 * (slot_bits <= 64).  Needs the private key; uses the key's scratch like
 * paillier_decrypt. */
pl_status paillier_decrypt_packed_u64(const pl_key* key, const uint32_t* d_packed, size_t count, int slot_bits,
                                      uint64_t* d_m, void* stream);

/* The same two calls with fewer cells per packed ciphertext: `slots` in
 * 1 .. paillier_pack_slots(key, slot_bits), 0 = the most that fit (what the
 * calls above use); pack and decrypt must be given the same value.  Each
 * packed ciphertext is one chain of (slots - 1) (B + 1) products mod n^2 run
 * one after another, so when there are too few packed ciphertexts to fill the
 * GPU, the chain's length sets the packing time; fewer slots shorten it at
 * the cost of ceil(count / slots) decryptions instead of
 * ceil(count / most).  The sums do not depend on it.  PL_EINVAL for slots
 * outside that range. */
pl_status paillier_pack_n(const pl_key* key, const uint32_t* d_ct, size_t count, int slot_bits, int slots,
                          uint32_t* d_packed, void* stream);
pl_status paillier_decrypt_packed_u64_n(const pl_key* key, const uint32_t* d_packed, size_t count, int slot_bits,
                                        int slots, uint64_t* d_m, void* stream);

/* ---- g/h packing: one plaintext per sample ----------------------------------
 * Sec. III.C has one encryption per g and per h (M x 2) because Paillier
 * encrypts a single number.  A Paillier plaintext has n_bits, so both fit:
 *     m = enc(g) + 2^B enc(h),   enc(v) = rint(v 2^24) + 2^24 (as paillier_encode)
 * and a histogram cell's product decrypts to S_g + 2^B S_h, which splits into
 * the two sums when S_g < 2^B and S_h < 2^B (M samples of at most 2^25 each
 * need B >= 25 + log2(M)).  One encryption, one product per (sample, feature)
 * and one decryption per cell then serve g and h: half of each.  26 <= B <= 64
 * (the paper has no counterpart; a decrypt-count reduction like the above).
 * Out-of-range inputs follow paillier_encode; enc(g) >= 2^B sets PL_ERANGE in
 * the device status word.
 *
 * d_m [count][2] uint64: m's low and high 64-bit words. */
pl_status paillier_encode_gh(const float* d_g, const float* d_h, size_t count, int B, uint64_t* d_m, void* stream);

/* As paillier_encrypt, with plaintexts of two 64-bit words (d_m [count][2],
 * e.g. from paillier_encode_gh) -> d_ct [count][2L]. */
pl_status paillier_encrypt_gh(const pl_key* key, const uint64_t* d_m, const uint32_t* d_r, size_t count,
                              uint32_t* d_ct, void* stream);

/* As paillier_hist_aggregate over ONE Montgomery-form ciphertext array
 * d_ctm [M][2L] (g/h packed): d_hist [num_nodes][F][K][2L], d_count
 * [num_nodes][F][K] (may be NULL). */
pl_status paillier_hist_aggregate_gh(const pl_key* key, const uint32_t* d_ctm, size_t M, const uint8_t* d_bins,
                                     int F, int K, const int32_t* d_node, int num_nodes, uint32_t* d_hist,
                                     int32_t* d_count, void* stream);

/* Decrypts g/h-packed cells d_ct [count][2L] into d_sums [count][2] uint64
 * (S_g, S_h), the layout paillier_decrypt_u64 gives for separate g and h
 * cells.  A plaintext with bits at or above 2B sets PL_ERANGE in the device
 * status word. */
pl_status paillier_decrypt_gh(const pl_key* key, const uint32_t* d_ct, size_t count, int B, uint64_t* d_sums,
                              void* stream);

/* The two packings together: cells packed by paillier_pack with slot_bits =
 * 2B (slots = paillier_pack_slots(key, 2B) cells per ciphertext); d_packed
 * holds ceil(cells / slots) ciphertexts; d_sums [cells][2] as above. */
pl_status paillier_decrypt_packed_gh(const pl_key* key, const uint32_t* d_packed, size_t cells, int B,
                                     uint64_t* d_sums, void* stream);

/* As paillier_decrypt_packed_gh for cells packed by paillier_pack_n with
 * slot_bits = 2B and the same `slots` (0 = the most that fit). */
pl_status paillier_decrypt_packed_gh_n(const pl_key* key, const uint32_t* d_packed, size_t cells, int B, int slots,
                                       uint64_t* d_sums, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PAILLIER_B300_PACK_H */
