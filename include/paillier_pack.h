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

/* Cells per packed ciphertext for a key and a slot width B (1 <= B <= 64). */
int paillier_pack_slots(const pl_key* key, int slot_bits);

/* Packs d_ct [count][2L] (canonical ciphertexts, e.g. histogram cells) into
 * d_packed [ceil(count / slots)][2L]; packed ciphertext i holds cells
 * i*slots .. i*slots + slots - 1 (slot 0 = lowest bits).  Public key enough. */
pl_status paillier_pack(const pl_key* key, const uint32_t* d_ct, size_t count, int slot_bits, uint32_t* d_packed,
                        void* stream);

/* Decrypts packed ciphertexts and writes the `count` original plaintexts as
 * uint64: d_m[i] = slot (i mod slots) of packed ciphertext i / slots.
 * Needs the private key; uses the key's scratch like paillier_decrypt. */
pl_status paillier_decrypt_packed_u64(const pl_key* key, const uint32_t* d_packed, size_t count, int slot_bits,
                                      uint64_t* d_m, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PAILLIER_B300_PACK_H */
