/*
 * paillier_testing.h -- entry points that expose the library's multi-precision
 * core on its own, so that tests can check it limb for limb against plain
 * integer arithmetic.  The paper has no counterpart: they exist for testing.
 */
#ifndef PAILLIER_B300_TESTING_H
#define PAILLIER_B300_TESTING_H

#include <stddef.h>
#include <stdint.h>

#include "paillier.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Montgomery product of the warp-cooperative kernel core:
 *   d_out[i] = d_a[i] * d_b[i] * 2^(-32 limbs) mod N     (canonical)
 * for `count` pairs; d_a, d_b, d_out are [count][limbs] uint32 on the device,
 * h_N is the odd modulus (host, `limbs` limbs, top limb non-zero).
 * Requires d_a[i] * d_b[i] < N * 2^(32 limbs) (e.g. both < N).
 * (limbs, lanes) must be one of the compiled pairs: (32,2) (32,4) (64,2)
 * (64,4) (64,8) (96,4) (96,8) (128,4) (128,8) (192,8) (192,16). */
int paillier_test_mont_mul(int limbs, int lanes, const uint32_t* h_N, const uint32_t* d_a,
                           const uint32_t* d_b, size_t count, uint32_t* d_out, void* stream);

/* The separated-form (SOS) Montgomery product of the exponentiation kernels,
 * one code body for products and squarings (a square forms every cross
 * product once):
 *   d_out[i] = d_a[i] * d_b[i] * 2^(-32 limbs) mod N      (d_b non-NULL)
 *   d_out[i] = d_a[i]^2 * 2^(-32 limbs) mod N             (d_b NULL)
 * canonical, for `count` values d_a[i], d_b[i] < N; d_a, d_b, d_out are
 * [count][limbs] uint32 on the device (d_out may be d_a), h_N is the odd
 * modulus (host, `limbs` limbs, top limb non-zero).  (limbs, lanes) must be
 * one of (32,2) (32,4) (64,4) (64,8) (96,4) (96,8) (a multiple of 4 limbs per
 * lane, at most 24); others return PL_EINVAL.  Asynchronous on `stream`. */
int paillier_test_mont_sos(int limbs, int lanes, const uint32_t* h_N, const uint32_t* d_a, const uint32_t* d_b,
                           size_t count, uint32_t* d_out, void* stream);

/* Lengths of the key's key-fixed exponentiation schedules (host only, no
 * device work), for the CRT halves h = 0 (prime p) and 1 (prime q): nop[h] is
 * the number of ops of the exponentiation mod x^2 (exponent x for encryption,
 * x - 1 for decryption; x the half's prime), nop1[h] (encryption only, may be
 * NULL; 0 for decryption) that of the first encryption stage mod x (exponent
 * x' mod (x - 1), x' the other prime).  The first op loads the leading window
 * from the table of odd powers, every other op is one Montgomery product (a
 * squaring or a product by a table entry).  key must be private; w in 2..7. */
int paillier_test_schedule_ops(const pl_key* key, int dec, int w, int* nop, int* nop1);

/* Checked builds only (build.py --checked): launches one thread that reports
 * a failed bounds check at `site` (0..30) without touching any memory, so
 * that a test can see the report travel to paillier_sync (PL_EDEVICE, the
 * word then cleared).  Returns PL_EINVAL (1) in the normal build. */
int paillier_test_bounds_report(int site, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PAILLIER_B300_TESTING_H */
