/*
 * paillier_bench.h -- measurement entry points.  The paper has no
 * counterpart: it reports end-to-end training times only (Sec. IV.B).
 */
#ifndef PAILLIER_B300_BENCH_H
#define PAILLIER_B300_BENCH_H

#include <stdint.h>

#include "paillier.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Integer multiply-add peak of the current GPU, measured for about
 * target_ms milliseconds on `stream` with one instruction mix:
 *   mix 0: 16-limb rows as even/odd PTX carry chains (mad.lo.cc/madc.hi.cc),
 *          the pattern of the Montgomery rows;
 *   mix 1: mad.wide.u32 into 64-bit accumulators;
 *   mix 2: independent mad.lo / mad.hi halves without carries.
 * Unit: IMAD/s, one IMAD being one 32-bit half (lo or hi) of a 32x32 -> 64
 * limb product.  *elapsed_ms (may be NULL) gets the timed duration.  The call
 * allocates and frees a small device buffer and synchronises the stream. */
pl_status paillier_imad_peak(int mix, double target_ms, double* imad_per_s, double* elapsed_ms, void* stream);

/* Float64 fused multiply-add peak of the current GPU (independent
 * fma.rn.f64 chains), measured like paillier_imad_peak.  Unit: FLOP/s, one
 * FMA being 2 FLOP.  The roofline of the CKKS embedding (FFT) kernels. */
pl_status paillier_fp64_peak(double target_ms, double* flop_per_s, double* elapsed_ms, void* stream);

/* Number of kernels the library has launched so far in this process. */
unsigned long long paillier_launch_count(void);

/* Per-kernel timing with CUDA events recorded around each launch on its own
 * stream (launches during stream capture are not timed).  paillier_profile(1)
 * clears the totals and starts timing; paillier_profile(0) stops it.
 * paillier_profile_read() waits for the recorded events and returns the
 * total milliseconds and launch count of one kernel name since the last
 * paillier_profile() call: "modexp_enc", "enc_crt", "modexp_dec", "dec_crt",
 * "to_mont", "hist_count", "hist_scan", "feat_scan", "hist_scatter",
 * "seg_product", "combine", "encode", "decode". */
pl_status paillier_profile(int enable);
pl_status paillier_profile_read(const char* kernel, double* total_ms, long long* launches);

#ifdef __cplusplus
}
#endif

#endif /* PAILLIER_B300_BENCH_H */
