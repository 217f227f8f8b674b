// Integer multiply-add peak of the GPU, measured with the instruction mixes
// the Montgomery kernels use.  The roofline of every kernel here is this
// measured rate (the work is bit-exact integer arithmetic: no tensor cores).
//
// Unit: one "IMAD" is one 32-bit multiply-add half of a 32x32 -> 64-bit limb
// product (mad.lo or mad.hi), so a limb product counts as 2.
//   mix 0 "carry rows": rows t[0..15] += a[0..15] * b as even/odd PTX carry
//          chains (mad.lo.cc / madc.hi.cc), plus one mul.lo per row pair --
//          the exact pattern of the CIOS rows;
//   mix 1 "wide": mad.wide.u32 into independent 64-bit accumulators (one
//          instruction per limb product, counted as 2);
//   mix 2 "lo/hi": independent mad.lo and mad.hi halves, no carries.
// Every product has distinct operands, so the compiler cannot fold them.
#include <cuda_runtime.h>

#include "../../include/paillier_bench.h"
#include "internal.h"
#include "mp.cuh"

namespace pl {
namespace {

template <int S>
__global__ void __launch_bounds__(256) k_imad_rows(uint32_t* out, int iters, uint32_t seed) {
  uint32_t t[S], a[S], x1 = 0, x2 = 0;
#pragma unroll
  for (int j = 0; j < S; ++j) { a[j] = seed * (j + 7) + threadIdx.x; t[j] = a[j] ^ 0x9e3779b9u; }
  uint32_t b = seed ^ threadIdx.x;
  for (int it = 0; it < iters; ++it) {
    row<S, 0>(t, x1, x2, a, b);
    b = t[0] * 0x01000193u;
    row<S, 0>(t, x1, x2, a, b);
    b = t[1] * 0x01000193u;
  }
  uint32_t x = x1 ^ x2;
#pragma unroll
  for (int j = 0; j < S; ++j) x ^= t[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x;
}

// 16 independent 64-bit accumulators += a_j * b with distinct a_j (every
// product is a different pair of operands, so nothing can be folded).
__global__ void __launch_bounds__(256) k_imad_wide(uint32_t* out, int iters, uint32_t seed) {
  uint64_t acc[16];
  uint32_t a[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) { a[j] = seed * (j + 7) + threadIdx.x; acc[j] = a[j]; }
  uint32_t b = seed ^ threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 16; ++j) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc[j]) : "r"(a[j]), "r"(b));
    b = (uint32_t)acc[it & 15] * 0x01000193u + it;
  }
  uint64_t y = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) y ^= acc[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (uint32_t)(y ^ (y >> 32));
}

// 16 independent lo and hi halves (mad.lo / mad.hi, no carries)
__global__ void __launch_bounds__(256) k_imad_lohi(uint32_t* out, int iters, uint32_t seed) {
  uint32_t lo[16], hi[16], a[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) { a[j] = seed * (j + 7) + threadIdx.x; lo[j] = a[j]; hi[j] = ~a[j]; }
  uint32_t b = seed ^ threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      asm volatile("mad.lo.u32 %0, %1, %2, %0;" : "+r"(lo[j]) : "r"(a[j]), "r"(b));
      asm volatile("mad.hi.u32 %0, %1, %2, %0;" : "+r"(hi[j]) : "r"(a[j]), "r"(b));
    }
    b = lo[it & 15] * 0x01000193u + it;
  }
  uint32_t y = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) y ^= lo[j] ^ hi[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = y;
}

// 16 independent float64 FMA chains (fma.rn.f64) with distinct operands
__global__ void __launch_bounds__(256) k_dfma(double* out, int iters, uint32_t seed) {
  double acc[16], a[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) { a[j] = 1.0 + 1e-9 * (seed * (j + 7) + threadIdx.x); acc[j] = a[j] * 1e-3; }
  double b = 0.999999 - 1e-12 * (seed ^ threadIdx.x);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 16; ++j) asm volatile("fma.rn.f64 %0, %1, %2, %0;" : "+d"(acc[j]) : "d"(a[j]), "d"(b));
    b = 0.999999 - 1e-18 * acc[it & 15];
  }
  double y = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) y += acc[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = y;
}

constexpr int kRowS = 16;
// IMAD per iteration and thread: 2 rows x 2 S multiply-add halves + 2 mul.lo
constexpr double kRowsImadPerIter = 2.0 * 2 * kRowS + 2;
constexpr double kWideImadPerIter = 2.0 * 16;  // 16 mad.wide (+1 mul.lo ignored), 2 IMAD each
constexpr double kLoHiImadPerIter = 2.0 * 16;  // 16 mad.lo + 16 mad.hi
constexpr double kDfmaFlopPerIter = 2.0 * 16;  // 16 fma.rn.f64 (+1 fma ignored), 2 FLOP each

// Runs launch(iters, seed) once to calibrate, then for about target_ms;
// returns the timed iterations and milliseconds.
template <typename F>
cudaError_t timed_probe(F launch, double target_ms, cudaStream_t s, int* iters_out, float* ms_out) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int iters = 2000;
  float ms = 0.f;
  launch(iters, 1);
  cudaEventRecord(e0, s);
  launch(iters, 2);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) {
    cudaEventElapsedTime(&ms, e0, e1);
    const double scale = target_ms / (ms > 0.01f ? ms : 0.01f);
    iters = (int)std::min(2.0e9, std::max(2000.0, iters * scale));
    cudaEventRecord(e0, s);
    launch(iters, 3);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *iters_out = iters;
  *ms_out = ms;
  return e;
}

}  // namespace
}  // namespace pl

extern "C" pl_status paillier_imad_peak(int mix, double target_ms, double* imad_per_s, double* elapsed_ms,
                                        void* stream) {
  using namespace pl;
  clear_error();
  if (!imad_per_s || mix < 0 || mix > 2 || !(target_ms > 0)) return fail(PL_EINVAL, "bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = sm_count() * 8, threads = 256;
  uint32_t* out = nullptr;
  PL_CUDA_TRY(cudaMalloc(&out, sizeof(uint32_t) * (size_t)blocks * threads));
  auto launch = [&](int iters, uint32_t seed) {
    if (mix == 0)
      k_imad_rows<kRowS><<<blocks, threads, 0, s>>>(out, iters, seed);
    else if (mix == 1)
      k_imad_wide<<<blocks, threads, 0, s>>>(out, iters, seed);
    else
      k_imad_lohi<<<blocks, threads, 0, s>>>(out, iters, seed);
  };
  int iters = 0;
  float ms = 0.f;
  const cudaError_t e = timed_probe(launch, target_ms, s, &iters, &ms);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "imad peak kernel");
  const double per = mix == 0 ? kRowsImadPerIter : (mix == 1 ? kWideImadPerIter : kLoHiImadPerIter);
  *imad_per_s = per * iters * (double)blocks * threads / (ms * 1e-3);
  if (elapsed_ms) *elapsed_ms = ms;
  return PL_OK;
}

extern "C" pl_status paillier_fp64_peak(double target_ms, double* flop_per_s, double* elapsed_ms, void* stream) {
  using namespace pl;
  clear_error();
  if (!flop_per_s || !(target_ms > 0)) return fail(PL_EINVAL, "bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = sm_count() * 8, threads = 256;
  double* out = nullptr;
  PL_CUDA_TRY(cudaMalloc(&out, sizeof(double) * (size_t)blocks * threads));
  auto launch = [&](int iters, uint32_t seed) { k_dfma<<<blocks, threads, 0, s>>>(out, iters, seed); };
  int iters = 0;
  float ms = 0.f;
  const cudaError_t e = timed_probe(launch, target_ms, s, &iters, &ms);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "fp64 peak kernel");
  *flop_per_s = kDfmaFlopPerIter * iters * (double)blocks * threads / (ms * 1e-3);
  if (elapsed_ms) *elapsed_ms = ms;
  return PL_OK;
}
