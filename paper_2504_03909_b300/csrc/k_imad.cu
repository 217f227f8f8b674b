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
//          instruction per limb product, counted as 2).
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

__global__ void __launch_bounds__(256) k_imad_wide(uint32_t* out, int iters, uint32_t seed) {
  uint64_t x[8];
  uint32_t a = seed ^ threadIdx.x, b = seed * 3 + 1;
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = seed + j * 77 + threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(x[j]) : "r"(a), "r"(b + j));
    a ^= (uint32_t)x[0];
  }
  uint64_t y = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) y ^= x[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (uint32_t)(y ^ (y >> 32));
}

constexpr int kRowS = 16;
// IMAD per iteration and thread: 2 rows x 2 S multiply-add halves + 2 mul.lo
constexpr double kRowsImadPerIter = 2.0 * 2 * kRowS + 2;
constexpr double kWideImadPerIter = 2.0 * 32;  // 32 mad.wide, 2 IMAD each

}  // namespace
}  // namespace pl

extern "C" pl_status paillier_imad_peak(int mix, double target_ms, double* imad_per_s, double* elapsed_ms,
                                        void* stream) {
  using namespace pl;
  clear_error();
  if (!imad_per_s || (mix != 0 && mix != 1) || !(target_ms > 0)) return fail(PL_EINVAL, "bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = sm_count() * 8, threads = 256;
  uint32_t* out = nullptr;
  PL_CUDA_TRY(cudaMalloc(&out, sizeof(uint32_t) * (size_t)blocks * threads));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&](int iters, uint32_t seed) {
    if (mix == 0)
      k_imad_rows<kRowS><<<blocks, threads, 0, s>>>(out, iters, seed);
    else
      k_imad_wide<<<blocks, threads, 0, s>>>(out, iters, seed);
  };
  // calibrate
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
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "imad peak kernel");
  const double per = mix == 0 ? kRowsImadPerIter : kWideImadPerIter;
  *imad_per_s = per * iters * (double)blocks * threads / (ms * 1e-3);
  if (elapsed_ms) *elapsed_ms = ms;
  return PL_OK;
}
