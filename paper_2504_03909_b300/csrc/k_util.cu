// Small utility kernels: seeded random limbs for the autotuner's timing inputs.
#include <cuda_runtime.h>

#include "internal.h"

namespace pl {
namespace {

__device__ __forceinline__ uint64_t splitmix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// rows x row_limbs random words; with zero_top the last limb of every row is 0
// (so the value is below any modulus of row_limbs limbs with a non-zero top limb)
__global__ void k_fill_random(uint32_t* p, size_t rows, int row_limbs, int zero_top, uint64_t seed) {
  const size_t n = rows * (size_t)row_limbs;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const bool top = (int)(i % row_limbs) == row_limbs - 1;
    p[i] = (zero_top && top) ? 0u : (uint32_t)splitmix(seed ^ (i * 0x2545F4914F6CDD1Dull));
  }
}

}  // namespace

pl_status launch_fill_random(uint32_t* p, size_t rows, int row_limbs, int zero_top, uint64_t seed, cudaStream_t s) {
  const size_t n = rows * (size_t)row_limbs;
  if (!n) return PL_OK;
  const int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)sm_count() * 16);
  k_fill_random<<<grid, 256, 0, s>>>(p, rows, row_limbs, zero_top, seed);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

}  // namespace pl
