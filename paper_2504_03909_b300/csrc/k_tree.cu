// Tree building on decrypted histograms: XGBoost's exact histogram gain per
// (node, feature, bin), best split per node, next-level node membership.
#include <cuda_runtime.h>

#include "../../include/paillier_tree.h"
#include "internal.h"

namespace pl {
namespace {

constexpr int kSplitBlock = 128;

// exact decoded value of a fixed-point sum of `cnt` encoded values
__device__ __forceinline__ double fx(uint64_t s, long long cnt) {
  return __ddiv_rn((double)(long long)(s - ((unsigned long long)cnt << 24)), 16777216.0);
}

__device__ __forceinline__ double score(double G, double H, double lambda) {
  return __ddiv_rn(__dmul_rn(G, G), __dadd_rn(H, lambda));
}

// one block per node; thread t scans features t, t + blockDim, ... over bins
__global__ void __launch_bounds__(kSplitBlock) k_split_find(const uint64_t* __restrict__ sums,
                                                           const int32_t* __restrict__ counts, int F, int K,
                                                           double lambda, double gamma, double mcw,
                                                           int32_t* __restrict__ best_f, int32_t* __restrict__ best_b,
                                                           double* __restrict__ best_gain) {
  const int v = blockIdx.x;
  __shared__ double sg[kSplitBlock];
  __shared__ int sf[kSplitBlock], sb[kSplitBlock];
  double bg = 0.0;
  int bf = -1, bb = -1;
  for (int f = threadIdx.x; f < F; f += blockDim.x) {
    const uint64_t* s = sums + (((size_t)v * F + f) * K) * 2;
    const int32_t* c = counts + ((size_t)v * F + f) * K;
    uint64_t Sg = 0, Sh = 0;
    long long C = 0;
    for (int b = 0; b < K; ++b) { Sg += s[2 * b]; Sh += s[2 * b + 1]; C += c[b]; }
    const double G = fx(Sg, C), H = fx(Sh, C);
    const double parent = score(G, H, lambda);
    uint64_t Lg = 0, Lh = 0;
    long long Lc = 0;
    for (int b = 0; b + 1 < K; ++b) {
      Lg += s[2 * b];
      Lh += s[2 * b + 1];
      Lc += c[b];
      const double GL = fx(Lg, Lc), HL = fx(Lh, Lc);
      const double GR = fx(Sg - Lg, C - Lc), HR = fx(Sh - Lh, C - Lc);
      if (!(HL >= mcw && HR >= mcw)) continue;
      const double gain =
          __dsub_rn(__dmul_rn(0.5, __dsub_rn(__dadd_rn(score(GL, HL, lambda), score(GR, HR, lambda)), parent)), gamma);
      if (gain > bg) { bg = gain; bf = f; bb = b; }  // first maximum in (f, b) order per thread
    }
  }
  sg[threadIdx.x] = bg;
  sf[threadIdx.x] = bf;
  sb[threadIdx.x] = bb;
  __syncthreads();
  if (threadIdx.x == 0) {
    // features were dealt round-robin: visit them in feature order, keep the first maximum
    double g = 0.0;
    int f0 = -1, b0 = -1;
    for (int t = 0; t < (int)blockDim.x && t < F; ++t) {
      if (sf[t] < 0) continue;
      if (sg[t] > g || (sg[t] == g && f0 >= 0 && sf[t] < f0)) { g = sg[t]; f0 = sf[t]; b0 = sb[t]; }
    }
    best_f[v] = f0;
    best_b[v] = b0;
    if (best_gain) best_gain[v] = f0 >= 0 ? g : 0.0;
  }
}

__global__ void k_split_apply(const uint8_t* __restrict__ bins, size_t M, const int32_t* __restrict__ node,
                              const int32_t* __restrict__ best_f, const int32_t* __restrict__ best_b,
                              int32_t* __restrict__ next) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
    const int v = node[i];
    int out = -1;
    if (v >= 0) {
      const int f = best_f[v];
      if (f >= 0) out = 2 * v + (bins[(size_t)f * M + i] > (uint8_t)best_b[v] ? 1 : 0);
    }
    next[i] = out;
  }
}

}  // namespace
}  // namespace pl

extern "C" {

pl_status paillier_split_find(const uint64_t* d_sums, const int32_t* d_counts, int nodes, int F, int K, double lambda,
                              double gamma, double min_child_weight, int32_t* d_best_f, int32_t* d_best_b,
                              double* d_best_gain, void* stream) {
  using namespace pl;
  clear_error();
  if (nodes < 1 || F < 1 || K < 2 || K > 256) return fail(PL_EINVAL, "need nodes >= 1, F >= 1, 2 <= K <= 256");
  if (!d_sums || !d_counts || !d_best_f || !d_best_b) return fail(PL_EINVAL, "NULL buffer");
  if (!(lambda >= 0) || !(min_child_weight >= 0)) return fail(PL_EINVAL, "lambda and min_child_weight must be >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_split_find<<<nodes, kSplitBlock, 0, s>>>(d_sums, d_counts, F, K, lambda, gamma, min_child_weight, d_best_f,
                                             d_best_b, d_best_gain);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

pl_status paillier_split_apply(const uint8_t* d_bins, size_t M, const int32_t* d_node, const int32_t* d_best_f,
                               const int32_t* d_best_b, int32_t* d_next, void* stream) {
  using namespace pl;
  clear_error();
  if (M == 0) return PL_OK;
  if (!d_bins || !d_node || !d_best_f || !d_best_b || !d_next) return fail(PL_EINVAL, "NULL buffer");
  const int grid = (int)std::min<size_t>((M + 255) / 256, (size_t)sm_count() * 8);
  k_split_apply<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_bins, M, d_node, d_best_f, d_best_b, d_next);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

}  // extern "C"
