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
                              int nodes, int F, const int32_t* __restrict__ best_f,
                              const int32_t* __restrict__ best_b, int32_t* __restrict__ next, int* status) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
    const int v = node[i];
    int out = -1;
    if (v >= nodes) {
      atomicOr(status, kStatusBadNode);
    } else if (v >= 0) {
      const int f = best_f[v];
      if (f >= F) {
        atomicOr(status, kStatusBadSplit);
      } else if (f >= 0) {
        out = 2 * v + (bins[(size_t)f * M + i] > (uint8_t)best_b[v] ? 1 : 0);
      }
    }
    next[i] = out;
  }
}

// per parent: which child is smaller (counts of the split feature's bins)
__global__ void k_child_sizes(const int32_t* __restrict__ counts, int nodes, int F, int K,
                              const int32_t* __restrict__ best_f, const int32_t* __restrict__ best_b,
                              int32_t* __restrict__ small_right, int* status) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nodes) return;
  const int f = best_f[v];
  if (f >= F) atomicOr(status, kStatusBadSplit);
  if (f < 0 || f >= F) { small_right[v] = 0; return; }
  const int32_t* c = counts + ((size_t)v * F + f) * K;
  long long left = 0, right = 0;
  for (int b = 0; b < K; ++b) (b <= best_b[v] ? left : right) += c[b];
  small_right[v] = right < left ? 1 : 0;
}

__global__ void k_child_select(const int32_t* __restrict__ next, size_t M, const int32_t* __restrict__ small_right,
                               int nodes, int32_t* __restrict__ small_node, int* status) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
    const int c = next[i];
    if (c >= 2 * nodes) atomicOr(status, kStatusBadNode);
    const bool in = c >= 0 && c < 2 * nodes;
    small_node[i] = (in && (c & 1) == small_right[c >> 1]) ? (c >> 1) : -1;
  }
}

__global__ void k_child_subtract(const uint64_t* __restrict__ ps, const int32_t* __restrict__ pc,
                                 const uint64_t* __restrict__ ss, const int32_t* __restrict__ sc,
                                 const int32_t* __restrict__ small_right, int nodes, size_t per_node,
                                 uint64_t* __restrict__ cs, int32_t* __restrict__ cc) {
  // per_node = F * K cells; every cell has a g and an h sum and one count
  const size_t total = (size_t)nodes * per_node;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t v = i / per_node, cell = i % per_node;
    const int sr = small_right[v] != 0 ? 1 : 0;
    const size_t small_child = 2 * v + sr, big_child = 2 * v + (1 - sr);
    for (int k = 0; k < 2; ++k) {
      const uint64_t s = ss[i * 2 + k];
      cs[(small_child * per_node + cell) * 2 + k] = s;
      cs[(big_child * per_node + cell) * 2 + k] = ps[i * 2 + k] - s;
    }
    cc[small_child * per_node + cell] = sc[i];
    cc[big_child * per_node + cell] = pc[i] - sc[i];
  }
}

__global__ void k_tree_decide(const uint8_t* __restrict__ bins, int F_party, int f_lo, size_t M,
                              const int32_t* __restrict__ tf, const int32_t* __restrict__ tb, int nodes,
                              uint8_t* __restrict__ go_right) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
    for (int t = 0; t < nodes; ++t) {
      const int f = tf[t];
      if (f < f_lo || f >= f_lo + F_party) continue;
      go_right[(size_t)t * M + i] = bins[(size_t)(f - f_lo) * M + i] > (uint8_t)tb[t] ? 1 : 0;
    }
  }
}

__global__ void k_tree_route(const uint8_t* __restrict__ go_right, size_t M, const int32_t* __restrict__ tf,
                             int depth, int32_t* __restrict__ leaf) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
    int v = 0, first = 0;  // node v of level l has level-order index first + v, first = 2^l - 1
    for (int l = 0; l < depth; ++l) {
      const int t = first + v;
      if (tf[t] < 0 || l == depth - 1) break;
      v = 2 * v + (go_right[(size_t)t * M + i] != 0 ? 1 : 0);
      first = 2 * first + 1;
    }
    leaf[i] = first + v;
  }
}

__global__ void k_leaf_weights(const uint64_t* __restrict__ sums, const int32_t* __restrict__ counts, int nodes,
                               int F, int K, double lambda, double* __restrict__ w) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nodes) return;
  const uint64_t* s = sums + ((size_t)v * F) * K * 2;  // feature 0
  const int32_t* c = counts + ((size_t)v * F) * K;
  uint64_t Sg = 0, Sh = 0;
  long long C = 0;
  for (int b = 0; b < K; ++b) { Sg += s[2 * b]; Sh += s[2 * b + 1]; C += c[b]; }
  const double G = fx(Sg, C), H = fx(Sh, C);
  w[v] = -__ddiv_rn(G, __dadd_rn(H, lambda));
}

// the current device's status word (null without a usable device)
int* tree_status() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  return status_word(dev);
}

}  // namespace
}  // namespace pl

extern "C" {

pl_status paillier_tree_decide(const uint8_t* d_bins_party, int F_party, int f_lo, size_t M, const int32_t* d_tree_f,
                               const int32_t* d_tree_b, int nodes, uint8_t* d_go_right, void* stream) {
  using namespace pl;
  clear_error();
  if (F_party < 1 || f_lo < 0 || nodes < 1) return fail(PL_EINVAL, "bad sizes");
  if (M == 0) return PL_OK;
  if (!d_bins_party || !d_tree_f || !d_tree_b || !d_go_right) return fail(PL_EINVAL, "NULL buffer");
  const int grid = (int)std::min<size_t>((M + 255) / 256, (size_t)sm_count() * 8);
  k_tree_decide<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_bins_party, F_party, f_lo, M, d_tree_f,
                                                                      d_tree_b, nodes, d_go_right);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

pl_status paillier_tree_route(const uint8_t* d_go_right, size_t M, const int32_t* d_tree_f, int depth,
                              int32_t* d_leaf, void* stream) {
  using namespace pl;
  clear_error();
  if (depth < 1 || depth > 30) return fail(PL_EINVAL, "depth must be 1..30");
  if (M == 0) return PL_OK;
  if (!d_go_right || !d_tree_f || !d_leaf) return fail(PL_EINVAL, "NULL buffer");
  const int grid = (int)std::min<size_t>((M + 255) / 256, (size_t)sm_count() * 8);
  k_tree_route<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_go_right, M, d_tree_f, depth, d_leaf);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

pl_status paillier_leaf_weights(const uint64_t* d_sums, const int32_t* d_counts, int nodes, int F, int K,
                                double lambda, double* d_w, void* stream) {
  using namespace pl;
  clear_error();
  if (nodes < 1 || F < 1 || K < 1) return fail(PL_EINVAL, "bad sizes");
  if (!d_sums || !d_counts || !d_w) return fail(PL_EINVAL, "NULL buffer");
  k_leaf_weights<<<(nodes + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(d_sums, d_counts, nodes, F, K,
                                                                                     lambda, d_w);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

pl_status paillier_child_select(const int32_t* d_next, size_t M, const int32_t* d_counts, int nodes, int F, int K,
                                const int32_t* d_best_f, const int32_t* d_best_b, int32_t* d_small_right,
                                int32_t* d_small_node, void* stream) {
  using namespace pl;
  clear_error();
  if (nodes < 1 || F < 1 || K < 1 || K > 256) return fail(PL_EINVAL, "bad sizes");
  if (!d_next || !d_counts || !d_best_f || !d_best_b || !d_small_right || !d_small_node)
    return fail(PL_EINVAL, "NULL buffer");
  int* st = tree_status();
  if (!st) return fail(PL_ECUDA, "no usable CUDA device");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_child_sizes<<<(nodes + 127) / 128, 128, 0, s>>>(d_counts, nodes, F, K, d_best_f, d_best_b, d_small_right, st);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  if (M) {
    const int grid = (int)std::min<size_t>((M + 255) / 256, (size_t)sm_count() * 8);
    k_child_select<<<grid, 256, 0, s>>>(d_next, M, d_small_right, nodes, d_small_node, st);
    note_launch();
    PL_CUDA_TRY(cudaGetLastError());
  }
  return PL_OK;
}

pl_status paillier_child_subtract(const uint64_t* d_parent_sums, const int32_t* d_parent_counts,
                                  const uint64_t* d_small_sums, const int32_t* d_small_counts,
                                  const int32_t* d_small_right, int nodes, int F, int K, uint64_t* d_child_sums,
                                  int32_t* d_child_counts, void* stream) {
  using namespace pl;
  clear_error();
  if (nodes < 1 || F < 1 || K < 1) return fail(PL_EINVAL, "bad sizes");
  if (!d_parent_sums || !d_parent_counts || !d_small_sums || !d_small_counts || !d_small_right || !d_child_sums ||
      !d_child_counts)
    return fail(PL_EINVAL, "NULL buffer");
  const size_t per = (size_t)F * K, total = per * nodes;
  const int grid = (int)std::min<size_t>((total + 255) / 256, (size_t)sm_count() * 8);
  k_child_subtract<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      d_parent_sums, d_parent_counts, d_small_sums, d_small_counts, d_small_right, nodes, per, d_child_sums,
      d_child_counts);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

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

pl_status paillier_split_apply(const uint8_t* d_bins, size_t M, int F, const int32_t* d_node, int nodes,
                               const int32_t* d_best_f, const int32_t* d_best_b, int32_t* d_next, void* stream) {
  using namespace pl;
  clear_error();
  if (F < 1 || nodes < 1) return fail(PL_EINVAL, "need F >= 1 and nodes >= 1");
  if (M == 0) return PL_OK;
  if (!d_bins || !d_node || !d_best_f || !d_best_b || !d_next) return fail(PL_EINVAL, "NULL buffer");
  int* st = tree_status();
  if (!st) return fail(PL_ECUDA, "no usable CUDA device");
  const int grid = (int)std::min<size_t>((M + 255) / 256, (size_t)sm_count() * 8);
  k_split_apply<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_bins, M, d_node, nodes, F, d_best_f, d_best_b,
                                                                      d_next, st);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

}  // extern "C"
