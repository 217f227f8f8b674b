// Passive-party kernels: the encrypted histogram (Sec. III.B: the encrypted
// gradients are accumulated by feature bin; Sec. III.C: each "addition" of
// Paillier ciphertexts is a product mod n^2).
//
// Pipeline for one tree level (all nodes at once):
//   k_hist_count   counts per (feature, node*K + bin)
//   k_hist_scan    per-feature offsets, and the number of work items (chunks of
//                  at most `tile` samples) per cell
//   k_feat_scan    offsets of each feature's chunks in the global work list
//   k_hist_scatter sample ids grouped by cell (a counting sort)
//   k_seg_product  persistent: each group of T lanes multiplies the Montgomery
//                  ciphertexts of one chunk (product of up to `tile` values)
//   k_combine      per cell: product of its chunk partials, leave Montgomery
//                  form, write the canonical cell (1 when empty) and the count
// The product is commutative, so the order in which the scatter places equal
// keys does not change any output bit.
#include <cuda_runtime.h>

#include "check.cuh"
#include "internal.h"
#include "mp.cuh"

namespace pl {
namespace {

constexpr int kBlock = 128;
constexpr int kScanBlock = 1024;

// key of sample i in feature f, or -1 if skipped; only_node >= 0 restricts to
// that node (then the key is the bin alone)
__device__ __forceinline__ int hist_key(int v, int b, int K, int num_nodes, int only_node, int* status) {
  if (v < 0) return -1;
  if (v >= num_nodes) { atomicOr(status, kStatusBadNode); return -1; }
  if (b >= K) { atomicOr(status, kStatusBadBin); return -1; }
  if (only_node >= 0) return v == only_node ? b : -1;
  return v * K + b;
}

__global__ void k_set_desc(HistDesc* D, int num_nodes, int NK, int only_node) {
  D->num_nodes = num_nodes;
  D->NK = NK;
  D->only_node = only_node;
  D->pad = 0;
}

__global__ void k_hist_count(const uint8_t* __restrict__ bins, size_t bstride, const int32_t* __restrict__ node,
                             size_t M, int K, const HistDesc* __restrict__ D, int* __restrict__ cnt, int* status) {
  const int f = blockIdx.y;
  const int num_nodes = D->num_nodes, only_node = D->only_node, NK = D->NK;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
    const int key = hist_key(node[i], bins[(size_t)f * bstride + i], K, num_nodes, only_node, status);
    if (key >= 0) atomicAdd(&cnt[(size_t)f * NK + key], 1);
  }
}

__global__ void k_hist_scatter(const uint8_t* __restrict__ bins, size_t bstride, const int32_t* __restrict__ node,
                               size_t M, int K, const HistDesc* __restrict__ D, const int* __restrict__ off,
                               int* __restrict__ cursor, int* __restrict__ idx, int* status) {
  const int f = blockIdx.y;
  const int num_nodes = D->num_nodes, only_node = D->only_node, NK = D->NK;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
    const int key = hist_key(node[i], bins[(size_t)f * bstride + i], K, num_nodes, only_node, status);
    if (key >= 0) {
      const int pos = off[(size_t)f * (NK + 1) + key] + atomicAdd(&cursor[(size_t)f * NK + key], 1);
      if (PL_BOUNDS(pos >= 0 && (size_t)pos < M, kBoundsScatter)) idx[(size_t)f * M + pos] = (int)i;
    }
  }
}

// exclusive scan of (a, b) pairs over the block; returns the totals in *ta, *tb
__device__ void block_scan2(long long& a, long long& b, long long* ta, long long* tb) {
  __shared__ long long wa[32], wb[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long xa = __shfl_up_sync(kFull, ia, o), xb = __shfl_up_sync(kFull, ib, o);
    if (lane >= o) { ia += xa; ib += xb; }
  }
  if (lane == 31) { wa[wid] = ia; wb[wid] = ib; }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    long long va = lane < nw ? wa[lane] : 0, vb = lane < nw ? wb[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long xa = __shfl_up_sync(kFull, va, o), xb = __shfl_up_sync(kFull, vb, o);
      if (lane >= o) { va += xa; vb += xb; }
    }
    if (lane < nw) { wa[lane] = va; wb[lane] = vb; }
  }
  __syncthreads();
  const long long pa = wid ? wa[wid - 1] : 0, pb = wid ? wb[wid - 1] : 0;
  *ta = wa[(blockDim.x >> 5) - 1];
  *tb = wb[(blockDim.x >> 5) - 1];
  a = pa + ia - a;
  b = pb + ib - b;
  __syncthreads();
}

// one block per feature: off[f][0..NK] (sample offsets), choff[f][0..NK]
// (chunk offsets within the feature), featch[f] (chunks of the feature)
__global__ void __launch_bounds__(kScanBlock) k_hist_scan(const int* __restrict__ cnt,
                                                          const HistDesc* __restrict__ D, int tile,
                                                          int* __restrict__ off, int* __restrict__ choff,
                                                          int* __restrict__ featch) {
  const int f = blockIdx.x;
  const int NK = D->NK;
  const int* c = cnt + (size_t)f * NK;
  const int per = (NK + blockDim.x - 1) / blockDim.x;
  const int j0 = min(NK, (int)threadIdx.x * per), j1 = min(NK, j0 + per);
  long long s1 = 0, s2 = 0;
  for (int j = j0; j < j1; ++j) { s1 += c[j]; s2 += (c[j] + tile - 1) / tile; }
  long long t1, t2;
  block_scan2(s1, s2, &t1, &t2);
  int* o = off + (size_t)f * (NK + 1);
  int* co = choff + (size_t)f * (NK + 1);
  for (int j = j0; j < j1; ++j) {
    o[j] = (int)s1;
    co[j] = (int)s2;
    s1 += c[j];
    s2 += (c[j] + tile - 1) / tile;
  }
  if (threadIdx.x == 0) {
    o[NK] = (int)t1;
    co[NK] = (int)t2;
    featch[f] = (int)t2;
  }
}

// single block: featoff[0..F] = exclusive scan of featch; featoff[F] = total chunks
__global__ void __launch_bounds__(kScanBlock) k_feat_scan(const int* __restrict__ featch, int F,
                                                          int* __restrict__ featoff) {
  const int per = (F + blockDim.x - 1) / blockDim.x;
  const int j0 = min(F, (int)threadIdx.x * per), j1 = min(F, j0 + per);
  long long s = 0, z = 0;
  for (int j = j0; j < j1; ++j) s += featch[j];
  long long t, tz;
  block_scan2(s, z, &t, &tz);
  for (int j = j0; j < j1; ++j) { featoff[j] = (int)s; s += featch[j]; }
  if (threadIdx.x == 0) featoff[F] = (int)t;
}

// last index i in [0, n) with a[i] <= x (a non-decreasing, a[0] <= x)
__device__ __forceinline__ int last_le(const int* a, int n, int x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// x R mod n^2 for every ciphertext (R^2 staged once per block)
template <int S, int T>
__global__ void __launch_bounds__(kBlock) k_to_mont(const __grid_constant__ N2Const P, const uint32_t* __restrict__ ct,
                                                    size_t count, uint32_t* __restrict__ ctm) {
  constexpr int NL = S * T;
  constexpr int IPW = 32 / T;
  __shared__ uint32_t r2[NL];
  for (int j = threadIdx.x; j < NL; j += blockDim.x) r2[j] = P.R2[j];
  __syncthreads();
  const int lane = threadIdx.x & 31, k = lane % T, gw = lane / T;
  uint32_t n[S], a[S], t[S];
  const_slice<S>(n, P.N, k);
  const size_t nchunk = (count + IPW - 1) / IPW;
  const size_t warp0 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t c = warp0; c < nchunk; c += nwarps) {
    const size_t i = c * IPW + gw;
    const bool valid = i < count;
    const size_t ii = valid ? i : count - 1;
    load_slice<S>(a, ct + ii * NL, k);
    mont_mul<S, T>(t, a, r2, 1, n, P.np, k);
    if (valid) store_slice<S>(ctm + ii * NL, t, k);
  }
}

// Segmented product over the work list of chunks.  Item = (chunk, g/h): ngh
// ciphertext arrays (2: g and h; 1: g/h packed), item = chunk ngh + gh.
template <int S, int T>
__global__ void __launch_bounds__(kBlock) k_seg_product(const __grid_constant__ N2Const P,
                                                        const uint32_t* __restrict__ ctm, size_t M, size_t ghs, int ngh,
                                                        const int* __restrict__ idx, const int* __restrict__ off,
                                                        const int* __restrict__ choff,
                                                        const int* __restrict__ featoff, int F,
                                                        const HistDesc* __restrict__ D, int tile,
                                                        uint32_t* __restrict__ partial) {
  constexpr int NL = S * T;
  const int NK = D->NK;
  constexpr int IPW = 32 / T;
  extern __shared__ uint32_t smem[];
  const int ipb = blockDim.x / T;
  const int lane = threadIdx.x & 31, k = lane % T, gw = lane / T, g = threadIdx.x / T;
  uint32_t* bs = smem + g;
  const int st = ipb;
  uint32_t n[S], a[S], t[S];
  const_slice<S>(n, P.N, k);
  const uint32_t np = P.np;
  const long long total = (long long)ngh * featoff[F];
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp0 * IPW; base < total; base += nwarps * IPW) {
    const long long item = base + gw;
    const bool valid = item < total;
    int len = 0;
    const uint32_t* src = ctm;
    const int* ids = idx;
    if (valid) {
      const int c = (int)(ngh == 2 ? item >> 1 : item), gh = (int)(ngh == 2 ? item & 1 : 0);
      const int f = last_le(featoff, F, c);
      const int local = c - featoff[f];
      const int* co = choff + (size_t)f * (NK + 1);
      const int key = last_le(co, NK, local);
      const int* o = off + (size_t)f * (NK + 1);
      const int j0 = o[key] + (local - co[key]) * tile;
      len = min(tile, o[key + 1] - j0);
      src = ctm + (size_t)gh * ghs * NL;
      ids = idx + (size_t)f * M + j0;
    }
    const int maxlen = __reduce_max_sync(kFull, len);
    // a sample id outside [0, M) (checked builds) reads sample 0 instead
    auto sample = [&](int j) { const int id = ids[j]; return PL_BOUNDS(id >= 0 && (size_t)id < M, kBoundsSample) ? id : 0; };
    if (len > 0) load_slice<S>(a, src + (size_t)sample(0) * NL, k);
    for (int j = 1; j < maxlen; ++j) {
      const bool act = j < len;
      const unsigned mask = __ballot_sync(kFull, act);
      if (act) {
        load_slice<S>(t, src + (size_t)sample(j) * NL, k);
        __syncwarp(mask);
        stage<S>(bs, st, t, k);
        __syncwarp(mask);
        mont_mul<S, T>(t, a, bs, st, n, np, k, mask);
#pragma unroll
        for (int q = 0; q < S; ++q) a[q] = t[q];
      }
      __syncwarp();
    }
    if (valid && len > 0) store_slice<S>(partial + (size_t)item * NL, a, k);
  }
}

// Per cell and g/h: product of the chunk partials, out of Montgomery form.
template <int S, int T>
__global__ void __launch_bounds__(kBlock) k_combine(const __grid_constant__ N2Const P,
                                                    const uint32_t* __restrict__ partial,
                                                    const int* __restrict__ off, const int* __restrict__ choff,
                                                    const int* __restrict__ featoff, int F,
                                                    const HistDesc* __restrict__ D, int K, int ngh,
                                                    uint32_t* __restrict__ hist, int32_t* __restrict__ count_out) {
  constexpr int NL = S * T;
  const int NK = D->NK, only_node = D->only_node;
  constexpr int IPW = 32 / T;
  extern __shared__ uint32_t smem[];
  const int ipb = blockDim.x / T;
  const int lane = threadIdx.x & 31, k = lane % T, gw = lane / T, g = threadIdx.x / T;
  uint32_t* bs = smem + g;
  const int st = ipb;
  uint32_t n[S], a[S], t[S];
  const_slice<S>(n, P.N, k);
  const uint32_t np = P.np;
  const long long total = (long long)ngh * F * NK;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp0 * IPW; base < total; base += nwarps * IPW) {
    const long long item = base + gw;
    const bool valid = item < total;
    int nch = 0, first = 0, gh = 0, f = 0, key = 0;
    if (valid) {
      const long long cell = ngh == 2 ? item >> 1 : item;
      gh = (int)(ngh == 2 ? item & 1 : 0);
      f = (int)(cell / NK);
      key = (int)(cell % NK);
      const int* co = choff + (size_t)f * (NK + 1);
      nch = co[key + 1] - co[key];
      first = featoff[f] + co[key];
    }
    const int maxn = __reduce_max_sync(kFull, nch);
    // a chunk outside the work list (checked builds) reads chunk 0 instead
    auto chunk = [&](int j) { return PL_BOUNDS(first + j < featoff[F], kBoundsChunk) ? first + j : 0; };
    if (nch > 0) load_slice_rw<S>(a, partial + ((size_t)chunk(0) * ngh + gh) * NL, k);
    for (int j = 1; j < maxn; ++j) {
      const bool act = j < nch;
      const unsigned mask = __ballot_sync(kFull, act);
      if (act) {
        load_slice_rw<S>(t, partial + ((size_t)chunk(j) * ngh + gh) * NL, k);
        __syncwarp(mask);
        stage<S>(bs, st, t, k);
        __syncwarp(mask);
        mont_mul<S, T>(t, a, bs, st, n, np, k, mask);
#pragma unroll
        for (int q = 0; q < S; ++q) a[q] = t[q];
      }
      __syncwarp();
    }
    // leave Montgomery form (times 1); an empty cell is the ciphertext 1
    {
      const bool act = nch > 0;
      const unsigned mask = __ballot_sync(kFull, act);
      if (act) {
#pragma unroll
        for (int q = 0; q < S; ++q) bs[(k * S + q) * st] = (k * S + q == 0) ? 1u : 0u;
        __syncwarp(mask);
        mont_mul<S, T>(t, a, bs, st, n, np, k, mask);
      } else {
#pragma unroll
        for (int q = 0; q < S; ++q) t[q] = (k * S + q == 0) ? 1u : 0u;
      }
      __syncwarp();
    }
    if (valid) {
      const int v = only_node >= 0 ? only_node : key / K;
      const int b = only_node >= 0 ? key : key % K;
      const size_t cellrow = ((size_t)v * F + f) * K + b;
      store_slice<S>(hist + (cellrow * ngh + gh) * NL, t, k);
      if (count_out && gh == 0 && k == 0) {
        const int* o = off + (size_t)f * (NK + 1);
        count_out[cellrow] = o[key + 1] - o[key];
      }
    }
  }
}

template <int S, int T>
int occupancy_grid(const void* fn, size_t smem) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kBlock, smem) != cudaSuccess || b < 1) b = 1;
  return b * sm_count();
}

template <int S, int T>
pl_status run_prepare(const N2Const& P, const uint32_t* ct, size_t count, uint32_t* ctm, cudaStream_t s) {
  static int grid = 0;
  if (!grid) grid = occupancy_grid<S, T>((const void*)k_to_mont<S, T>, 0);
  const size_t ipw = 32 / T;
  const size_t blocks_needed = ((count + ipw - 1) / ipw + (kBlock / 32) - 1) / (kBlock / 32);
  const int g = (int)std::min<size_t>((size_t)grid, blocks_needed);
  {
    ProfScope _ps("to_mont", s);
    k_to_mont<S, T><<<g, kBlock, 0, s>>>(P, ct, count, ctm);
  }
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

template <int S, int T>
pl_status run_hist_products(const N2Const& P, const uint32_t* ctm, size_t M, size_t ghs, int ngh, const HistBufs& B,
                            const HistDesc* D, int F, int NK_max, int K, int tile, uint32_t* hist, int32_t* count_out,
                            cudaStream_t s) {
  const size_t smem = (size_t)S * T * (kBlock / T) * sizeof(uint32_t);
  static int grid_seg = 0, grid_comb = 0;
  if (!grid_seg) grid_seg = occupancy_grid<S, T>((const void*)k_seg_product<S, T>, smem);
  if (!grid_comb) grid_comb = occupancy_grid<S, T>((const void*)k_combine<S, T>, smem);
  {
    ProfScope _ps("seg_product", s);
    k_seg_product<S, T><<<grid_seg, kBlock, smem, s>>>(P, ctm, M, ghs, ngh, B.idx, B.off, B.choff, B.featoff, F, D,
                                                       tile, B.partial);
  }
  PL_CUDA_TRY(cudaGetLastError());
  const size_t ipw = 32 / T;
  const size_t items = (size_t)ngh * F * NK_max;
  const size_t blocks_needed = ((items + ipw - 1) / ipw + (kBlock / 32) - 1) / (kBlock / 32);
  const int gc = (int)std::min<size_t>((size_t)grid_comb, blocks_needed);
  {
    ProfScope _ps("combine", s);
    k_combine<S, T><<<gc, kBlock, smem, s>>>(P, B.partial, B.off, B.choff, B.featoff, F, D, K, ngh, hist, count_out);
  }
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

#define PL_N2_CASES(X) X(64, 4) X(64, 8) X(64, 16) X(128, 4) X(128, 8) X(128, 16) X(192, 8) X(192, 16) X(192, 32)

pl_status dispatch_prepare(int NL, int T, const N2Const& P, const uint32_t* ct, size_t count, uint32_t* ctm,
                           cudaStream_t s) {
#define PL_CASE(LL, TT) \
  if (NL == LL && T == TT) return run_prepare<LL / TT, TT>(P, ct, count, ctm, s);
  PL_N2_CASES(PL_CASE)
#undef PL_CASE
  return fail(PL_EINVAL, "no mod n^2 kernel for this (limbs, lanes) pair");
}

pl_status dispatch_products(int NL, int T, const N2Const& P, const uint32_t* ctm, size_t M, size_t ghs, int ngh,
                            const HistBufs& B, const HistDesc* D, int F, int NK_max, int K, int tile, uint32_t* hist,
                            int32_t* count_out, cudaStream_t s) {
#define PL_CASE(LL, TT)                                                                                        \
  if (NL == LL && T == TT)                                                                                     \
    return run_hist_products<LL / TT, TT>(P, ctm, M, ghs, ngh, B, D, F, NK_max, K, tile, hist, count_out, s);
  PL_N2_CASES(PL_CASE)
#undef PL_CASE
  return fail(PL_EINVAL, "no mod n^2 kernel for this (limbs, lanes) pair");
}

}  // namespace

bool agg_supported(int NL, int T) {
#define PL_CASE(LL, TT) \
  if (NL == LL && T == TT) return true;
  PL_N2_CASES(PL_CASE)
#undef PL_CASE
  return false;
}

HistLayout hist_layout(size_t M, int F, int NK_max, int tile, int NL) {
  HistLayout h{};
  const size_t max_chunks = (size_t)F * ((M + tile - 1) / tile + std::min<size_t>((size_t)NK_max, M));
  Carve cv;
  h.o_cnt = cv.take(sizeof(int) * (size_t)F * NK_max);
  h.o_off = cv.take(sizeof(int) * (size_t)F * (NK_max + 1));
  h.o_choff = cv.take(sizeof(int) * (size_t)F * (NK_max + 1));
  h.o_featch = cv.take(sizeof(int) * (size_t)F);
  h.o_featoff = cv.take(sizeof(int) * ((size_t)F + 1));
  h.o_desc = cv.take(sizeof(HistDesc));
  h.o_idx = cv.take(sizeof(int) * (size_t)F * (M ? M : 1));
  h.o_part = cv.take(sizeof(uint32_t) * (size_t)NL * 2 * (max_chunks ? max_chunks : 1));
  h.bytes = cv.off;
  return h;
}

HistBufs hist_bufs(const HistLayout& h, void* base) {
  char* b = static_cast<char*>(base);
  return HistBufs{reinterpret_cast<int*>(b + h.o_cnt),     reinterpret_cast<int*>(b + h.o_off),
                  reinterpret_cast<int*>(b + h.o_choff),   reinterpret_cast<int*>(b + h.o_featch),
                  reinterpret_cast<int*>(b + h.o_featoff), reinterpret_cast<HistDesc*>(b + h.o_desc),
                  reinterpret_cast<int*>(b + h.o_idx),     reinterpret_cast<uint32_t*>(b + h.o_part)};
}

pl_status launch_set_desc(HistDesc* D, int num_nodes, int NK, int only_node, cudaStream_t s) {
  k_set_desc<<<1, 1, 0, s>>>(D, num_nodes, NK, only_node);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

// One group-by + segmented product + combine; the node selection and NK come
// from B.desc on the device, buffers are sized for NK_max.
pl_status hist_enqueue(const pl_key* key, const AggCfg& cfg, const HistBufs& B, int NK_max, const uint32_t* d_ctm,
                       size_t M, size_t ghs, const uint8_t* d_bins, size_t bstride, int F, int K,
                       const int32_t* d_node, uint32_t* d_hist, int32_t* d_count, int* st, cudaStream_t s, int ngh) {
  const int tile = cfg.tile;
  PL_CUDA_TRY(cudaMemsetAsync(B.cnt, 0, sizeof(int) * (size_t)F * NK_max, s));
  const int gx = (int)std::min<size_t>((M + 255) / 256, 1024);
  dim3 grid(gx > 0 ? gx : 1, F);
  {
    ProfScope _ps("hist_count", s);
    k_hist_count<<<grid, 256, 0, s>>>(d_bins, bstride, d_node, M, K, B.desc, B.cnt, st);
  }
  PL_CUDA_TRY(cudaGetLastError());
  {
    ProfScope _ps("hist_scan", s);
    k_hist_scan<<<F, kScanBlock, 0, s>>>(B.cnt, B.desc, tile, B.off, B.choff, B.featch);
  }
  PL_CUDA_TRY(cudaGetLastError());
  {
    ProfScope _ps("feat_scan", s);
    k_feat_scan<<<1, kScanBlock, 0, s>>>(B.featch, F, B.featoff);
  }
  PL_CUDA_TRY(cudaGetLastError());
  PL_CUDA_TRY(cudaMemsetAsync(B.cnt, 0, sizeof(int) * (size_t)F * NK_max, s));
  {
    ProfScope _ps("hist_scatter", s);
    k_hist_scatter<<<grid, 256, 0, s>>>(d_bins, bstride, d_node, M, K, B.desc, B.off, B.cnt, B.idx, st);
  }
  PL_CUDA_TRY(cudaGetLastError());
  return dispatch_products(2 * key->L, cfg.T, key->n2c, d_ctm, M, ghs, ngh, B, B.desc, F, NK_max, K, tile, d_hist,
                           d_count, s);
}

pl_status launch_ct_prepare(pl_key* key, const uint32_t* d_ct, size_t count, uint32_t* d_ctm, cudaStream_t s) {
  if (count == 0) return PL_OK;
  return dispatch_prepare(2 * key->L, key->agg_cfg.T, key->n2c, d_ct, count, d_ctm, s);
}

pl_status launch_hist(pl_key* key, const uint32_t* d_ctm, size_t M, size_t ghs, const uint8_t* d_bins,
                      size_t bstride, int F, int K, const int32_t* d_node, int num_nodes, uint32_t* d_hist,
                      int32_t* d_count, bool per_node, int* st, cudaStream_t s, Scratch* scratch, int ngh) {
  const AggCfg cfg = key->agg_cfg;
  const int NK_max = per_node ? K : num_nodes * K;
  const HistLayout h = hist_layout(M, F, NK_max, per_node ? kWholeCell : cfg.tile, 2 * key->L);
  Scratch* sc = scratch ? scratch : key->scratch_for_current_device();
  if (!sc) return fail(PL_ECUDA, "no current device");
  void* base = sc->get(h.bytes, s);
  if (!base) return fail(PL_ENOMEM, "scratch allocation failed");
  const HistBufs B = hist_bufs(h, base);
  if (!per_node) {
    pl_status rc = launch_set_desc(B.desc, num_nodes, num_nodes * K, -1, s);
    if (rc) return rc;
    return hist_enqueue(key, cfg, B, NK_max, d_ctm, M, ghs, d_bins, bstride, F, K, d_node, d_hist, d_count, st, s,
                        ngh);
  }
  // the plain per-node method: one set of launches per node and one work
  // item (one lane group) per whole cell, no splitting of large cells
  const AggCfg plain{cfg.T, kWholeCell};
  for (int v = 0; v < num_nodes; ++v) {
    pl_status rc = launch_set_desc(B.desc, num_nodes, K, v, s);
    if (rc) return rc;
    rc = hist_enqueue(key, plain, B, NK_max, d_ctm, M, ghs, d_bins, bstride, F, K, d_node, d_hist, d_count, st, s,
                      ngh);
    if (rc) return rc;
  }
  return PL_OK;
}

}  // namespace pl

// ---------------------------------------------------------------------------
// Packing of histogram cells for fewer decryptions (see paillier_pack.h).
namespace pl {
namespace {

// One lane group per packed ciphertext: Horner over `slots` cells mod n^2,
// cells past `count` taken as the ciphertext 1 (an encryption of 0).
template <int S, int T>
__global__ void __launch_bounds__(kBlock) k_pack(const __grid_constant__ N2Const P, const uint32_t* __restrict__ ct,
                                                 size_t count, int slots, int B, uint32_t* __restrict__ packed,
                                                 size_t npacked) {
  constexpr int NL = S * T;
  constexpr int IPW = 32 / T;
  extern __shared__ uint32_t smem[];
  uint32_t* r2 = smem;                 // R^2 mod n^2, one shared copy
  uint32_t* cols = smem + NL;          // per-group multiplicand columns
  for (int j = threadIdx.x; j < NL; j += blockDim.x) r2[j] = P.R2[j];
  __syncthreads();
  const int ipb = blockDim.x / T;
  const int lane = threadIdx.x & 31, k = lane % T, gw = lane / T, g = threadIdx.x / T;
  uint32_t* bs = cols + g;
  const int st = ipb;
  uint32_t n[S], a[S], t[S], acc[S];
  const_slice<S>(n, P.N, k);
  const uint32_t np = P.np;
  const size_t nchunk = (npacked + IPW - 1) / IPW;
  const size_t warp0 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t c = warp0; c < nchunk; c += nwarps) {
    const size_t pi = c * IPW + gw;
    const bool valid = pi < npacked;
    const size_t base = (valid ? pi : npacked - 1) * (size_t)slots;
    // Montgomery form of cell `idx` (or of 1 past the end) into acc-shaped registers
    auto cell_mont = [&](size_t idx, uint32_t (&dst)[S]) {
      if (idx < count) {
        load_slice<S>(a, ct + idx * NL, k);
      } else {
#pragma unroll
        for (int j = 0; j < S; ++j) a[j] = (k * S + j == 0) ? 1u : 0u;
      }
      mont_mul<S, T>(dst, a, r2, 1, n, np, k);
    };
    cell_mont(base + slots - 1, acc);
    for (int j = slots - 2; j >= 0; --j) {
      for (int sq = 0; sq < B; ++sq) {
        __syncwarp();
        stage<S>(bs, st, acc, k);
        __syncwarp();
        mont_mul<S, T>(t, acc, bs, st, n, np, k);
#pragma unroll
        for (int q = 0; q < S; ++q) acc[q] = t[q];
      }
      cell_mont(base + j, t);
      __syncwarp();
      stage<S>(bs, st, t, k);
      __syncwarp();
      mont_mul<S, T>(t, acc, bs, st, n, np, k);
#pragma unroll
      for (int q = 0; q < S; ++q) acc[q] = t[q];
    }
    // leave Montgomery form
    __syncwarp();
#pragma unroll
    for (int q = 0; q < S; ++q) bs[(k * S + q) * st] = (k * S + q == 0) ? 1u : 0u;
    __syncwarp();
    mont_mul<S, T>(t, acc, bs, st, n, np, k);
    if (valid) store_slice<S>(packed + pi * NL, t, k);
  }
}

template <int S, int T>
pl_status run_pack(const N2Const& P, const uint32_t* ct, size_t count, int slots, int B, uint32_t* packed,
                   size_t npacked, cudaStream_t s) {
  constexpr int NL = S * T;
  const size_t smem = (size_t)NL * sizeof(uint32_t) * (1 + kBlock / T);
  static int grid = 0;
  if (!grid) grid = occupancy_grid<S, T>((const void*)k_pack<S, T>, smem);
  const size_t ipw = 32 / T;
  const size_t blocks_needed = ((npacked + ipw - 1) / ipw + (kBlock / 32) - 1) / (kBlock / 32);
  const int g = (int)std::min<size_t>((size_t)grid, blocks_needed);
  {
    ProfScope _ps("pack", s);
    k_pack<S, T><<<g, kBlock, smem, s>>>(P, ct, count, slots, B, packed, npacked);
  }
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

// plaintext [np][L] -> count values of B bits; bits past slots * B must be 0
__global__ void k_unpack(const uint32_t* __restrict__ plain, int L, size_t count, int slots, int B,
                         uint64_t* __restrict__ out, int* status) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const size_t pi = i / slots;
    const int j = (int)(i % slots);
    const uint32_t* x = plain + pi * L;
    const int bit = j * B;
    const int w = bit >> 5, sh = bit & 31;
    uint64_t v = (uint64_t)x[w] >> sh;
    if (w + 1 < L) v |= (uint64_t)x[w + 1] << (32 - sh);
    if (sh && w + 2 < L) v |= (uint64_t)x[w + 2] << (64 - sh);
    if (B < 64) v &= (1ull << B) - 1;
    out[i] = v;
    if (j == 0) {  // one check per packed plaintext: nothing above the last slot
      const int top = slots * B;
      uint32_t hi = 0;
      for (int q = top >> 5; q < L; ++q) hi |= (q == (top >> 5)) ? (x[q] >> (top & 31)) : x[q];
      if ((top & 31) == 0 && (top >> 5) < L) hi |= x[top >> 5];
      if (hi) atomicOr(status, kStatusRange);
    }
  }
}

}  // namespace

pl_status launch_pack(const pl_key* key, const uint32_t* ct, size_t count, int slots, int B, uint32_t* packed,
                      cudaStream_t s) {
  const size_t npacked = (count + slots - 1) / slots;
  if (!npacked) return PL_OK;
  const int NL = 2 * key->L;
  // each packed ciphertext is one long chain of products: with few of them,
  // twice the lanes per instance (where that kernel exists) shortens the
  // chain; at 2048-bit a 32-lane packing kernel (4 limbs per lane, packing
  // only) takes the 16-lane calls that still leave the GPU half empty
  // (measured: 13.5 against 18.6 ms for 500 packed ciphertexts, 25.5 against
  // 27.8 ms for 1,776)
  int T = key->agg_cfg.T;
  if (agg_supported(NL, 2 * T) && double_lanes_pays(npacked, T)) T *= 2;
  if (NL == 128 && T == 16 && double_lanes_pays(npacked, T)) T = 32;
#define PL_CASE(LL, TT) \
  if (NL == LL && T == TT) return run_pack<LL / TT, TT>(key->n2c, ct, count, slots, B, packed, npacked, s);
  PL_N2_CASES(PL_CASE)
  PL_CASE(128, 32)
#undef PL_CASE
  return fail(PL_EINVAL, "no mod n^2 kernel for this (limbs, lanes) pair");
}

pl_status launch_unpack(const uint32_t* plain, int L, size_t count, int slots, int B, uint64_t* out, int* st,
                        cudaStream_t s) {
  if (!count) return PL_OK;
  const int grid = (int)std::min<size_t>((count + 255) / 256, (size_t)sm_count() * 8);
  {
    ProfScope _ps("unpack", s);
    k_unpack<<<grid, 256, 0, s>>>(plain, L, count, slots, B, out, st);
  }
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

}  // namespace pl
