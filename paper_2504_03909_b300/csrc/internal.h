// Library-internal declarations shared by the host translation units.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/paillier.h"
#include "../../include/paillier_bench.h"
#include "hostmp.h"
#include "kparams.h"

namespace pl {

// ---- errors ---------------------------------------------------------------
void set_error(const std::string& msg);
void clear_error();
pl_status fail(pl_status code, const std::string& msg);
pl_status cuda_fail(cudaError_t e, const char* what);

#define PL_CUDA_TRY(call)                                   \
  do {                                                      \
    cudaError_t _e = (call);                                \
    if (_e != cudaSuccess) return ::pl::cuda_fail(_e, #call); \
  } while (0)

// ---- device status word (one per device, allocated on first use) ---------
int* status_word(int device);

// ---- scratch: one device buffer per key and device, grown on demand -------
struct Scratch {
  int device = -1;
  void* ptr = nullptr;
  size_t cap = 0;
  // stream-ordered mode (serving slots): grows with cudaFreeAsync /
  // cudaMallocAsync on the caller's stream instead of synchronising the device
  bool async = false;
  cudaStream_t astream = nullptr;
  ~Scratch();
  // returns a buffer of at least `bytes` (reallocates when it is too small);
  // nullptr on failure
  void* get(size_t bytes, cudaStream_t s = nullptr);
  // stream-ordered release (async mode)
  void release(cudaStream_t s);
};

// bump allocation inside one scratch request
struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  }
};

// ---- launch configuration (set by the autotuner or by the caller) --------
struct ModexpCfg {
  int T = 4;  // lanes per instance
  int w = 5;  // window bits
};
// a tile this large never splits a cell: one work item per non-empty cell
constexpr int kWholeCell = 1 << 30;
struct AggCfg {
  int T = 8;      // lanes per instance (mod n^2)
  int tile = 64;  // ciphertexts per work item of the segmented product
};

}  // namespace pl

// The key object behind the opaque C handle.
struct pl_key {
  int n_bits = 0, L = 0, Lh = 0;
  bool priv = false;
  plh::Big n, n2, p, q;
  pl::N2Const n2c{};
  // private part
  pl::HalfConst half[2]{};
  plh::Big e_enc1[2];    // encryption, mod x: the other prime mod (x - 1)
  plh::Big e_enc2[2];    // encryption, mod x^2: x itself
  plh::Big e_dec[2];     // p - 1, q - 1
  pl::EncCrtParams enc{};
  pl::DecCrtParams dec{};
  // launch configuration
  pl::ModexpCfg enc_cfg, dec_cfg;
  pl::AggCfg agg_cfg;
  // per-window exponentiation schedules (built on demand)
  std::map<int, std::unique_ptr<pl::ModexpParams>> enc_params, dec_params;
  std::mutex mu;
  // scratch per device (the second one holds results that outlive a call's
  // first scratch use, e.g. packed plaintexts between decryption and unpacking)
  std::map<int, std::unique_ptr<pl::Scratch>> scratch, scratch_aux;

  const pl::ModexpParams* modexp_params(bool dec, int w);
  pl::Scratch* scratch_for_current_device(bool aux = false);
};

namespace pl {
// launchers (kernels translation units)
pl_status launch_encode(const float* d_v, size_t count, uint64_t* d_m, int* st, cudaStream_t s);
pl_status launch_encode_gh(const float* d_g, const float* d_h, size_t count, int B, uint64_t* d_m, int* st,
                           cudaStream_t s);
pl_status launch_decode(const uint64_t* d_s, const int32_t* d_cnt, size_t count, double* d_out, cudaStream_t s);
// st: device status word (kStatusNonUnit for randomness sharing a factor with n); may be null
pl_status launch_encrypt(pl_key* key, const uint64_t* d_m, const uint32_t* d_r, size_t count, uint32_t* d_ct,
                         int* st, cudaStream_t s, Scratch* scratch = nullptr, int mw = 1);
pl_status launch_decrypt(pl_key* key, const uint32_t* d_ct, size_t count, void* d_out, bool u64, int* st,
                         cudaStream_t s, Scratch* scratch = nullptr);
size_t decrypt_scratch_bytes(const pl_key* key, size_t count);

// Sliding-window schedule of exponent e (> 0) for window w (layout in
// ModexpParams); returns the number of ops, or -1 if more than maxops.
int sliding_schedule(const plh::Big& e, int w, uint8_t* op, int maxops);

// Window-table entries per instance (the odd powers below 2^w).
__host__ __device__ constexpr size_t table_entries(int w) { return (size_t)1 << (w - 1); }
pl_status launch_ct_prepare(pl_key* key, const uint32_t* d_ct, size_t count, uint32_t* d_ctm, cudaStream_t s);
// ngh: ciphertext arrays per sample (2: g and h at stride ghs; 1: one g/h-packed
// array); d_hist [num_nodes][F][K][ngh][2L]
pl_status launch_hist(pl_key* key, const uint32_t* d_ctm, size_t M, size_t ghs, const uint8_t* d_bins,
                      size_t bstride, int F, int K, const int32_t* d_node, int num_nodes, uint32_t* d_hist,
                      int32_t* d_count, bool per_node, int* st, cudaStream_t s, Scratch* scratch = nullptr,
                      int ngh = 2);
int sm_count();
// Whether a call of `instances` independent product chains at T lanes each
// runs faster at 2T lanes.  Below about 1.5 warps per SM sub-partition the SMs
// are latency-bound and an instance at 2T lanes finishes about 1.5-1.7x
// sooner; above it the configured lanes have the higher throughput (measured
// on B300 for encryption and decryption at 2048-bit and packing at 2048- and
// 3072-bit: the crossover lies between 1.3 and 1.7 warps per sub-partition).
inline bool double_lanes_pays(size_t instances, int T) {
  const size_t warps = (instances * (size_t)T + 31) / 32;
  return 2 * warps <= (size_t)12 * (size_t)sm_count();
}
pl_status launch_pack(const pl_key* key, const uint32_t* ct, size_t count, int slots, int B, uint32_t* packed,
                      cudaStream_t s);
pl_status launch_unpack(const uint32_t* plain, int L, size_t count, int slots, int B, uint64_t* out, int* st,
                        cudaStream_t s);

// ---- histogram pass pieces shared with the level plan ----------------------
struct HistBufs {
  int* cnt;
  int* off;
  int* choff;
  int* featch;
  int* featoff;
  HistDesc* desc;
  int* idx;
  uint32_t* partial;
};
struct HistLayout {
  size_t o_cnt, o_off, o_choff, o_featch, o_featoff, o_desc, o_idx, o_part, bytes;
};
bool agg_supported(int NL, int T);
HistLayout hist_layout(size_t M, int F, int NK_max, int tile, int NL);
HistBufs hist_bufs(const HistLayout& h, void* base);
pl_status launch_set_desc(HistDesc* D, int num_nodes, int NK, int only_node, cudaStream_t s);
pl_status hist_enqueue(const pl_key* key, const AggCfg& cfg, const HistBufs& B, int NK_max, const uint32_t* d_ctm,
                       size_t M, size_t ghs, const uint8_t* d_bins, size_t bstride, int F, int K,
                       const int32_t* d_node, uint32_t* d_hist, int32_t* d_count, int* st, cudaStream_t s,
                       int ngh = 2);

// ---- tracing: launch counter and optional per-kernel CUDA-event timing ----
void note_launch();
void adjust_launch_count(long long delta);
bool modexp_supported(int L, int T);
pl_status launch_fill_random(uint32_t* p, size_t rows, int row_limbs, int zero_top, uint64_t seed, cudaStream_t s);
// Records CUDA events around one launch on `s` when profiling is on.
struct ProfScope {
  const char* name;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr;
  ProfScope(const char* kernel, cudaStream_t stream);
  ~ProfScope();
};
}  // namespace pl
