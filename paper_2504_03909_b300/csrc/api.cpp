// C-ABI entry points: argument checks, then the launchers.
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "check.cuh"
#include "../../include/paillier_pack.h"

#include <cstdio>
#include <vector>

namespace pl {

#ifdef PL_CHECKED
// the bounds words of every translation unit (registered at load time)
static std::vector<int (*)()>& bounds_readers() {
  static std::vector<int (*)()> v;
  return v;
}
static std::mutex g_bounds_mu;
void register_bounds_reader(int (*read_and_clear)()) {
  std::lock_guard<std::mutex> lock(g_bounds_mu);
  bounds_readers().push_back(read_and_clear);
}
static int read_all_bounds() {
  std::lock_guard<std::mutex> lock(g_bounds_mu);
  int v = 0;
  for (auto fn : bounds_readers()) v |= fn();
  return v;
}
#endif

namespace {
thread_local std::string g_err;
std::mutex g_status_mu;
std::map<int, int*> g_status;
}  // namespace

void set_error(const std::string& msg) { g_err = msg; }
void clear_error() { g_err.clear(); }
pl_status fail(pl_status code, const std::string& msg) {
  g_err = msg;
  return code;
}
pl_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? PL_ENOMEM : PL_ECUDA;
}

int* status_word(int device) {
  std::lock_guard<std::mutex> lock(g_status_mu);
  auto it = g_status.find(device);
  if (it != g_status.end()) return it->second;
  int* p = nullptr;
  if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
  if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
  g_status[device] = p;
  return p;
}

Scratch::~Scratch() {
  if (ptr) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    cudaDeviceSynchronize();
    cudaFree(ptr);
    cudaSetDevice(prev);
  }
}

void* Scratch::get(size_t bytes, cudaStream_t s) {
  if (bytes <= cap && ptr) return ptr;
  if (async) {
    if (ptr) cudaFreeAsync(ptr, s);
    ptr = nullptr;
    cap = 0;
    if (cudaMallocAsync(&ptr, bytes, s) != cudaSuccess) {
      cudaGetLastError();
      ptr = nullptr;
      return nullptr;
    }
    cap = bytes;
    return ptr;
  }
  if (ptr) {
    cudaDeviceSynchronize();
    cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
  }
  size_t want = bytes + bytes / 4 + (1 << 20);
  if (cudaMalloc(&ptr, want) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      ptr = nullptr;
      return nullptr;
    }
    want = bytes;
  }
  cap = want;
  return ptr;
}

void Scratch::release(cudaStream_t s) {
  if (ptr && async) cudaFreeAsync(ptr, s);
  if (!async) return;
  ptr = nullptr;
  cap = 0;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  }
  return n;
}

static int* current_status() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  return status_word(dev);
}

namespace {
std::atomic<unsigned long long> g_launches{0};
std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
struct Pending { std::string name; cudaEvent_t e0, e1; };
std::vector<Pending> g_pending;
std::map<std::string, std::pair<double, long long>> g_prof_acc;

void drain_pending() {  // caller holds g_prof_mu
  for (auto& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      auto& a = g_prof_acc[p.name];
      a.first += ms;
      a.second += 1;
    }
    cudaEventDestroy(p.e0);
    cudaEventDestroy(p.e1);
  }
  g_pending.clear();
}
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void adjust_launch_count(long long delta) { g_launches.fetch_add((unsigned long long)delta, std::memory_order_relaxed); }

ProfScope::ProfScope(const char* kernel, cudaStream_t stream) : name(kernel), s(stream) {
  nvtxRangePushA(kernel);  // a named range around every launch, for timeline tools
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  if (cudaEventCreate(&e0) != cudaSuccess) { e0 = nullptr; return; }
  cudaEventRecord(e0, s);
}

ProfScope::~ProfScope() {
  nvtxRangePop();
  note_launch();
  if (!e0) return;
  cudaEvent_t e1;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return; }
  cudaEventRecord(e1, s);
  std::lock_guard<std::mutex> lock(g_prof_mu);
  g_pending.push_back({name, e0, e1});
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace pl

using namespace pl;

extern "C" {

const char* paillier_last_error(void) { return pl::g_err.c_str(); }

unsigned long long paillier_launch_count(void) { return pl::g_launches.load(); }

pl_status paillier_profile(int enable) {
  std::lock_guard<std::mutex> lock(pl::g_prof_mu);
  pl::drain_pending();
  pl::g_prof_acc.clear();
  pl::g_prof_on.store(enable != 0);
  return PL_OK;
}

pl_status paillier_profile_read(const char* kernel, double* total_ms, long long* launches) {
  clear_error();
  if (!kernel || !total_ms) return fail(PL_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(pl::g_prof_mu);
  pl::drain_pending();
  auto it = pl::g_prof_acc.find(kernel);
  *total_ms = it == pl::g_prof_acc.end() ? 0.0 : it->second.first;
  if (launches) *launches = it == pl::g_prof_acc.end() ? 0 : it->second.second;
  return PL_OK;
}

pl_status paillier_sync(void* stream, int* device_status) {
  if (device_status) *device_status = 0;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
#ifdef PL_CHECKED
  {
    const int b = read_all_bounds();
    if (b) {
      char msg[96];
      std::snprintf(msg, sizeof msg, "bounds check failed (sites 0x%x)", b);
      return fail(PL_EDEVICE, msg);
    }
  }
#endif
  int* sw = current_status();
  if (!sw) return fail(PL_ECUDA, "status word unavailable");
  int v = 0;
  e = cudaMemcpy(&v, sw, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status)");
  if (v) {
    e = cudaMemset(sw, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(status)");
  }
  if (device_status) *device_status = v;
  if (v & kStatusTimeout) return fail(PL_ETIMEDOUT, "a bounded device wait ran out");
  if (v & kStatusRange) return fail(PL_ERANGE, "a decrypted value does not fit 64 bits");
  if (v & (kStatusBadBin | kStatusBadNode | kStatusEncode | kStatusCapacity | kStatusNonUnit | kStatusBadSplit)) {
    std::string m = "device reported bad input:";
    if (v & kStatusBadBin) m += " bin >= K;";
    if (v & kStatusBadNode) m += " node >= num_nodes;";
    if (v & kStatusEncode) m += " value outside [-1, 2^15];";
    if (v & kStatusCapacity) m += " work list over capacity;";
    if (v & kStatusNonUnit) m += " encryption randomness shares a factor with n;";
    if (v & kStatusBadSplit) m += " split feature >= F;";
    return fail(PL_EDEVICE, m);
  }
  return PL_OK;
}

pl_status paillier_encode(const float* d_v, size_t count, uint64_t* d_m, void* stream) {
  clear_error();
  if (count && (!d_v || !d_m)) return fail(PL_EINVAL, "NULL buffer");
  int* st = current_status();
  if (!st) return fail(PL_ECUDA, "status word unavailable");
  return launch_encode(d_v, count, d_m, st, static_cast<cudaStream_t>(stream));
}

pl_status paillier_decode(const uint64_t* d_s, const int32_t* d_cnt, size_t count, double* d_out, void* stream) {
  clear_error();
  if (count && (!d_s || !d_cnt || !d_out)) return fail(PL_EINVAL, "NULL buffer");
  return launch_decode(d_s, d_cnt, count, d_out, static_cast<cudaStream_t>(stream));
}

pl_status paillier_encrypt(const pl_key* key, const uint64_t* d_m, const uint32_t* d_r, size_t count,
                           uint32_t* d_ct, void* stream) {
  clear_error();
  if (!key) return fail(PL_EINVAL, "key is NULL");
  if (!key->priv) return fail(PL_EINVAL, "encryption here needs the private key (CRT split of r^n)");
  if (count == 0) return PL_OK;
  if (!d_m || !d_r || !d_ct) return fail(PL_EINVAL, "NULL buffer");
  if (!aligned16(d_r) || !aligned16(d_ct)) return fail(PL_EINVAL, "buffers must be 16-byte aligned");
  if (count > (size_t)1 << 30) return fail(PL_EINVAL, "count too large");
  int* st = current_status();
  if (!st) return fail(PL_ECUDA, "no usable CUDA device");
  return launch_encrypt(const_cast<pl_key*>(key), d_m, d_r, count, d_ct, st, static_cast<cudaStream_t>(stream));
}

pl_status paillier_ct_prepare(const pl_key* key, const uint32_t* d_ct, size_t count, uint32_t* d_ctm,
                              void* stream) {
  clear_error();
  if (!key) return fail(PL_EINVAL, "key is NULL");
  if (count == 0) return PL_OK;
  if (!d_ct || !d_ctm) return fail(PL_EINVAL, "NULL buffer");
  if (!aligned16(d_ct) || !aligned16(d_ctm)) return fail(PL_EINVAL, "buffers must be 16-byte aligned");
  if (!current_status()) return fail(PL_ECUDA, "no usable CUDA device");
  return launch_ct_prepare(const_cast<pl_key*>(key), d_ct, count, d_ctm, static_cast<cudaStream_t>(stream));
}

static pl_status hist_common(const pl_key* key, const uint32_t* d_ctm, size_t M, const uint8_t* d_bins, int F,
                             int K, const int32_t* d_node, int num_nodes, uint32_t* d_hist, int32_t* d_count,
                             void* stream, bool per_node) {
  clear_error();
  if (!key) return fail(PL_EINVAL, "key is NULL");
  if (F < 1 || K < 1 || K > 256 || num_nodes < 1) return fail(PL_EINVAL, "need F >= 1, 1 <= K <= 256, num_nodes >= 1");
  if ((long long)num_nodes * K > (1ll << 20)) return fail(PL_EINVAL, "num_nodes * K must be <= 2^20");
  if ((long long)F * num_nodes * K > (1ll << 28)) return fail(PL_EINVAL, "F * num_nodes * K too large");
  if (M > (size_t)1 << 30) return fail(PL_EINVAL, "M too large");
  if (!d_hist) return fail(PL_EINVAL, "NULL histogram buffer");
  if (M && (!d_ctm || !d_bins || !d_node)) return fail(PL_EINVAL, "NULL input buffer");
  if (!aligned16(d_hist) || (d_ctm && !aligned16(d_ctm))) return fail(PL_EINVAL, "buffers must be 16-byte aligned");
  int* st = current_status();
  if (!st) return fail(PL_ECUDA, "no usable CUDA device");
  return launch_hist(const_cast<pl_key*>(key), d_ctm, M, M, d_bins, M, F, K, d_node, num_nodes, d_hist, d_count,
                     per_node, st, static_cast<cudaStream_t>(stream));
}

pl_status paillier_hist_aggregate(const pl_key* key, const uint32_t* d_ctm, size_t M, const uint8_t* d_bins, int F,
                                  int K, const int32_t* d_node, int num_nodes, uint32_t* d_hist, int32_t* d_count,
                                  void* stream) {
  return hist_common(key, d_ctm, M, d_bins, F, K, d_node, num_nodes, d_hist, d_count, stream, false);
}

pl_status paillier_hist_aggregate_per_node(const pl_key* key, const uint32_t* d_ctm, size_t M,
                                           const uint8_t* d_bins, int F, int K, const int32_t* d_node,
                                           int num_nodes, uint32_t* d_hist, int32_t* d_count, void* stream) {
  return hist_common(key, d_ctm, M, d_bins, F, K, d_node, num_nodes, d_hist, d_count, stream, true);
}

static pl_status decrypt_common(const pl_key* key, const uint32_t* d_ct, size_t count, void* d_m, bool u64,
                                void* stream) {
  clear_error();
  if (!key) return fail(PL_EINVAL, "key is NULL");
  if (!key->priv) return fail(PL_EINVAL, "decryption needs the private key");
  if (count == 0) return PL_OK;
  if (!d_ct || !d_m) return fail(PL_EINVAL, "NULL buffer");
  if (!aligned16(d_ct) || !aligned16(d_m)) return fail(PL_EINVAL, "buffers must be 16-byte aligned");
  if (count > (size_t)1 << 30) return fail(PL_EINVAL, "count too large");
  int* st = current_status();
  if (!st) return fail(PL_ECUDA, "no usable CUDA device");
  return launch_decrypt(const_cast<pl_key*>(key), d_ct, count, d_m, u64, st, static_cast<cudaStream_t>(stream));
}

pl_status paillier_decrypt(const pl_key* key, const uint32_t* d_ct, size_t count, uint32_t* d_m, void* stream) {
  return decrypt_common(key, d_ct, count, d_m, false, stream);
}

pl_status paillier_decrypt_u64(const pl_key* key, const uint32_t* d_ct, size_t count, uint64_t* d_m, void* stream) {
  return decrypt_common(key, d_ct, count, d_m, true, stream);
}

int paillier_pack_slots(const pl_key* key, int slot_bits) {
  if (!key || slot_bits < 1 || slot_bits > 128) return 0;
  return (key->n_bits - 2) / slot_bits;
}

// cells per packed ciphertext: `slots` (1 .. the most that fit), 0 = the most that fit; -1 if invalid
static int resolve_slots(const pl_key* key, int slot_bits, int slots) {
  const int most = paillier_pack_slots(key, slot_bits);
  if (most < 1 || slots < 0 || slots > most) return -1;
  return slots ? slots : most;
}

pl_status paillier_pack_n(const pl_key* key, const uint32_t* d_ct, size_t count, int slot_bits, int slots,
                          uint32_t* d_packed, void* stream) {
  clear_error();
  if (!key) return fail(PL_EINVAL, "key is NULL");
  if (paillier_pack_slots(key, slot_bits) < 1) return fail(PL_EINVAL, "slot_bits must be 1..128");
  const int s = resolve_slots(key, slot_bits, slots);
  if (s < 1) return fail(PL_EINVAL, "slots must be 0..paillier_pack_slots(key, slot_bits)");
  if (count == 0) return PL_OK;
  if (!d_ct || !d_packed) return fail(PL_EINVAL, "NULL buffer");
  if (!aligned16(d_ct) || !aligned16(d_packed)) return fail(PL_EINVAL, "buffers must be 16-byte aligned");
  if (!current_status()) return fail(PL_ECUDA, "no usable CUDA device");
  return launch_pack(key, d_ct, count, s, slot_bits, d_packed, static_cast<cudaStream_t>(stream));
}

pl_status paillier_pack(const pl_key* key, const uint32_t* d_ct, size_t count, int slot_bits, uint32_t* d_packed,
                        void* stream) {
  return paillier_pack_n(key, d_ct, count, slot_bits, 0, d_packed, stream);
}

pl_status paillier_decrypt_packed_u64_n(const pl_key* key, const uint32_t* d_packed, size_t count, int slot_bits,
                                        int slots, uint64_t* d_m, void* stream) {
  clear_error();
  if (!key) return fail(PL_EINVAL, "key is NULL");
  if (!key->priv) return fail(PL_EINVAL, "decryption needs the private key");
  if (slot_bits < 1 || slot_bits > 64) return fail(PL_EINVAL, "slot_bits must be 1..64");
  const int sl = resolve_slots(key, slot_bits, slots);
  if (sl < 1) return fail(PL_EINVAL, "slots must be 0..paillier_pack_slots(key, slot_bits)");
  if (count == 0) return PL_OK;
  if (!d_packed || !d_m) return fail(PL_EINVAL, "NULL buffer");
  if (!aligned16(d_packed)) return fail(PL_EINVAL, "buffers must be 16-byte aligned");
  int* st = current_status();
  if (!st) return fail(PL_ECUDA, "no usable CUDA device");
  pl_key* k = const_cast<pl_key*>(key);
  const size_t npacked = (count + sl - 1) / sl;
  Scratch* aux = k->scratch_for_current_device(true);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* plain = static_cast<uint32_t*>(aux ? aux->get(npacked * key->L * sizeof(uint32_t), s) : nullptr);
  if (!plain) return fail(PL_ENOMEM, "scratch allocation failed");
  pl_status rc = launch_decrypt(k, d_packed, npacked, plain, false, st, s);
  if (rc) return rc;
  return launch_unpack(plain, key->L, count, sl, slot_bits, d_m, st, s);
}

pl_status paillier_decrypt_packed_u64(const pl_key* key, const uint32_t* d_packed, size_t count, int slot_bits,
                                      uint64_t* d_m, void* stream) {
  return paillier_decrypt_packed_u64_n(key, d_packed, count, slot_bits, 0, d_m, stream);
}

pl_status paillier_encode_gh(const float* d_g, const float* d_h, size_t count, int B, uint64_t* d_m, void* stream) {
  clear_error();
  if (B < 26 || B > 64) return fail(PL_EINVAL, "B must be 26..64");
  if (count == 0) return PL_OK;
  if (!d_g || !d_h || !d_m) return fail(PL_EINVAL, "NULL buffer");
  if (count > (size_t)1 << 30) return fail(PL_EINVAL, "count too large");
  int* st = current_status();
  if (!st) return fail(PL_ECUDA, "no usable CUDA device");
  return launch_encode_gh(d_g, d_h, count, B, d_m, st, static_cast<cudaStream_t>(stream));
}

pl_status paillier_encrypt_gh(const pl_key* key, const uint64_t* d_m, const uint32_t* d_r, size_t count,
                              uint32_t* d_ct, void* stream) {
  clear_error();
  if (!key) return fail(PL_EINVAL, "key is NULL");
  if (!key->priv) return fail(PL_EINVAL, "encryption here needs the private key (CRT split of r^n)");
  if (count == 0) return PL_OK;
  if (!d_m || !d_r || !d_ct) return fail(PL_EINVAL, "NULL buffer");
  if (!aligned16(d_r) || !aligned16(d_ct)) return fail(PL_EINVAL, "buffers must be 16-byte aligned");
  if (count > (size_t)1 << 30) return fail(PL_EINVAL, "count too large");
  int* st = current_status();
  if (!st) return fail(PL_ECUDA, "no usable CUDA device");
  return launch_encrypt(const_cast<pl_key*>(key), d_m, d_r, count, d_ct, st, static_cast<cudaStream_t>(stream),
                        nullptr, 2);
}

pl_status paillier_hist_aggregate_gh(const pl_key* key, const uint32_t* d_ctm, size_t M, const uint8_t* d_bins,
                                     int F, int K, const int32_t* d_node, int num_nodes, uint32_t* d_hist,
                                     int32_t* d_count, void* stream) {
  clear_error();
  if (!key) return fail(PL_EINVAL, "key is NULL");
  if (F < 1 || K < 1 || K > 256 || num_nodes < 1) return fail(PL_EINVAL, "need F >= 1, 1 <= K <= 256, num_nodes >= 1");
  if ((long long)num_nodes * K > (1ll << 20)) return fail(PL_EINVAL, "num_nodes * K must be <= 2^20");
  if ((long long)F * num_nodes * K > (1ll << 28)) return fail(PL_EINVAL, "F * num_nodes * K too large");
  if (M > (size_t)1 << 30) return fail(PL_EINVAL, "M too large");
  if (!d_hist) return fail(PL_EINVAL, "NULL histogram buffer");
  if (M && (!d_ctm || !d_bins || !d_node)) return fail(PL_EINVAL, "NULL input buffer");
  if (!aligned16(d_hist) || (d_ctm && !aligned16(d_ctm))) return fail(PL_EINVAL, "buffers must be 16-byte aligned");
  int* st = current_status();
  if (!st) return fail(PL_ECUDA, "no usable CUDA device");
  return launch_hist(const_cast<pl_key*>(key), d_ctm, M, 0, d_bins, M, F, K, d_node, num_nodes, d_hist, d_count,
                     false, st, static_cast<cudaStream_t>(stream), nullptr, 1);
}

// decrypt `nct` ciphertexts into the aux scratch, then split each plaintext
// into `per` cells of 2B bits, each into (low B bits, next B bits)
static pl_status decrypt_split(const pl_key* key, const uint32_t* d_ct, size_t nct, size_t cells, int per, int B,
                               uint64_t* d_sums, void* stream) {
  int* st = current_status();
  if (!st) return fail(PL_ECUDA, "no usable CUDA device");
  pl_key* k = const_cast<pl_key*>(key);
  Scratch* aux = k->scratch_for_current_device(true);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* plain = static_cast<uint32_t*>(aux ? aux->get(nct * key->L * sizeof(uint32_t), s) : nullptr);
  if (!plain) return fail(PL_ENOMEM, "scratch allocation failed");
  pl_status rc = launch_decrypt(k, d_ct, nct, plain, false, st, s);
  if (rc) return rc;
  return launch_unpack(plain, key->L, 2 * cells, 2 * per, B, d_sums, st, s);
}

pl_status paillier_decrypt_gh(const pl_key* key, const uint32_t* d_ct, size_t count, int B, uint64_t* d_sums,
                              void* stream) {
  clear_error();
  if (!key) return fail(PL_EINVAL, "key is NULL");
  if (!key->priv) return fail(PL_EINVAL, "decryption needs the private key");
  if (B < 26 || B > 64) return fail(PL_EINVAL, "B must be 26..64");
  if (count == 0) return PL_OK;
  if (!d_ct || !d_sums) return fail(PL_EINVAL, "NULL buffer");
  if (!aligned16(d_ct)) return fail(PL_EINVAL, "buffers must be 16-byte aligned");
  if (count > (size_t)1 << 30) return fail(PL_EINVAL, "count too large");
  return decrypt_split(key, d_ct, count, count, 1, B, d_sums, stream);
}

pl_status paillier_decrypt_packed_gh_n(const pl_key* key, const uint32_t* d_packed, size_t cells, int B, int slots,
                                       uint64_t* d_sums, void* stream) {
  clear_error();
  if (!key) return fail(PL_EINVAL, "key is NULL");
  if (!key->priv) return fail(PL_EINVAL, "decryption needs the private key");
  if (B < 26 || B > 64) return fail(PL_EINVAL, "B must be 26..64");
  if (paillier_pack_slots(key, 2 * B) < 1) return fail(PL_EINVAL, "no slot of 2B bits fits the key");
  const int sl = resolve_slots(key, 2 * B, slots);
  if (sl < 1) return fail(PL_EINVAL, "slots must be 0..paillier_pack_slots(key, 2B)");
  if (cells == 0) return PL_OK;
  if (!d_packed || !d_sums) return fail(PL_EINVAL, "NULL buffer");
  if (!aligned16(d_packed)) return fail(PL_EINVAL, "buffers must be 16-byte aligned");
  if (cells > (size_t)1 << 30) return fail(PL_EINVAL, "count too large");
  return decrypt_split(key, d_packed, (cells + sl - 1) / sl, cells, sl, B, d_sums, stream);
}

pl_status paillier_decrypt_packed_gh(const pl_key* key, const uint32_t* d_packed, size_t cells, int B,
                                     uint64_t* d_sums, void* stream) {
  return paillier_decrypt_packed_gh_n(key, d_packed, cells, B, 0, d_sums, stream);
}

}  // extern "C"
