// Launch-configuration autotuner: times every compiled candidate of an op on
// synthetic data with CUDA events and installs the fastest in the key.
// Results can be cached in a JSON-lines file keyed by (op, n_bits, SM count).
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/paillier_level.h"
#include "internal.h"

namespace {

struct Cand {
  int lanes, param;
};

std::vector<Cand> candidates(const pl_key* key, int op) {
  std::vector<Cand> c;
  if (op == PL_OP_ENCRYPT || op == PL_OP_DECRYPT) {
    for (int T : {2, 4, 8})
      if (pl::modexp_supported(key->L, T))
        for (int w : {4, 5, 6, 7}) c.push_back({T, w});
  } else {
    for (int T : {4, 8, 16})
      if (pl::agg_supported(2 * key->L, T))
        for (int tile : {16, 32, 64, 128, 256}) c.push_back({T, tile});
  }
  return c;
}

bool cache_lookup(const char* path, int op, int n_bits, int sms, Cand* out) {
  if (!path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (std::fgets(line, sizeof(line), f)) {
    int o, nb, sm, la, pa;
    if (std::sscanf(line, " {\"op\": %d, \"n_bits\": %d, \"sms\": %d, \"lanes\": %d, \"param\": %d", &o, &nb, &sm, &la,
                    &pa) == 5 &&
        o == op && nb == n_bits && sm == sms) {
      *out = {la, pa};  // the last matching line wins
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void cache_append(const char* path, int op, int n_bits, int sms, Cand c, double ms) {
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "{\"op\": %d, \"n_bits\": %d, \"sms\": %d, \"lanes\": %d, \"param\": %d, \"ms\": %.4f}\n", op, n_bits,
               sms, c.lanes, c.param, ms);
  std::fclose(f);
}

}  // namespace

extern "C" {

pl_status paillier_get_config(const pl_key* key, int op, int* lanes, int* param) {
  using namespace pl;
  if (!key) return fail(PL_EINVAL, "key is NULL");
  int l, p;
  if (op == PL_OP_ENCRYPT) { l = key->enc_cfg.T; p = key->enc_cfg.w; }
  else if (op == PL_OP_DECRYPT) { l = key->dec_cfg.T; p = key->dec_cfg.w; }
  else if (op == PL_OP_HIST) { l = key->agg_cfg.T; p = key->agg_cfg.tile; }
  else return fail(PL_EINVAL, "unknown op");
  if (lanes) *lanes = l;
  if (param) *param = p;
  return PL_OK;
}

pl_status paillier_set_config(pl_key* key, int op, int lanes, int param) {
  using namespace pl;
  clear_error();
  if (!key) return fail(PL_EINVAL, "key is NULL");
  if (op == PL_OP_ENCRYPT || op == PL_OP_DECRYPT) {
    if (!key->priv) return fail(PL_EINVAL, "a public key has no exponentiation kernels");
    if (!modexp_supported(key->L, lanes)) return fail(PL_EINVAL, "no exponentiation kernel with these lanes");
    if (param < 2 || param > 7) return fail(PL_EINVAL, "window must be 2..7");
    (op == PL_OP_ENCRYPT ? key->enc_cfg : key->dec_cfg) = {lanes, param};
    return PL_OK;
  }
  if (op == PL_OP_HIST) {
    if (!agg_supported(2 * key->L, lanes)) return fail(PL_EINVAL, "no mod n^2 kernel with these lanes");
    if (param < 1 || param > 4096) return fail(PL_EINVAL, "tile must be 1..4096");
    key->agg_cfg = {lanes, param};
    return PL_OK;
  }
  return fail(PL_EINVAL, "unknown op");
}

pl_status paillier_autotune(pl_key* key, int op, const char* cache_path, void* stream, int* lanes, int* param) {
  using namespace pl;
  clear_error();
  if (!key) return fail(PL_EINVAL, "key is NULL");
  if (op != PL_OP_ENCRYPT && op != PL_OP_DECRYPT && op != PL_OP_HIST) return fail(PL_EINVAL, "unknown op");
  if (op != PL_OP_HIST && !key->priv) return fail(PL_EINVAL, "a public key has no exponentiation kernels");
  const int sms = sm_count();
  Cand best{0, 0};
  if (cache_lookup(cache_path, op, key->n_bits, sms, &best)) {
    pl_status rc = paillier_set_config(key, op, best.lanes, best.param);
    if (rc == PL_OK) {
      if (lanes) *lanes = best.lanes;
      if (param) *param = best.param;
      return PL_OK;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* st = status_word([] { int d = 0; cudaGetDevice(&d); return d; }());
  if (!st) return fail(PL_ECUDA, "status word unavailable");
  const int L = key->L;
  // synthetic inputs, sized to many waves of the GPU so that the window
  // tables' cache behaviour is that of a full-size launch
  const size_t count = (size_t)sms * 256;                  // values (encrypt / decrypt)
  const size_t M = (size_t)sms * 256, F = 8, K = 256;      // histogram
  std::vector<void*> bufs;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    bufs.push_back(p);
    return p;
  };
  std::vector<Cand> cands = candidates(key, op);
  if (cands.empty()) return fail(PL_EINVAL, "no candidates for this key size");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&] {  // every path out after this point
    cudaStreamSynchronize(s);
    for (void* p : bufs) cudaFree(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(PL_ECUDA, "autotune events");
  }
  double best_ms = 1e30;
  pl_status rc = PL_OK;
  const ModexpCfg enc0 = key->enc_cfg, dec0 = key->dec_cfg;
  const AggCfg agg0 = key->agg_cfg;
  if (op == PL_OP_ENCRYPT || op == PL_OP_DECRYPT) {
    auto* in = static_cast<uint32_t*>(alloc(count * 2 * L * 4));
    auto* m = static_cast<uint64_t*>(alloc(count * 8));
    auto* out = static_cast<uint32_t*>(alloc(count * 2 * L * 4));
    if (!in || !m || !out) { cleanup(); return fail(PL_ENOMEM, "autotune buffers"); }
    launch_fill_random(in, count, 2 * L, 0, 1, s);
    launch_fill_random(reinterpret_cast<uint32_t*>(m), count, 2, 0, 2, s);
    for (const Cand& c : cands) {
      (op == PL_OP_ENCRYPT ? key->enc_cfg : key->dec_cfg) = {c.lanes, c.param};
      auto run = [&] {
        return op == PL_OP_ENCRYPT ? launch_encrypt(key, m, in, count, out, st, s)
                                   : launch_decrypt(key, in, count, out, false, st, s);
      };
      rc = run();  // warm-up (also loads the kernel)
      if (rc) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < 1 && !rc; ++r) rc = run();
      cudaEventRecord(e1, s);
      if (rc) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) { best_ms = ms; best = c; }
    }
  } else {
    auto* ctm = static_cast<uint32_t*>(alloc(2 * M * 2 * L * 4));
    auto* bins = static_cast<uint8_t*>(alloc(F * M));
    auto* node = static_cast<int32_t*>(alloc(M * 4));
    auto* hist = static_cast<uint32_t*>(alloc(F * K * 2 * 2 * L * 4));
    const HistLayout hl = hist_layout(M, (int)F, (int)K, 16, 2 * L);  // the smallest tile needs the most room
    void* scr = alloc(hl.bytes);
    if (!ctm || !bins || !node || !hist || !scr) { cleanup(); return fail(PL_ENOMEM, "autotune buffers"); }
    launch_fill_random(ctm, 2 * M, 2 * L, 1, 3, s);
    launch_fill_random(reinterpret_cast<uint32_t*>(bins), F * M / 4, 1, 0, 4, s);
    cudaMemsetAsync(node, 0, M * 4, s);
    const HistBufs B = hist_bufs(hl, scr);
    launch_set_desc(B.desc, 1, (int)K, -1, s);
    for (const Cand& c : cands) {
      const AggCfg cfg{c.lanes, c.param};
      auto run = [&] {
        return hist_enqueue(key, cfg, B, (int)K, ctm, M, M, bins, M, (int)F, (int)K, node, hist, nullptr, st, s);
      };
      rc = run();
      if (rc) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < 2 && !rc; ++r) rc = run();
      cudaEventRecord(e1, s);
      if (rc) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) { best_ms = ms; best = c; }
    }
  }
  cleanup();
  key->enc_cfg = enc0;
  key->dec_cfg = dec0;
  key->agg_cfg = agg0;
  if (rc) return rc;
  // (random inputs set no status bits: decryption writes full-width plaintexts
  // and every uint8 bin is < K = 256)
  rc = paillier_set_config(key, op, best.lanes, best.param);
  if (rc) return rc;
  cache_append(cache_path, op, key->n_bits, sms, best, op == PL_OP_HIST ? best_ms / 2 : best_ms);
  if (lanes) *lanes = best.lanes;
  if (param) *param = best.param;
  return PL_OK;
}

}  // extern "C"
