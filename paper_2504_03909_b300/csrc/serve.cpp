// Continuous-batching request loop: FIFO admission by free slot and HBM
// budget, concurrent execution on per-slot streams, completion by event query.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/paillier_serve.h"
#include "internal.h"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
  pl_request r{};
  int state = PL_REQ_QUEUED;
  int err = PL_OK;
  double t_submit = 0, latency = -1;
  size_t bytes = 0;
};

struct Slot {
  cudaStream_t s = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  uint64_t req = 0;
  pl::Scratch scratch;
  int* d_status = nullptr;
  int* h_status = nullptr;
  void* allocs[6] = {};
};

size_t round_up(size_t x) { return (x + 255) & ~size_t(255); }

// device memory one request needs while it runs
size_t request_bytes(const pl_request& r) {
  const size_t L = (size_t)r.key->L;
  const size_t ncell = (size_t)r.num_nodes * r.F * r.K;
  const size_t hcells = ncell * (r.gh_bits ? 1 : 2);  // histogram ciphertexts
  size_t b = round_up(hcells * 2 * L * 4) + round_up(ncell * 4) + round_up(ncell * 2 * 8);
  if (!r.d_node) b += round_up(r.M * 4);
  const pl::HistLayout h = pl::hist_layout(r.M, r.F, r.num_nodes * r.K, r.key->agg_cfg.tile, (int)(2 * L));
  size_t dec_cells = hcells;
  if (r.pack_bits > 0) {
    const int slot_bits = r.gh_bits ? 2 * r.gh_bits : r.pack_bits;
    const size_t slots = (size_t)(r.key->n_bits - 2) / (size_t)slot_bits;
    dec_cells = (hcells + slots - 1) / slots;
    b += round_up(dec_cells * 2 * L * 4) + round_up(dec_cells * L * 4);  // packed ciphertexts + plaintexts
  } else if (r.gh_bits) {
    b += round_up(dec_cells * L * 4);  // plaintexts before the split
  }
  b += std::max(h.bytes, pl::decrypt_scratch_bytes(r.key, dec_cells));
  return b;
}

}  // namespace

struct pl_server {
  int device = 0;
  size_t budget = 0, in_flight = 0, peak_bytes = 0;
  std::vector<Slot> slots;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::thread th;
  bool stop = false;
  uint64_t next_id = 1;
  long long n_sub = 0, n_done = 0, n_fail = 0, n_cancel = 0;
  int running = 0, peak_running = 0;

  void finish(Slot& sl, int err) {
    Req& q = reqs[sl.req];
    q.latency = now_ms() - q.t_submit;
    if (err == PL_OK && *sl.h_status != 0) err = (*sl.h_status & pl::kStatusRange) ? PL_ERANGE : PL_EDEVICE;
    q.err = err;
    q.state = err == PL_OK ? PL_REQ_DONE : PL_REQ_FAILED;
    (err == PL_OK ? n_done : n_fail)++;
    in_flight -= q.bytes;
    sl.busy = false;
    --running;
    done_cv.notify_all();
  }

  // enqueue one request on a slot's stream; returns a status (the slot stays
  // busy until its completion event, even after a launch error, so that
  // stream-ordered frees have run before the slot is reused)
  pl_status launch(Slot& sl, Req& q) {
    using namespace pl;
    const pl_request& r = q.r;
    pl_key* key = const_cast<pl_key*>(r.key);
    const size_t L = (size_t)key->L;
    const size_t ncell = (size_t)r.num_nodes * r.F * r.K;
    const size_t cells = ncell * 2;
    cudaStream_t s = sl.s;
    for (auto& a : sl.allocs) a = nullptr;
    pl_status rc = PL_OK;
    auto amalloc = [&](int i, size_t bytes) -> void* {
      if (cudaMallocAsync(&sl.allocs[i], bytes, s) != cudaSuccess) {
        cudaGetLastError();
        sl.allocs[i] = nullptr;
        rc = fail(PL_ENOMEM, "stream-ordered allocation failed");
      }
      return sl.allocs[i];
    };
    const int ngh = r.gh_bits ? 1 : 2;
    const size_t hcells = ncell * ngh;
    auto* hist = static_cast<uint32_t*>(amalloc(0, hcells * 2 * L * 4));
    auto* counts = static_cast<int32_t*>(amalloc(1, ncell * 4));
    auto* sums = static_cast<uint64_t*>(amalloc(2, cells * 8));
    const int32_t* node = r.d_node;
    if (!node) node = static_cast<int32_t*>(amalloc(3, r.M * 4));
    if (rc == PL_OK) {
      cudaMemsetAsync(sl.d_status, 0, sizeof(int), s);
      if (!r.d_node) cudaMemsetAsync(const_cast<int32_t*>(node), 0, r.M * 4, s);
      rc = launch_hist(key, r.d_ctm, r.M, r.gh_stride, r.d_bins, r.bins_stride, r.F, r.K, node, r.num_nodes, hist,
                       counts, false, sl.d_status, s, &sl.scratch, ngh);
    }
    if (rc == PL_OK && r.pack_bits > 0) {
      const int slot_bits = r.gh_bits ? 2 * r.gh_bits : r.pack_bits;
      const int slots = (key->n_bits - 2) / slot_bits;
      const size_t npacked = (hcells + slots - 1) / slots;
      auto* packed = static_cast<uint32_t*>(amalloc(4, npacked * 2 * L * 4));
      auto* plain = static_cast<uint32_t*>(amalloc(5, npacked * L * 4));
      if (rc == PL_OK) rc = launch_pack(key, hist, hcells, slots, slot_bits, packed, s);
      if (rc == PL_OK) rc = launch_decrypt(key, packed, npacked, plain, false, sl.d_status, s, &sl.scratch);
      if (rc == PL_OK)  // g/h cells: each 2B-bit slot is two B-bit sums
        rc = r.gh_bits ? launch_unpack(plain, (int)L, cells, 2 * slots, r.gh_bits, sums, sl.d_status, s)
                       : launch_unpack(plain, (int)L, cells, slots, r.pack_bits, sums, sl.d_status, s);
    } else if (rc == PL_OK && r.gh_bits) {
      auto* plain = static_cast<uint32_t*>(amalloc(5, hcells * L * 4));
      if (rc == PL_OK) rc = launch_decrypt(key, hist, hcells, plain, false, sl.d_status, s, &sl.scratch);
      if (rc == PL_OK) rc = launch_unpack(plain, (int)L, cells, 2, r.gh_bits, sums, sl.d_status, s);
    } else if (rc == PL_OK) {
      rc = launch_decrypt(key, hist, cells, sums, true, sl.d_status, s, &sl.scratch);
    }
    if (rc == PL_OK) {
      cudaMemcpyAsync(r.h_sums, sums, cells * 8, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(r.h_counts, counts, ncell * 4, cudaMemcpyDeviceToHost, s);
    }
    cudaMemcpyAsync(sl.h_status, sl.d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    for (auto& a : sl.allocs)
      if (a) cudaFreeAsync(a, s);
    sl.scratch.release(s);
    cudaEventRecord(sl.done, s);
    return rc;
  }

  void loop() {
    cudaSetDevice(device);
    std::unordered_map<int, pl_status> launch_err;  // slot -> error of its launch
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      // completions
      for (size_t i = 0; i < slots.size(); ++i) {
        Slot& sl = slots[i];
        if (!sl.busy) continue;
        const cudaError_t e = cudaEventQuery(sl.done);
        if (e == cudaErrorNotReady) continue;
        int err = e == cudaSuccess ? PL_OK : PL_ECUDA;
        auto it = launch_err.find((int)i);
        if (it != launch_err.end()) {
          if (err == PL_OK) err = it->second;
          launch_err.erase(it);
        }
        finish(sl, err);
      }
      if (stop && queue.empty() && running == 0) break;
      // admissions: FIFO, the head waits for a slot and for budget
      while (!queue.empty() && !stop) {
        auto fs = std::find_if(slots.begin(), slots.end(), [](const Slot& x) { return !x.busy; });
        if (fs == slots.end()) break;
        Req& q = reqs[queue.front()];
        if (in_flight + q.bytes > budget) break;
        const uint64_t id = queue.front();
        queue.pop_front();
        q.state = PL_REQ_RUNNING;
        in_flight += q.bytes;
        peak_bytes = std::max(peak_bytes, in_flight);
        fs->busy = true;
        fs->req = id;
        ++running;
        peak_running = std::max(peak_running, running);
        const pl_status rc = launch(*fs, q);
        if (rc != PL_OK) launch_err[(int)(fs - slots.begin())] = rc;
      }
      if (running == 0 && queue.empty()) {
        if (stop) break;
        cv.wait(lk, [&] { return stop || !queue.empty(); });
      } else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      }
    }
  }
};

extern "C" {

pl_status pl_server_create(int slots, size_t hbm_budget, pl_server** out) {
  using namespace pl;
  clear_error();
  if (!out || slots < 1 || slots > 256 || hbm_budget == 0) return fail(PL_EINVAL, "need 1 <= slots <= 256 and a budget");
  auto* srv = new (std::nothrow) pl_server();
  if (!srv) return fail(PL_ENOMEM, "host allocation failed");
  cudaError_t e = cudaGetDevice(&srv->device);
  if (e != cudaSuccess) { delete srv; return cuda_fail(e, "cudaGetDevice"); }
  // keep freed pool memory cached: stream-ordered allocations are reused without going back to the driver
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, srv->device) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  srv->budget = hbm_budget;
  srv->slots.resize((size_t)slots);
  for (auto& sl : srv->slots) {
    sl.scratch.async = true;
    sl.scratch.device = srv->device;
    if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&sl.d_status, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&sl.h_status, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      pl_server_destroy(srv);
      return fail(PL_ECUDA, "slot set-up failed");
    }
    *sl.h_status = 0;
  }
  srv->th = std::thread([srv] { srv->loop(); });
  *out = srv;
  return PL_OK;
}

pl_status pl_server_request_bytes(const pl_request* req, size_t* bytes) {
  using namespace pl;
  if (!req || !bytes || !req->key || req->num_nodes < 1 || req->F < 1 || req->K < 1) return fail(PL_EINVAL, "bad request");
  *bytes = request_bytes(*req);
  return PL_OK;
}

pl_status pl_server_submit(pl_server* srv, const pl_request* req, uint64_t* ticket) {
  using namespace pl;
  clear_error();
  if (!srv || !req || !ticket) return fail(PL_EINVAL, "NULL argument");
  const pl_request& r = *req;
  if (!r.key || !r.key->priv) return fail(PL_EINVAL, "a request needs a private key");
  if (r.M < 1 || r.F < 1 || r.K < 1 || r.K > 256 || r.num_nodes < 1) return fail(PL_EINVAL, "bad request sizes");
  if (!r.d_node && r.num_nodes != 1) return fail(PL_EINVAL, "num_nodes must be 1 without a node array");
  if ((long long)r.num_nodes * r.K > (1ll << 20) || r.M > ((size_t)1 << 30)) return fail(PL_EINVAL, "request too large");
  if ((!r.gh_bits && r.gh_stride < r.M) || r.bins_stride < r.M) return fail(PL_EINVAL, "strides must be >= M");
  if (r.gh_bits != 0 && (r.gh_bits < 26 || r.gh_bits > 64)) return fail(PL_EINVAL, "gh_bits must be 0 or 26..64");
  if (!r.d_ctm || !r.d_bins || !r.h_sums || !r.h_counts) return fail(PL_EINVAL, "NULL buffer");
  if (reinterpret_cast<uintptr_t>(r.d_ctm) & 15u) return fail(PL_EINVAL, "d_ctm must be 16-byte aligned");
  if (!agg_supported(2 * r.key->L, r.key->agg_cfg.T)) return fail(PL_EINVAL, "key configuration not supported");
  if (r.pack_bits < 0 || r.pack_bits > 64) return fail(PL_EINVAL, "pack_bits must be 0..64");
  Req q;
  q.r = r;
  q.bytes = request_bytes(r);
  std::lock_guard<std::mutex> lock(srv->mu);
  if (q.bytes > srv->budget) return fail(PL_EBUSY, "request needs more device memory than the whole budget");
  q.t_submit = now_ms();
  const uint64_t id = srv->next_id++;
  srv->reqs[id] = q;
  srv->queue.push_back(id);
  ++srv->n_sub;
  *ticket = id;
  srv->cv.notify_all();
  return PL_OK;
}

pl_status pl_server_poll(pl_server* srv, uint64_t ticket, int* state, double* latency_ms, int* error) {
  using namespace pl;
  if (!srv) return fail(PL_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return fail(PL_EINVAL, "unknown ticket");
  if (state) *state = it->second.state;
  if (latency_ms) *latency_ms = it->second.latency;
  if (error) *error = it->second.err;
  return PL_OK;
}

pl_status pl_server_wait(pl_server* srv, uint64_t ticket, int timeout_ms, int* state, double* latency_ms) {
  using namespace pl;
  if (!srv) return fail(PL_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return fail(PL_EINVAL, "unknown ticket");
  const bool ok = srv->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
    const int st = srv->reqs[ticket].state;
    return st != PL_REQ_QUEUED && st != PL_REQ_RUNNING;
  });
  const Req& q = srv->reqs[ticket];
  if (state) *state = q.state;
  if (latency_ms) *latency_ms = q.latency;
  if (!ok) return fail(PL_ETIMEDOUT, "request still pending");
  return PL_OK;
}

pl_status pl_server_cancel(pl_server* srv, uint64_t ticket) {
  using namespace pl;
  if (!srv) return fail(PL_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return fail(PL_EINVAL, "unknown ticket");
  if (it->second.state != PL_REQ_QUEUED) return fail(PL_EINVAL, "request already admitted");
  srv->queue.erase(std::remove(srv->queue.begin(), srv->queue.end(), ticket), srv->queue.end());
  it->second.state = PL_REQ_CANCELLED;
  ++srv->n_cancel;
  srv->done_cv.notify_all();
  return PL_OK;
}

pl_status pl_server_stats(pl_server* srv, long long* submitted, long long* completed, long long* failed,
                          long long* cancelled, int* peak_running, size_t* peak_bytes) {
  using namespace pl;
  if (!srv) return fail(PL_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(srv->mu);
  if (submitted) *submitted = srv->n_sub;
  if (completed) *completed = srv->n_done;
  if (failed) *failed = srv->n_fail;
  if (cancelled) *cancelled = srv->n_cancel;
  if (peak_running) *peak_running = srv->peak_running;
  if (peak_bytes) *peak_bytes = srv->peak_bytes;
  return PL_OK;
}

void pl_server_destroy(pl_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    for (uint64_t id : srv->queue) {
      srv->reqs[id].state = PL_REQ_CANCELLED;
      ++srv->n_cancel;
    }
    srv->queue.clear();
    srv->stop = true;
    srv->cv.notify_all();
    srv->done_cv.notify_all();
  }
  if (srv->th.joinable()) srv->th.join();
  cudaSetDevice(srv->device);
  for (auto& sl : srv->slots) {
    if (sl.s) cudaStreamSynchronize(sl.s);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.d_status) cudaFree(sl.d_status);
    if (sl.h_status) cudaFreeHost(sl.h_status);
    if (sl.s) cudaStreamDestroy(sl.s);
  }
  delete srv;
}

}  // extern "C"
