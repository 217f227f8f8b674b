// Continuous-batching request loop: admission by free slot, HBM budget and
// size class, concurrent execution on per-slot streams, launch groups issued
// by the loop as the device consumes them, completion by event query.
//
// Scheduling on the device.  The exponentiation and segmented-product kernels
// are persistent (a grid of the resident blocks loops over the work), so one
// launch of a large request holds every SM until it ends; a small request that
// arrives meanwhile waits for it (measured before this policy: requests of
// about 5 ms of work had a p50 of 159 ms and a p99 of 1.8 s at offered load
// 0.7).  Two rules bound that wait:
//   * a request's work is issued as launches of at most `chunk_imad` modelled
//     multiply-adds each (the histogram by groups of features, packing and
//     decryption by ranges of ciphertexts), so the GPU changes hands at least
//     every few tens of milliseconds; every launch computes the same cells as
//     one launch would, so the results are the same bits;
//   * requests run on a stream of their size class's priority (small: below
//     `small_imad`; large: above `large_imad`; medium between): at each such
//     boundary the block scheduler takes the pending blocks of the smaller
//     class first; a large request that has run for `promote_ms` continues at
//     the medium priority (its later groups ordered after its earlier ones by
//     an event), which bounds how long it keeps yielding.
// Admission: FIFO within each class, so a small request may pass a medium or
// large one that cannot start; medium and large requests together hold at most
// slots - `reserved` slots, so that small requests always find one free in
// time (measured with FIFO admission over all classes: small requests had a
// p99 of 1.8 s, waiting for one of 8 slots held by long requests).
// Packing: each packed ciphertext is a serial chain of (slots - 1)(B + 1)
// products, so a request with few cells keeps at least kPackChains packed
// ciphertexts (request_slots): shorter chains for a few more decryptions
// (measured: small requests' p50 69 -> 48 ms for 2.5 % of capacity).
#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <functional>
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
  int cls = 0;  // size class: 0 small, 1 medium, 2 large
  int state = PL_REQ_QUEUED;
  int err = PL_OK;
  double t_submit = 0, latency = -1;
  size_t bytes = 0;
};

struct Slot {
  cudaStream_t cs[3] = {};  // one stream per size class, in decreasing priority
  cudaStream_t s = nullptr;  // the stream of the request it runs
  int cls = 0;               // that request's class
  // the request's launch groups, issued by the server loop at most two ahead of
  // the device (step_ev[i & 1] is recorded after group i); `last` copies the
  // results out, frees the request's memory and records `done`
  std::vector<std::function<pl_status()>> plan;
  std::function<void(pl_status)> last;
  size_t next = 0;
  bool issued_all = false;
  pl_status err = PL_OK;
  cudaEvent_t step_ev[2] = {};
  cudaEvent_t xfer = nullptr;  // orders a promoted request's next groups after its earlier ones
  double t_start = 0;          // when the request was admitted (ms)
  int prio = 0;                // the priority level its groups run at now (0 highest)
  cudaEvent_t done = nullptr;
  bool busy = false;
  uint64_t req = 0;
  pl::Scratch scratch;
  int* d_status = nullptr;
  int* h_status = nullptr;
  void* allocs[6] = {};
};

size_t round_up(size_t x) { return (x + 255) & ~size_t(255); }

// modelled multiply-adds (IMAD: one 32-bit half of a limb product) of one Montgomery product on nl limbs
double mont_imad(double nl) { return 4 * nl * nl + nl; }
double hist_imad(const pl_request& r) {
  return (r.gh_bits ? 1.0 : 2.0) * (double)r.M * r.F * mont_imad(2.0 * r.key->L);
}

// automatic packing: packed ciphertexts a request of little histogram work
// keeps at least (packing stays latency-bound on the GPU up to about this many
// chains), and the histogram work from which a request packs as many cells as fit
constexpr size_t kPackChains = 1024;
constexpr double kPackFullImad = 3e12;

// cells per packed ciphertext of a request, 0: no packing (also when one cell
// per ciphertext would be chosen: the cells are then decrypted directly)
int request_slots(const pl_request& r) {
  if (r.pack_bits <= 0) return 0;
  const int slot_bits = r.gh_bits ? 2 * r.gh_bits : r.pack_bits;
  int slots = (r.key->n_bits - 2) / slot_bits;
  if (r.pack_slots > 0) {
    slots = std::min(slots, r.pack_slots);
  } else if (hist_imad(r) < kPackFullImad) {
    const size_t hcells = (size_t)r.num_nodes * r.F * r.K * (r.gh_bits ? 1 : 2);
    slots = (int)std::min<size_t>((size_t)slots, (hcells + kPackChains - 1) / kPackChains);
  }
  return slots >= 2 ? slots : 0;
}

// device memory one request needs while it runs
size_t request_bytes(const pl_request& r) {
  const size_t L = (size_t)r.key->L;
  const size_t ncell = (size_t)r.num_nodes * r.F * r.K;
  const size_t hcells = ncell * (r.gh_bits ? 1 : 2);  // histogram ciphertexts
  size_t b = round_up(hcells * 2 * L * 4) + round_up(ncell * 4) + round_up(ncell * 2 * 8);
  if (!r.d_node) b += round_up(r.M * 4);
  const pl::HistLayout h = pl::hist_layout(r.M, r.F, r.num_nodes * r.K, r.key->agg_cfg.tile, (int)(2 * L));
  size_t dec_cells = hcells;
  if (const size_t slots = (size_t)request_slots(r)) {
    dec_cells = (hcells + slots - 1) / slots;
    b += round_up(dec_cells * 2 * L * 4) + round_up(dec_cells * L * 4);  // packed ciphertexts + plaintexts
  } else if (r.gh_bits) {
    b += round_up(dec_cells * L * 4);  // plaintexts before the split
  }
  b += std::max(h.bytes, pl::decrypt_scratch_bytes(r.key, dec_cells));
  return b;
}

// modelled multiply-adds of the pieces of a request
double dec_imad(const pl_key* key) {
  // two CRT halves, about n_bits / 2 (1 + 1/6) products on L limbs each (sliding 6-bit windows)
  const double L = key->L;
  return 2.0 * (key->n_bits / 2.0) * (7.0 / 6.0) * mont_imad(L);
}
struct Work {
  double hist_per_feature, pack_per_ct, dec_per_ct, total;
};
Work request_work(const pl_request& r) {
  const double L2 = 2.0 * r.key->L;
  const int ngh = r.gh_bits ? 1 : 2;
  const double hcells = (double)r.num_nodes * r.F * r.K * ngh;
  Work w{};
  w.hist_per_feature = (double)ngh * (double)r.M * mont_imad(L2);
  w.dec_per_ct = dec_imad(r.key);
  double dec_cts = hcells;
  if (const int islots = request_slots(r)) {
    const int slot_bits = r.gh_bits ? 2 * r.gh_bits : r.pack_bits;
    const double slots = islots;
    w.pack_per_ct = slots * (slot_bits + 1) * mont_imad(L2);
    dec_cts = std::ceil(hcells / slots);
    w.total += dec_cts * w.pack_per_ct;
  }
  w.total += r.F * w.hist_per_feature + dec_cts * w.dec_per_ct;
  return w;
}

// smallest decryption launch of a split request: about half a wave of the
// 3072-bit exponentiation kernel, so that splitting costs little throughput
constexpr size_t kDecryptLaunchMin = 2048;

// items per launch so that one launch stays within `budget` (at least `floor_items`)
size_t per_launch(double budget, double per_item, size_t floor_items) {
  const double n = per_item > 0 ? std::floor(budget / per_item) : 1e18;
  return std::max<size_t>(floor_items, (size_t)std::max(1.0, std::min(n, 1e15)));
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
  // launch-size, priority and admission policy (see the top of this file)
  double chunk_imad = 0.3e12, small_imad = 0.3e12, large_imad = 3e12;
  int reserved = 0;
  long long n_class[3] = {0, 0, 0}, n_launch_groups = 0;
  int running_cls[3] = {0, 0, 0};
  int peak_nonsmall = 0;
  double promote_ms = 250;  // a large request running longer moves up to the medium priority (<= 0: never)
  long long n_promoted = 0;

  int classify(const pl_request& r) const {
    const double w = request_work(r).total;
    return w < small_imad ? 0 : (w <= large_imad ? 1 : 2);
  }

  void finish(Slot& sl, int err) {
    if (err == PL_OK) err = sl.err;
    Req& q = reqs[sl.req];
    q.latency = now_ms() - q.t_submit;
    if (err == PL_OK && *sl.h_status != 0) err = (*sl.h_status & pl::kStatusRange) ? PL_ERANGE : PL_EDEVICE;
    q.err = err;
    q.state = err == PL_OK ? PL_REQ_DONE : PL_REQ_FAILED;
    (err == PL_OK ? n_done : n_fail)++;
    in_flight -= q.bytes;
    sl.busy = false;
    --running;
    --running_cls[sl.cls];
    done_cv.notify_all();
  }

  // Sets up one request on a slot: its stream, its memory and its plan of
  // launch groups (issued later by `issue`).  The slot stays busy until its
  // completion event, even after an error, so that the stream-ordered frees
  // have run before the slot is reused.
  void launch(Slot& sl, Req& q) {
    using namespace pl;
    const pl_request r = q.r;
    pl_key* key = const_cast<pl_key*>(r.key);
    const size_t L = (size_t)key->L;
    const size_t ncell = (size_t)r.num_nodes * r.F * r.K;
    const size_t cells = ncell * 2;
    const Work wk = request_work(r);
    sl.cls = q.cls;
    sl.prio = q.cls;
    sl.t_start = now_ms();
    sl.s = sl.cs[q.cls];
    sl.plan.clear();
    sl.next = 0;
    sl.issued_all = false;
    sl.err = PL_OK;
    cudaStream_t s = sl.s;
    Slot* slp = &sl;
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
    const int slots = request_slots(r);
    const int slot_bits = slots ? (r.gh_bits ? 2 * r.gh_bits : r.pack_bits) : 0;
    const size_t npacked = slots ? (hcells + slots - 1) / slots : 0;
    uint32_t* packed = nullptr;
    uint32_t* plain = nullptr;
    if (slots) {
      packed = static_cast<uint32_t*>(amalloc(4, npacked * 2 * L * 4));
      plain = static_cast<uint32_t*>(amalloc(5, npacked * L * 4));
    } else if (r.gh_bits) {
      plain = static_cast<uint32_t*>(amalloc(5, hcells * L * 4));
    }
    // results out, memory freed, completion recorded (run once, after the last group or an error)
    sl.last = [slp, r, sums, counts, cells, ncell](pl_status err) {
      cudaStream_t st = slp->s;  // the stream of the request's last group (it may have been promoted)
      if (err == PL_OK) {
        cudaMemcpyAsync(r.h_sums, sums, cells * 8, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(r.h_counts, counts, ncell * 4, cudaMemcpyDeviceToHost, st);
      }
      cudaMemcpyAsync(slp->h_status, slp->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
      for (auto& a : slp->allocs)
        if (a) cudaFreeAsync(a, st);
      slp->scratch.release(st);
      cudaEventRecord(slp->done, st);
    };
    if (rc != PL_OK) {
      sl.err = rc;
      return;
    }
    cudaMemsetAsync(sl.d_status, 0, sizeof(int), s);
    if (!r.d_node) cudaMemsetAsync(const_cast<int32_t*>(node), 0, r.M * 4, s);
    auto& plan = sl.plan;
    // the histogram: a root-only request in groups of features (its cells are
    // contiguous per feature); with a node array, one group
    const size_t fg = r.num_nodes == 1 ? per_launch(chunk_imad, wk.hist_per_feature, 1) : (size_t)r.F;
    for (size_t f0 = 0; f0 < (size_t)r.F; f0 += fg) {
      const int nf = (int)std::min(fg, (size_t)r.F - f0);
      plan.push_back([=]() {
        return launch_hist(key, r.d_ctm, r.M, r.gh_stride, r.d_bins + f0 * r.bins_stride, r.bins_stride, nf, r.K,
                           node, r.num_nodes, hist + f0 * r.K * ngh * 2 * L, counts + f0 * r.K, false,
                           slp->d_status, slp->s, &slp->scratch, ngh);
      });
    }
    // decryption of n ciphertexts at `in` in ranges of bounded work (at least
    // kDecryptLaunchMin per launch); u64: 64-bit outputs, else L-limb plaintexts
    auto decrypt_ranges = [&](const uint32_t* in, size_t n, void* out, bool u64) {
      const size_t step = per_launch(chunk_imad, wk.dec_per_ct, kDecryptLaunchMin);
      for (size_t c0 = 0; c0 < n; c0 += step) {
        const size_t nc = std::min(step, n - c0);
        void* o = u64 ? static_cast<void*>(static_cast<uint64_t*>(out) + c0)
                      : static_cast<void*>(static_cast<uint32_t*>(out) + c0 * L);
        const uint32_t* src = in + c0 * 2 * L;
        plan.push_back([=]() { return launch_decrypt(key, src, nc, o, u64, slp->d_status, slp->s, &slp->scratch); });
      }
    };
    if (slots) {
      // packing in ranges of whole packed ciphertexts
      const size_t pstep = per_launch(chunk_imad, wk.pack_per_ct, 1);
      for (size_t p0 = 0; p0 < npacked; p0 += pstep) {
        const size_t np_ = std::min(pstep, npacked - p0);
        const size_t c0 = p0 * (size_t)slots;
        const size_t nc = std::min(np_ * (size_t)slots, hcells - c0);
        plan.push_back([=]() {
          return launch_pack(key, hist + c0 * 2 * L, nc, slots, slot_bits, packed + p0 * 2 * L, slp->s);
        });
      }
      decrypt_ranges(packed, npacked, plain, false);
      // g/h cells: each 2B-bit slot is two B-bit sums
      const int uslots = r.gh_bits ? 2 * slots : slots;
      const int ubits = r.gh_bits ? r.gh_bits : r.pack_bits;
      plan.push_back([=]() { return launch_unpack(plain, (int)L, cells, uslots, ubits, sums, slp->d_status, slp->s); });
    } else if (r.gh_bits) {
      decrypt_ranges(hist, hcells, plain, false);
      plan.push_back([=]() {
        return launch_unpack(plain, (int)L, cells, 2, r.gh_bits, sums, slp->d_status, slp->s);
      });
    } else {
      decrypt_ranges(hist, cells, sums, true);
    }
    n_launch_groups += (long long)plan.size();
  }

  // Issues the slot's next launch groups while at most two are in flight on
  // the device; after the last group (or an error) runs `last`.
  void issue(Slot& sl) {
    while (!sl.issued_all) {
      if (sl.err != PL_OK || sl.next == sl.plan.size()) {
        sl.last(sl.err);
        sl.issued_all = true;
        break;
      }
      if (sl.next >= 2 && cudaEventQuery(sl.step_ev[sl.next & 1]) == cudaErrorNotReady) break;
      // aging: a large request that has run for promote_ms continues at the
      // medium priority, so that it stops yielding to every medium request
      if (sl.prio == 2 && promote_ms > 0 && now_ms() - sl.t_start > promote_ms) {
        cudaEventRecord(sl.xfer, sl.s);
        cudaStreamWaitEvent(sl.cs[1], sl.xfer, 0);
        sl.s = sl.cs[1];
        sl.prio = 1;
        ++n_promoted;
      }
      const pl_status rc = sl.plan[sl.next]();
      cudaEventRecord(sl.step_ev[sl.next & 1], sl.s);
      ++sl.next;
      if (rc != PL_OK) sl.err = rc;
    }
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      // launch groups of the running requests, then completions
      for (auto& sl : slots)
        if (sl.busy) issue(sl);
      for (auto& sl : slots) {
        if (!sl.busy || !sl.issued_all) continue;
        const cudaError_t e = cudaEventQuery(sl.done);
        if (e == cudaErrorNotReady) continue;
        finish(sl, e == cudaSuccess ? PL_OK : PL_ECUDA);
      }
      if (stop && queue.empty() && running == 0) break;
      // admissions: FIFO within each size class; a request that cannot start
      // (no budget, or a medium/large one finding its share of the slots taken)
      // holds back the later requests of its class only
      bool blocked[3] = {false, false, false};
      for (auto it = queue.begin(); it != queue.end() && !stop;) {
        auto fs = std::find_if(slots.begin(), slots.end(), [](const Slot& x) { return !x.busy; });
        if (fs == slots.end()) break;
        Req& q = reqs[*it];
        const int c = q.cls;
        bool ok = !blocked[c] && in_flight + q.bytes <= budget;
        if (ok && c != 0 && running - running_cls[0] >= (int)slots.size() - reserved) ok = false;
        if (!ok) {
          blocked[c] = true;
          if (blocked[0] && blocked[1] && blocked[2]) break;  // nothing further can start now
          ++it;
          continue;
        }
        const uint64_t id = *it;
        it = queue.erase(it);
        q.state = PL_REQ_RUNNING;
        in_flight += q.bytes;
        peak_bytes = std::max(peak_bytes, in_flight);
        fs->busy = true;
        fs->req = id;
        ++running;
        ++running_cls[c];
        ++n_class[c];
        peak_running = std::max(peak_running, running);
        peak_nonsmall = std::max(peak_nonsmall, running - running_cls[0]);
        launch(*fs, q);
        issue(*fs);
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
  srv->reserved = slots >= 2 ? std::max(1, slots / 4) : 0;
  int prio_least = 0, prio_greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) {
    cudaGetLastError();
    prio_least = prio_greatest = 0;
  }
  // lower numbers are higher priorities: small, medium, large
  const int prio[3] = {prio_greatest, (prio_least + prio_greatest) / 2, prio_least};
  for (auto& sl : srv->slots) {
    sl.scratch.async = true;
    sl.scratch.device = srv->device;
    if (cudaStreamCreateWithPriority(&sl.cs[0], cudaStreamNonBlocking, prio[0]) != cudaSuccess ||
        cudaStreamCreateWithPriority(&sl.cs[1], cudaStreamNonBlocking, prio[1]) != cudaSuccess ||
        cudaStreamCreateWithPriority(&sl.cs[2], cudaStreamNonBlocking, prio[2]) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.step_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.step_ev[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.xfer, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&sl.d_status, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&sl.h_status, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      pl_server_destroy(srv);
      return fail(PL_ECUDA, "slot set-up failed");
    }
    *sl.h_status = 0;
    sl.s = sl.cs[2];
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

pl_status pl_server_request_plan(const pl_request* req, int* slots, double* work_imad) {
  using namespace pl;
  clear_error();
  if (!req || !req->key || req->num_nodes < 1 || req->F < 1 || req->K < 1) return fail(PL_EINVAL, "bad request");
  if (req->pack_bits < 0 || req->pack_bits > 64 || req->pack_slots < 0)
    return fail(PL_EINVAL, "pack_bits must be 0..64 and pack_slots >= 0");
  if (slots) *slots = request_slots(*req);
  if (work_imad) *work_imad = request_work(*req).total;
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
  if (r.pack_slots < 0) return fail(PL_EINVAL, "pack_slots must be >= 0");
  Req q;
  q.r = r;
  q.bytes = request_bytes(r);
  std::lock_guard<std::mutex> lock(srv->mu);
  q.cls = srv->classify(r);
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

pl_status pl_server_set_policy(pl_server* srv, double chunk_imad, double small_imad, double large_imad,
                               int reserved_slots) {
  using namespace pl;
  clear_error();
  if (!srv) return fail(PL_EINVAL, "server is NULL");
  if (!(chunk_imad > 0) || !(small_imad >= 0) || !(large_imad >= small_imad))
    return fail(PL_EINVAL, "need chunk_imad > 0 and 0 <= small_imad <= large_imad");
  std::lock_guard<std::mutex> lock(srv->mu);
  if (reserved_slots < 0 || reserved_slots >= (int)srv->slots.size())
    return fail(PL_EINVAL, "reserved_slots must be in [0, slots)");
  srv->chunk_imad = chunk_imad;
  srv->small_imad = small_imad;
  srv->large_imad = large_imad;
  srv->reserved = reserved_slots;
  return PL_OK;
}

pl_status pl_server_set_aging(pl_server* srv, double promote_ms) {
  using namespace pl;
  clear_error();
  if (!srv) return fail(PL_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(srv->mu);
  srv->promote_ms = promote_ms;
  return PL_OK;
}

pl_status pl_server_policy_stats(pl_server* srv, long long* per_class, long long* launch_groups,
                                 int* peak_nonsmall, long long* promoted) {
  using namespace pl;
  if (!srv) return fail(PL_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(srv->mu);
  if (per_class)
    for (int c = 0; c < 3; ++c) per_class[c] = srv->n_class[c];
  if (launch_groups) *launch_groups = srv->n_launch_groups;
  if (peak_nonsmall) *peak_nonsmall = srv->peak_nonsmall;
  if (promoted) *promoted = srv->n_promoted;
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
    for (auto st : sl.cs)
      if (st) cudaStreamSynchronize(st);
    if (sl.done) cudaEventDestroy(sl.done);
    for (auto ev : sl.step_ev)
      if (ev) cudaEventDestroy(ev);
    if (sl.xfer) cudaEventDestroy(sl.xfer);
    if (sl.d_status) cudaFree(sl.d_status);
    if (sl.h_status) cudaFreeHost(sl.h_status);
    for (auto st : sl.cs)
      if (st) cudaStreamDestroy(st);
  }
  delete srv;
}

}  // extern "C"
