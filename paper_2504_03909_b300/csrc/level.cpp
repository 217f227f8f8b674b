// Batched tree-level path: one pass over all nodes of a level, captured once
// into a CUDA graph and replayed for every level (the level's node count is
// written to device memory before each replay; the kernels read it there).
#include <cstring>
#include <vector>

#include "../../include/paillier_level.h"
#include "internal.h"

struct pl_level_plan {
  const pl_key* key = nullptr;
  size_t M = 0;
  int F = 0, K = 0, max_nodes = 0, NK_max = 0;
  int ngh = 2;  // ciphertext arrays per sample: 2 (g, h) or 1 (g/h packed)
  pl::AggCfg cfg;
  int device = 0;
  void* buf = nullptr;
  pl::HistBufs B{};
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* ptrs[5] = {};
  int captures = 0, replays = 0, kernels = 0;

  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
  ~pl_level_plan() {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    cudaDeviceSynchronize();
    drop_graph();
    if (cap) cudaStreamDestroy(cap);
    if (buf) cudaFree(buf);
    cudaSetDevice(prev);
  }
};

extern "C" {

static pl_status plan_create(const pl_key* key, size_t M, int F, int K, int max_nodes, int ngh, pl_level_plan** out) {
  using namespace pl;
  clear_error();
  if (!key || !out) return fail(PL_EINVAL, "NULL argument");
  if (F < 1 || K < 1 || K > 256 || max_nodes < 1) return fail(PL_EINVAL, "need F >= 1, 1 <= K <= 256, max_nodes >= 1");
  if ((long long)max_nodes * K > (1ll << 20)) return fail(PL_EINVAL, "max_nodes * K must be <= 2^20");
  if (M > (size_t)1 << 30) return fail(PL_EINVAL, "M too large");
  auto* p = new (std::nothrow) pl_level_plan();
  if (!p) return fail(PL_ENOMEM, "host allocation failed");
  p->key = key;
  p->M = M;
  p->F = F;
  p->K = K;
  p->max_nodes = max_nodes;
  p->NK_max = max_nodes * K;
  p->ngh = ngh;
  p->cfg = key->agg_cfg;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaGetDevice"); }
  const HistLayout h = hist_layout(M, F, p->NK_max, p->cfg.tile, 2 * key->L);
  e = cudaMalloc(&p->buf, h.bytes);
  if (e != cudaSuccess) { p->buf = nullptr; delete p; return cuda_fail(e, "cudaMalloc(level plan)"); }
  p->B = hist_bufs(h, p->buf);
  e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) { p->cap = nullptr; delete p; return cuda_fail(e, "cudaStreamCreate"); }
  *out = p;
  return PL_OK;
}

pl_status paillier_level_plan_create(const pl_key* key, size_t M, int F, int K, int max_nodes, pl_level_plan** out) {
  return plan_create(key, M, F, K, max_nodes, 2, out);
}

pl_status paillier_level_plan_create_gh(const pl_key* key, size_t M, int F, int K, int max_nodes,
                                        pl_level_plan** out) {
  return plan_create(key, M, F, K, max_nodes, 1, out);
}

pl_status paillier_level_run(pl_level_plan* plan, const uint32_t* d_ctm, const uint8_t* d_bins, const int32_t* d_node,
                             int num_nodes, uint32_t* d_hist, int32_t* d_count, void* stream) {
  using namespace pl;
  clear_error();
  if (!plan) return fail(PL_EINVAL, "plan is NULL");
  if (num_nodes < 1 || num_nodes > plan->max_nodes) return fail(PL_EINVAL, "num_nodes out of the plan's range");
  if (!d_hist || (plan->M && (!d_ctm || !d_bins || !d_node))) return fail(PL_EINVAL, "NULL buffer");
  if ((reinterpret_cast<uintptr_t>(d_hist) | reinterpret_cast<uintptr_t>(d_ctm)) & 15u)
    return fail(PL_EINVAL, "buffers must be 16-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != plan->device) return fail(PL_EINVAL, "plan belongs to another device");
  int* st = status_word(dev);
  if (!st) return fail(PL_ECUDA, "status word unavailable");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  pl_status rc = launch_set_desc(plan->B.desc, num_nodes, num_nodes * plan->K, -1, s);
  if (rc) return rc;
  const void* ptrs[5] = {d_ctm, d_bins, d_node, d_hist, d_count};
  if (!plan->exec || std::memcmp(ptrs, plan->ptrs, sizeof(ptrs)) != 0) {
    plan->drop_graph();
    const unsigned long long before = paillier_launch_count();
    e = cudaStreamBeginCapture(plan->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    rc = hist_enqueue(plan->key, plan->cfg, plan->B, plan->NK_max, d_ctm, plan->M, plan->M, d_bins, plan->M,
                      plan->F, plan->K, d_node, d_hist, d_count, st, plan->cap, plan->ngh);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(plan->cap, &g);
    // kernels are counted when a replay launches them, not when they are captured
    adjust_launch_count((long long)before - (long long)paillier_launch_count());
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    plan->graph = g;
    e = cudaGraphInstantiate(&plan->exec, g, 0);
    if (e != cudaSuccess) { plan->exec = nullptr; plan->drop_graph(); return cuda_fail(e, "cudaGraphInstantiate"); }
    size_t n = 0;
    cudaGraphGetNodes(g, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    cudaGraphGetNodes(g, nodes.data(), &n);
    int kn = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kn;
    }
    plan->kernels = kn;
    std::memcpy(plan->ptrs, ptrs, sizeof(ptrs));
    ++plan->captures;
  }
  e = cudaGraphLaunch(plan->exec, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  adjust_launch_count(plan->kernels);
  ++plan->replays;
  return PL_OK;
}

pl_status paillier_level_plan_stats(const pl_level_plan* plan, int* captures, int* replays, int* kernels) {
  if (!plan) return pl::fail(PL_EINVAL, "plan is NULL");
  if (captures) *captures = plan->captures;
  if (replays) *replays = plan->replays;
  if (kernels) *kernels = plan->kernels;
  return PL_OK;
}

void paillier_level_plan_free(pl_level_plan* plan) { delete plan; }

}  // extern "C"
