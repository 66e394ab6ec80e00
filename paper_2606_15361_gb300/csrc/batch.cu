// Many beams per step: every beam is its own plan (its own DM grid, chunk length, options
// and workspace), and one call advances all of them by one chunk each.
//
// Every stage of a step runs for all beams at once, in a fixed handful of launches:
//  * the encoders: three launches (histogram, levels, pack) whose CTAs are spread over the
//    beams by a prefix of their CTA counts;
//  * the trees: one persistent launch per kernel instantiation, whose resident CTAs take
//    (beam, DM tile, time tile) work items from a device counter until none is left;
//  * the matched filters: one launch, one CTA per (beam, DM row);
//  * the candidate stages: one cooperative launch whose stages are separated by bounded
//    grid-wide barriers.
// The per-beam arguments travel by value in each launch's parameter block. With graphs
// enabled the whole step is
// captured on a private stream and launched as one CUDA graph on the caller's stream; the
// next step's capture updates the instantiated graph in place (cudaGraphExecUpdate)
// whenever the topology is unchanged, so a steady stream of chunks re-uses one executable
// graph.

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <functional>
#include <new>
#include <vector>

#include "snd_internal.h"

using snd::Plan;

namespace snd {

int enqueue_plans(Plan* const* plans, int n, const uint8_t* const* d_chunks, const int32_t* nsamp, cudaStream_t s,
                  cudaStream_t owner) {
  std::vector<ChunkPos> pos(n);
  std::vector<const Plan*> cp(plans, plans + n);
  std::vector<const Plan*> tp, post;
  std::vector<ChunkPos> ppos;
  std::vector<int64_t> ep, en;
  for (int i = 0; i < n; ++i) pos[i] = chunk_pos(*plans[i], nsamp[i]);
  // 1. every encoder (three launches for all bit-ring plans; each clears its block counters)
  if (launch_encode_batch(cp.data(), d_chunks, nsamp, n, s) != cudaSuccess) return SND_ERR_CUDA;
  // 2. the trees: one persistent launch per kernel instantiation
  for (int i = 0; i < n; ++i) {
    Plan& p = *plans[i];
    if (pos[i].e_new <= pos[i].e_prev) continue;
    if (p.mode == SND_MODE_ZFLOAT) {
      if (launch_tree_z(p, pos[i].e_prev, pos[i].e_new, nullptr, s) != cudaSuccess) return SND_ERR_CUDA;
    } else if ((p.flags & SND_FLAG_REFERENCE_TREE) || ((p.flags & SND_FLAG_LEVEL_RATES) && p.mode != SND_MODE_BINARY)) {
      if (launch_tree(p, pos[i].e_prev, pos[i].e_new, s) != cudaSuccess) return SND_ERR_CUDA;
    } else {
      tp.push_back(&p);
      ep.push_back(pos[i].e_prev);
      en.push_back(pos[i].e_new);
    }
  }
  if (!tp.empty() && launch_tree_batch(tp.data(), ep.data(), en.data(), static_cast<int>(tp.size()), s) != cudaSuccess)
    return SND_ERR_CUDA;
  // 3. every matched filter in one launch, 4. every candidate stage in one cooperative launch
  for (int i = 0; i < n; ++i) {
    if (plans[i]->mode == SND_MODE_ZFLOAT) continue;
    post.push_back(plans[i]);
    ppos.push_back(pos[i]);
  }
  if (!post.empty()) {
    const int np = static_cast<int>(post.size());
    if (launch_mf_batch(post.data(), ppos.data(), np, s) != cudaSuccess) return SND_ERR_CUDA;
    if (launch_candidates_batch(post.data(), ppos.data(), np, s) != cudaSuccess) return SND_ERR_CUDA;
  }
  for (int i = 0; i < n; ++i) chunk_commit(*plans[i], pos[i], nsamp[i], owner);
  return SND_OK;
}

int GraphRunner::run(cudaStream_t s, const std::function<int(cudaStream_t)>& enqueue) {
  // capture on a private stream (the caller's may be the legacy default stream, which cannot
  // be captured); the graph is then launched on the caller's stream, in its order
  if (!capture && cudaStreamCreateWithFlags(&capture, cudaStreamNonBlocking) != cudaSuccess) return SND_ERR_CUDA;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SND_ERR_CUDA;
  const int rc = enqueue(capture);
  const cudaError_t ec = cudaStreamEndCapture(capture, &g);
  if (rc || ec != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    return rc ? rc : SND_ERR_CUDA;
  }
  cudaError_t e = cudaSuccess;
  if (exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(exec, g, &info) != cudaSuccess) {
      cudaGetLastError();  // an update that does not apply is not an error: instantiate anew
      cudaGraphExecDestroy(exec);
      exec = nullptr;
    } else {
      ++updates;
    }
  }
  if (!exec) {
    e = cudaGraphInstantiate(&exec, g, 0);
    ++instantiations;
  }
  cudaGraphDestroy(g);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
  return e == cudaSuccess ? SND_OK : SND_ERR_CUDA;
}

GraphRunner::~GraphRunner() {
  if (exec) cudaGraphExecDestroy(exec);
  if (capture) cudaStreamDestroy(capture);
}

}  // namespace snd

namespace {

struct Batch {
  std::vector<Plan*> plans;
  bool graph = false;
  snd::GraphRunner runner;
  int sticky = 0;
};

int fail(Batch& b, int code) {
  if (!b.sticky) b.sticky = code;
  return code;
}

}  // namespace

extern "C" int snd_batch_create(const snd_plan_t* plans, int32_t nplans, snd_batch_t* out) {
  if (out) *out = nullptr;
  if (!out || !plans || nplans < 1 || nplans > 4096) return SND_ERR_ARG;
  for (int i = 0; i < nplans; ++i) {
    if (!plans[i]) return SND_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return SND_ERR_ARG;
  }
  Batch* b = nullptr;
  try {
    snd::alloc_point();
    b = new Batch();
    snd::alloc_point();  // the plan list
    for (int i = 0; i < nplans; ++i) b->plans.push_back(reinterpret_cast<Plan*>(plans[i]));
  } catch (const std::bad_alloc&) {
    delete b;
    return SND_ERR_NOMEM;
  }
  *out = reinterpret_cast<snd_batch_t>(b);
  return SND_OK;
}

extern "C" int snd_batch_set_graph(snd_batch_t h, int32_t enable) {
  if (!h) return SND_ERR_ARG;
  reinterpret_cast<Batch*>(h)->graph = enable != 0;
  return SND_OK;
}

extern "C" int snd_batch_execute(snd_batch_t h, const uint8_t* const* d_chunks, const int32_t* nsamp, void* stream) {
  if (!h || !d_chunks || !nsamp) return SND_ERR_ARG;
  Batch& b = *reinterpret_cast<Batch*>(h);
  if (b.sticky) return b.sticky;
  for (size_t i = 0; i < b.plans.size(); ++i) {
    const Plan& p = *b.plans[i];
    if (p.sticky) return p.sticky;
    if (!p.bound) return SND_ERR_STATE;
    if (!d_chunks[i]) return SND_ERR_ARG;
    if (nsamp[i] < 1 || nsamp[i] > p.max_chunk) return SND_ERR_CHUNK;
    if (p.profiling) return SND_ERR_STATE;  // per-stage events are not recorded in a batch
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Plan* const* plans = b.plans.data();
  const int n = static_cast<int>(b.plans.size());
  nvtxRangePushA("snd.batch_step");
  const int rc = b.graph ? b.runner.run(s, [&](cudaStream_t cs) {
    return snd::enqueue_plans(plans, n, d_chunks, nsamp, cs, s);
  })
                         : snd::enqueue_plans(plans, n, d_chunks, nsamp, s, s);
  nvtxRangePop();
  return rc ? fail(b, rc) : SND_OK;
}

extern "C" int snd_batch_graph_stats(snd_batch_t h, int64_t* instantiations, int64_t* updates) {
  if (!h) return SND_ERR_ARG;
  const Batch& b = *reinterpret_cast<Batch*>(h);
  if (instantiations) *instantiations = b.runner.instantiations;
  if (updates) *updates = b.runner.updates;
  return SND_OK;
}

extern "C" void snd_batch_destroy(snd_batch_t h) { delete reinterpret_cast<Batch*>(h); }
