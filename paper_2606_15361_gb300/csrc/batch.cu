// Many beams per step: every beam is its own plan (its own DM grid, chunk length, options
// and workspace), and one call advances all of them by one chunk each.
//
// The tree, the dominant stage, runs as few launches as possible: beams whose plans share
// a kernel instantiation and block shape go into one k_tree_multi launch, whose CTAs are
// spread over the beams by a prefix of their tile counts (the per-beam arguments travel by
// value in the launch's parameter block). The encoders, and then the matched filter and
// candidate stages, run per beam spread over four side streams forked from and joined back
// to the caller's stream around the tree launches. With graphs enabled the whole step is
// captured on a private stream and launched as one CUDA graph on the caller's stream; the
// next step's capture updates the instantiated graph in place (cudaGraphExecUpdate)
// whenever the topology is unchanged, so a steady stream of chunks re-uses one executable
// graph.

#include <algorithm>
#include <functional>
#include <new>
#include <vector>

#include "snd_internal.h"

using snd::Plan;

namespace snd {

int ForkJoin::init(int n) {
  if (!streams.empty()) return SND_OK;
  for (int i = 0; i < n; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SND_ERR_CUDA;
    streams.push_back(st);
  }
  for (int i = 0; i < 2 * n; ++i) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return SND_ERR_CUDA;
    events.push_back(e);
  }
  return SND_OK;
}

cudaError_t ForkJoin::fork(cudaStream_t main) {
  const size_t n = streams.size();
  cudaError_t e = cudaEventRecord(events[0], main);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(streams[i], events[0], 0);
  return e;
}

cudaError_t ForkJoin::join(cudaStream_t main) {
  const size_t n = streams.size();
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
    e = cudaEventRecord(events[n + i], streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(main, events[n + i], 0);
  }
  return e;
}

ForkJoin::~ForkJoin() {
  for (cudaEvent_t e : events) cudaEventDestroy(e);
  for (cudaStream_t st : streams) cudaStreamDestroy(st);
}

int enqueue_plans(Plan* const* plans, int n, const uint8_t* const* d_chunks, const int32_t* nsamp, cudaStream_t s,
                  cudaStream_t owner, ForkJoin* fj) {
  std::vector<ChunkPos> pos(n);
  std::vector<const Plan*> tp;
  std::vector<int64_t> ep, en;
  const int ns = fj ? static_cast<int>(fj->streams.size()) : 0;
  auto side = [&](int i) { return ns ? fj->streams[i % ns] : s; };
  if (ns && fj->fork(s) != cudaSuccess) return SND_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    Plan& p = *plans[i];
    pos[i] = chunk_pos(p, nsamp[i]);
    if (launch_encode(p, d_chunks[i], nsamp[i], side(i)) != cudaSuccess) return SND_ERR_CUDA;
  }
  if (ns && fj->join(s) != cudaSuccess) return SND_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    Plan& p = *plans[i];
    if (pos[i].e_new <= pos[i].e_prev) continue;
    if (p.mode == SND_MODE_ZFLOAT) {
      if (launch_tree_z(p, pos[i].e_prev, pos[i].e_new, nullptr, s) != cudaSuccess) return SND_ERR_CUDA;
    } else if (p.flags & SND_FLAG_REFERENCE_TREE) {
      if (launch_tree(p, pos[i].e_prev, pos[i].e_new, s) != cudaSuccess) return SND_ERR_CUDA;
    } else {
      tp.push_back(&p);
      ep.push_back(pos[i].e_prev);
      en.push_back(pos[i].e_new);
    }
  }
  if (!tp.empty() && launch_tree_batch(tp.data(), ep.data(), en.data(), static_cast<int>(tp.size()), s) != cudaSuccess)
    return SND_ERR_CUDA;
  if (ns && fj->fork(s) != cudaSuccess) return SND_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    Plan& p = *plans[i];
    if (p.mode == SND_MODE_ZFLOAT) continue;
    if (chunk_post(p, pos[i], nullptr, side(i), [](int, auto&& f) { return f(); }) != cudaSuccess)
      return SND_ERR_CUDA;
  }
  if (ns && fj->join(s) != cudaSuccess) return SND_ERR_CUDA;
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
  snd::ForkJoin fj;  // side streams for the per-beam stages
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
  Batch* b = new (std::nothrow) Batch();
  if (!b) return SND_ERR_NOMEM;
  for (int i = 0; i < nplans; ++i) {
    if (!plans[i]) {
      delete b;
      return SND_ERR_ARG;
    }
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) {
        delete b;
        return SND_ERR_ARG;
      }
    b->plans.push_back(reinterpret_cast<Plan*>(plans[i]));
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
  if (n > 1 && b.fj.init(std::min(n, 4)) != SND_OK) return fail(b, SND_ERR_CUDA);
  snd::ForkJoin* fj = n > 1 ? &b.fj : nullptr;
  const int rc = b.graph ? b.runner.run(s, [&](cudaStream_t cs) {
    return snd::enqueue_plans(plans, n, d_chunks, nsamp, cs, s, fj);
  })
                         : snd::enqueue_plans(plans, n, d_chunks, nsamp, s, s, fj);
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
