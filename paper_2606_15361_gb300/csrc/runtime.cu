// Stream runtime of the SND library: workspace binding, per-chunk launch sequence on the
// caller's stream, and the candidate read-back. Streaming follows Methods, "Pipeline
// overview", in ring-buffer form: after a chunk the plane samples [E_prev, E_new) with
// E = max(0, samples consumed - D) are emitted (each has its full delay history), and the
// matched filter scores start times [F_prev, F_new) with F = max(0, E - (Wmax - 1)).

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "snd_internal.h"

using snd::Plan;

namespace snd {

ChunkPos chunk_pos(const Plan& p, int32_t nsamp) {
  ChunkPos c;
  c.e_prev = p.E;
  c.e_new = std::max<int64_t>(0, p.T + nsamp - p.D);
  c.f_prev = p.F;
  c.f_new = std::max<int64_t>(0, c.e_new - (p.wmax - 1));
  c.nb = static_cast<int>(c.f_new - c.f_prev);
  return c;
}

void chunk_commit(Plan& p, const ChunkPos& c, int32_t nsamp, cudaStream_t s) {
  p.T += nsamp;
  p.E = c.e_new;
  p.F = (p.mode == SND_MODE_ZFLOAT) ? p.F : c.f_new;
  p.last_stream = s;
  p.pending_host = -1;
}

}  // namespace snd

namespace {

int fail(Plan& p, int code) {
  if (!p.sticky) p.sticky = code;
  return code;
}

template <typename T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

template <typename T>
cudaError_t upload(void* base, size_t off, const std::vector<T>& v, cudaStream_t s) {
  if (v.empty()) return cudaSuccess;
  return cudaMemcpyAsync(at<T>(base, off), v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

cudaError_t mark(Plan& p, cudaStream_t s, size_t* slot) {
  if (p.ev_used == p.ev_pool.size()) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
    p.ev_pool.push_back(ev);
  }
  *slot = p.ev_used++;
  return cudaEventRecord(p.ev_pool[*slot], s);
}

// Run one stage inside an NVTX range named for it (host-side enqueue time in a timeline
// profiler), bracketed by an event pair when profiling.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

const char* stage_name(int id) {
  static const char* const names[SND_NUM_STAGES] = {"snd.encode", "snd.tree", "snd.matched_filter", "snd.candidates"};
  return (id >= 0 && id < SND_NUM_STAGES) ? names[id] : "snd.stage";
}

template <typename F>
cudaError_t stage(Plan& p, int id, cudaStream_t s, F&& f) {
  NvtxRange range(stage_name(id));
  if (!p.profiling) return f();
  size_t a = 0, b = 0;
  cudaError_t e = mark(p, s, &a);
  if (e == cudaSuccess) e = f();
  if (e == cudaSuccess) e = mark(p, s, &b);
  if (e == cudaSuccess) p.ev_marks.push_back({id, {a, b}});
  return e;
}

int run_chunk(Plan& p, const uint8_t* d_chunk, int32_t nsamp, cudaStream_t s, void* d_plane_out,
              int32_t* nemit_out) {
  NvtxRange range("snd.execute");
  const snd::ChunkPos c = snd::chunk_pos(p, nsamp);
  cudaError_t e = stage(p, SND_STAGE_ENCODE, s, [&] { return snd::launch_encode(p, d_chunk, nsamp, s); });
  if (p.mode == SND_MODE_ZFLOAT) {
    // labelled-payload plane only: no matched filter or candidates
    if (e == cudaSuccess && c.e_new > c.e_prev)
      e = stage(p, SND_STAGE_TREE, s, [&] { return snd::launch_tree_z(p, c.e_prev, c.e_new, d_plane_out, s); });
  } else {
    if (e == cudaSuccess && c.e_new > c.e_prev)
      e = stage(p, SND_STAGE_TREE, s, [&] { return snd::launch_tree(p, c.e_prev, c.e_new, s); });
    if (e == cudaSuccess) e = snd::chunk_post(p, c, d_plane_out, s, [&](int id, auto&& f) { return stage(p, id, s, f); });
  }
  if (e != cudaSuccess) return fail(p, SND_ERR_CUDA);
  snd::chunk_commit(p, c, nsamp, s);
  if (nemit_out) *nemit_out = static_cast<int32_t>(c.e_new - c.e_prev);
  return SND_OK;
}

}  // namespace

extern "C" int snd_bind_workspace(snd_plan_t plan, void* d_ws, size_t bytes, void* stream) {
  if (!plan) return SND_ERR_ARG;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (!d_ws || bytes < p.ws_bytes || (reinterpret_cast<uintptr_t>(d_ws) & 255u)) return SND_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  snd::DevPtrs& dp = p.dp;
  const auto& o = p.off;
  dp.ring = at<uint32_t>(d_ws, o.ring);
  dp.hist = at<uint32_t>(d_ws, o.hist);
  dp.levels = at<int32_t>(d_ws, o.levels);
  dp.plane = at<int32_t>(d_ws, o.plane);
  dp.mask = at<uint32_t>(d_ws, o.mask);
  dp.mask2 = at<uint32_t>(d_ws, o.mask2);
  dp.mask3 = at<uint32_t>(d_ws, o.mask3);
  dp.cells = at<snd::MfCell>(d_ws, o.cells);
  dp.counters = at<uint32_t>(d_ws, o.counters);
  dp.row_runs = at<int32_t>(d_ws, o.row_runs);
  dp.run_start = at<int32_t>(d_ws, o.run_start);
  dp.run_end = at<int32_t>(d_ws, o.run_end);
  dp.run_row = at<int32_t>(d_ws, o.run_row);
  dp.parent = at<int32_t>(d_ws, o.parent);
  dp.npix = at<int32_t>(d_ws, o.npix);
  dp.peak = at<unsigned long long>(d_ws, o.peak);
  dp.pwidth = at<int32_t>(d_ws, o.pwidth);
  dp.bcand = at<snd_candidate_t>(d_ws, o.bcand);
  dp.cand = at<snd_candidate_t>(d_ws, o.cand);
  dp.staging = at<uint8_t>(d_ws, o.staging);
  dp.staging2 = at<uint8_t>(d_ws, o.staging2);
  dp.width_mask = at<uint16_t>(d_ws, o.width_mask);
  dp.dm_f32 = at<float>(d_ws, o.dm_f32);
  dp.tp_off = at<int32_t>(d_ws, o.tp_off);
  dp.gepk = at<uint32_t>(d_ws, o.gepk);
  dp.gleaf = at<int32_t>(d_ws, o.gleaf);
  dp.gmeta = at<uint32_t>(d_ws, o.gmeta);
  dp.tile_wb = at<int32_t>(d_ws, o.tile_wb);
  dp.delays = at<int32_t>(d_ws, o.delays);
  dp.dmeta = at<uint16_t>(d_ws, o.dmeta);
  dp.dbase = at<int32_t>(d_ws, o.dbase);
  dp.level_fires = at<unsigned long long>(d_ws, o.level_fires);
  const bool z = p.mode == SND_MODE_ZFLOAT;
  dp.zring = z ? at<void>(d_ws, o.zring) : nullptr;
  dp.ztab = z ? at<void>(d_ws, o.ztab) : nullptr;
  dp.zwb = z ? at<int32_t>(d_ws, o.zwb) : nullptr;
  dp.zcarry = z ? at<int32_t>(d_ws, o.zcarry) : nullptr;
  std::vector<float> dmf(p.dms.begin(), p.dms.end());
  // uploads still in flight target the previous workspace
  if (p.up_stream && cudaStreamSynchronize(p.up_stream) != cudaSuccess) {
    p.bound = false;
    return SND_ERR_CUDA;
  }
  p.up_free_set[0] = p.up_free_set[1] = false;
  p.up_next = 0;
  cudaError_t e = cudaMemsetAsync(d_ws, 0, p.ws_bytes, s);
  if (e == cudaSuccess) e = upload(d_ws, o.width_mask, p.width_mask, s);
  if (e == cudaSuccess) e = upload(d_ws, o.dm_f32, dmf, s);
  if (e == cudaSuccess) e = upload(d_ws, o.tp_off, p.tp_off, s);
  if (e == cudaSuccess) e = upload(d_ws, o.gepk, p.gepk, s);
  if (e == cudaSuccess) e = upload(d_ws, o.gleaf, p.gleaf, s);
  if (e == cudaSuccess) e = upload(d_ws, o.gmeta, p.gmeta, s);
  if (e == cudaSuccess) e = upload(d_ws, o.tile_wb, p.tile_wb, s);
  if (e == cudaSuccess) e = upload(d_ws, o.delays, p.delays, s);
  if (e == cudaSuccess) e = upload(d_ws, o.dmeta, p.dmeta, s);
  if (e == cudaSuccess) e = upload(d_ws, o.dbase, p.dbase, s);
  if (e == cudaSuccess && z) e = upload(d_ws, o.zwb, p.zwb, s);
  if (e == cudaSuccess && z) e = upload(d_ws, o.zcarry, p.zcarry, s);
  if (e != cudaSuccess) {
    p.bound = false;
    return SND_ERR_CUDA;
  }
  p.ws = d_ws;
  p.ws_have = bytes;
  p.bound = true;
  p.last_stream = s;
  p.T = p.E = p.F = 0;
  p.sticky = 0;
  p.pending_host = 0;
  p.launches = 0;
  p.ev_used = 0;
  p.ev_marks.clear();
  return SND_OK;
}

extern "C" int snd_level_rates(snd_plan_t plan, uint64_t* fires_out, double* rates_out, int32_t cap,
                               int32_t* nlevels_out) {
  if (!plan || cap < 0) return SND_ERR_ARG;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (!p.bound || !(p.flags & SND_FLAG_LEVEL_RATES)) return SND_ERR_STATE;
  if (p.sticky) return p.sticky;
  if (cudaStreamSynchronize(p.last_stream) != cudaSuccess) return fail(p, SND_ERR_CUDA);
  unsigned long long f[snd::kMaxLevels];
  if (cudaMemcpy(f, p.dp.level_fires, sizeof(f), cudaMemcpyDeviceToHost) != cudaSuccess) return fail(p, SND_ERR_CUDA);
  if (nlevels_out) *nlevels_out = p.nlev;
  for (int l = 0; l < p.nlev && l < cap; ++l) {
    if (fires_out) fires_out[l] = f[l];
    const double den = static_cast<double>(p.level_nodes[l]) * p.ndm * static_cast<double>(p.E);
    if (rates_out) rates_out[l] = den > 0 ? static_cast<double>(f[l]) / den : 0.0;
  }
  return SND_OK;
}

extern "C" int snd_debug_loop_limit(snd_plan_t plan, int64_t limit, int64_t wait_cycles) {
  if (!plan || limit < 0 || wait_cycles < 0) return SND_ERR_ARG;
  reinterpret_cast<Plan*>(plan)->loop_limit = limit;
  reinterpret_cast<Plan*>(plan)->wait_limit = wait_cycles;
  return SND_OK;
}

extern "C" int snd_profile(snd_plan_t plan, int enable) {
  if (!plan) return SND_ERR_ARG;
  reinterpret_cast<Plan*>(plan)->profiling = enable != 0;
  return SND_OK;
}

extern "C" int snd_profile_read(snd_plan_t plan, double* ms_out, int64_t* count_out) {
  if (!plan) return SND_ERR_ARG;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  double ms[SND_NUM_STAGES] = {0, 0, 0, 0};
  int64_t cnt[SND_NUM_STAGES] = {0, 0, 0, 0};
  int rc = SND_OK;
  for (const auto& m : p.ev_marks) {
    float t = 0.f;
    if (cudaEventSynchronize(p.ev_pool[m.second.second]) != cudaSuccess ||
        cudaEventElapsedTime(&t, p.ev_pool[m.second.first], p.ev_pool[m.second.second]) != cudaSuccess) {
      rc = SND_ERR_CUDA;
      break;
    }
    ms[m.first] += t;
    cnt[m.first] += 1;
  }
  p.ev_marks.clear();
  p.ev_used = 0;
  for (int i = 0; i < SND_NUM_STAGES; ++i) {
    if (ms_out) ms_out[i] = ms[i];
    if (count_out) count_out[i] = cnt[i];
  }
  return rc;
}

snd::Plan::~Plan() {
  for (cudaEvent_t ev : ev_pool) cudaEventDestroy(ev);
  if (up_stream) {
    cudaStreamSynchronize(up_stream);
    cudaStreamDestroy(up_stream);
  }
  for (int b = 0; b < 2; ++b) {
    if (up_done[b]) cudaEventDestroy(up_done[b]);
    if (up_free[b]) cudaEventDestroy(up_free[b]);
  }
}

extern "C" int snd_execute(snd_plan_t plan, const uint8_t* d_chunk, int32_t nsamp, void* stream,
                           void* d_plane_out, int32_t* nemit_out) {
  if (!plan) return SND_ERR_ARG;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (p.sticky) return p.sticky;
  if (!p.bound) return SND_ERR_STATE;
  if (!d_chunk) return SND_ERR_ARG;
  if (nsamp < 1 || nsamp > p.max_chunk) return SND_ERR_CHUNK;
  return run_chunk(p, d_chunk, nsamp, static_cast<cudaStream_t>(stream), d_plane_out, nemit_out);
}

extern "C" int snd_execute_host(snd_plan_t plan, const uint8_t* h_chunk, int32_t nsamp, void* stream,
                                void* d_plane_out, int32_t* nemit_out) {
  if (!plan) return SND_ERR_ARG;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (p.sticky) return p.sticky;
  if (!p.bound) return SND_ERR_STATE;
  if (!h_chunk) return SND_ERR_ARG;
  if (nsamp < 1 || nsamp > p.max_chunk) return SND_ERR_CHUNK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = static_cast<size_t>(nsamp) * p.nchan;
  if (!p.up_stream) {
    if (cudaStreamCreateWithFlags(&p.up_stream, cudaStreamNonBlocking) != cudaSuccess) {
      p.up_stream = nullptr;
      return fail(p, SND_ERR_CUDA);
    }
    for (int b = 0; b < 2; ++b)
      if (cudaEventCreateWithFlags(&p.up_done[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&p.up_free[b], cudaEventDisableTiming) != cudaSuccess)
        return fail(p, SND_ERR_CUDA);
  }
  // buffer b was last read by the chunk before the previous one: wait for that chunk only,
  // not for the rest of `stream`, so this copy overlaps the previous chunk's kernels
  const int b = p.up_next;
  uint8_t* buf = b ? p.dp.staging2 : p.dp.staging;
  if (p.up_free_set[b] && cudaStreamWaitEvent(p.up_stream, p.up_free[b], 0) != cudaSuccess)
    return fail(p, SND_ERR_CUDA);
  if (cudaMemcpyAsync(buf, h_chunk, bytes, cudaMemcpyHostToDevice, p.up_stream) != cudaSuccess ||
      cudaEventRecord(p.up_done[b], p.up_stream) != cudaSuccess || cudaStreamWaitEvent(s, p.up_done[b], 0) != cudaSuccess)
    return fail(p, SND_ERR_CUDA);
  const int rc = run_chunk(p, buf, nsamp, s, d_plane_out, nemit_out);
  if (rc != SND_OK) return rc;
  if (cudaEventRecord(p.up_free[b], s) != cudaSuccess) return fail(p, SND_ERR_CUDA);
  p.up_free_set[b] = true;
  p.up_next = b ^ 1;
  return SND_OK;
}

extern "C" int snd_candidates(snd_plan_t plan, snd_candidate_t* host_out, int32_t cap, int32_t* n_out) {
  if (n_out) *n_out = 0;
  if (!plan || !n_out || cap < 0 || (cap > 0 && !host_out)) return SND_ERR_ARG;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (!p.bound) return SND_ERR_STATE;
  if (p.sticky) return p.sticky;
  if (cudaStreamSynchronize(p.last_stream) != cudaSuccess) return fail(p, SND_ERR_CUDA);
  uint32_t cnt[snd::kCntSlots];
  if (cudaMemcpy(cnt, p.dp.counters, sizeof(cnt), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(p, SND_ERR_CUDA);
  const int n = static_cast<int>(cnt[snd::kCntCands]);
  const int take = n < cap ? n : cap;
  if (take > 0 &&
      cudaMemcpy(host_out, p.dp.cand, sizeof(snd_candidate_t) * take, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(p, SND_ERR_CUDA);
  uint32_t zero[2] = {0, 0};
  if (cudaMemcpy(p.dp.counters + snd::kCntCands, zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(p, SND_ERR_CUDA);
  *n_out = take;
  p.pending_host = 0;
  const uint32_t st = cnt[snd::kCntStatus];
  p.last_status = st;
  if (st & (snd::kStatusTauTimeout | snd::kStatusUnionTimeout | snd::kStatusTreeTimeout | snd::kStatusGridTimeout |
            snd::kStatusMfTimeout))
    return SND_ERR_TIMEOUT;
  if (st & (snd::kStatusCellOverflow | snd::kStatusRunOverflow | snd::kStatusCandOverflow |
            snd::kStatusBlockCandOverflow | snd::kStatusBounds))
    return SND_ERR_OVERFLOW;
  if (n > cap) return SND_ERR_OVERFLOW;
  return SND_OK;
}
