// Multi-rate bands with cross-band candidate merging (Methods, "Multi-rate extension";
// Eq. scrunch).
//
// Every trial DM d runs at scrunch S(d) = the largest power of two with
// S*dt <= tau_smear(d) = K_DM d df / f_c^3 (Eq. scrunch as printed; df = channel spacing,
// f_c = band centre). DMs with one S form a band, run by an ordinary plan on the band's DM
// subset at sample interval S*dt, fed with the chunk averaged over S samples (round half
// up, so the band keeps the uint8 encoder). Candidates of all bands are mapped to native
// time (t_S * S) and the global DM index and merged by single linkage: two candidates
// join when |dDM| <= 20 pc cm^-3 and |dt| <= 200 ms; each cluster keeps its largest S/N
// (ties: smaller DM index, then smaller time). The merged list is sorted by (t, DM index).

#include <algorithm>
#include <cmath>
#include <functional>
#include <cstring>
#include <new>
#include <vector>

#include "snd_internal.h"

using snd::Plan;

namespace {

constexpr double kKdm = 4.148808e3;
constexpr double kMergeDm = 20.0;      // pc cm^-3
constexpr double kMergeSeconds = 0.2;  // 200 ms

struct Band {
  int S = 1;
  snd_plan_t plan = nullptr;
  std::vector<int32_t> gidx;  // global DM index of each band row
  size_t off_ws = 0, off_staging = 0, off_map = 0;
};

struct MultiRate {
  int nchan = 0, ndm = 0, s_max = 1, max_chunk = 0, cap = 0;
  double dt = 0;
  std::vector<double> dms;
  std::vector<Band> bands;
  size_t ws_bytes = 0;
  size_t off_all = 0, off_parent = 0, off_best = 0, off_tie = 0, off_out = 0, off_cnt = 0, off_dm = 0, off_native = 0;
  void* ws = nullptr;
  bool bound = false;
  bool graph = false;
  snd::GraphRunner runner;
  cudaStream_t last_stream = nullptr;
  int sticky = 0;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// scrunched[r][c] = (sum_{i<S} chunk[r*S+i][c] + S/2) / S
__global__ void k_scrunch(const uint8_t* __restrict__ in, int nout, int nchan, int S, uint8_t* __restrict__ out) {
  const size_t total = static_cast<size_t>(nout) * nchan;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t r = i / nchan, c = i - r * nchan;
    const uint8_t* src = in + r * S * nchan + c;
    int s = 0;
    for (int k = 0; k < S; ++k) s += src[static_cast<size_t>(k) * nchan];
    out[i] = static_cast<uint8_t>((s + S / 2) / S);
  }
}

// Append one band's candidates in native units (time * S, width * S, global DM index).
__global__ void k_gather(const snd_candidate_t* __restrict__ band, const uint32_t* __restrict__ band_counters,
                         int band_cap, const int32_t* __restrict__ gidx, int S, snd_candidate_t* __restrict__ all,
                         uint32_t* __restrict__ count, int cap, uint32_t* __restrict__ status,
                         uint32_t* __restrict__ band_status) {
  const int n = min(static_cast<int>(band_counters[snd::kCntCands]), band_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(band_status, band_counters[snd::kCntStatus]);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    snd_candidate_t c = band[i];
    c.dm_index = gidx[c.dm_index];
    c.t *= S;
    c.width *= S;
    const uint32_t at = atomicAdd(count, 1u);
    if (at < static_cast<uint32_t>(cap)) {
      all[at] = c;
    } else {
      atomicOr(status, snd::kStatusCandOverflow);
    }
  }
}

__device__ int mr_find(int* parent, int x) {
  for (int it = 0; it < (1 << 20); ++it) {
    const int p = reinterpret_cast<volatile int*>(parent)[x];
    if (p == x) return x;
    x = p;
  }
  return x;
}

// All-pairs linking (the lists are short): candidate i joins every later j with
// |t_j - t_i| <= tw and |DM_j - DM_i| <= 20, by lock-free union towards the smaller index.
__global__ void k_link(const snd_candidate_t* __restrict__ all, const uint32_t* __restrict__ count, int cap,
                       const double* __restrict__ dm, double tw, int* parent, uint32_t* status) {
  const int n = min(static_cast<int>(*count), cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const snd_candidate_t ci = all[i];
    for (int j = i + 1; j < n; ++j) {
      const snd_candidate_t cj = all[j];
      const double dtm = fabs(static_cast<double>(cj.t - ci.t));
      const double ddm = fabs(dm[cj.dm_index] - dm[ci.dm_index]);
      if (dtm > tw || ddm > kMergeDm) continue;
      int a = i, b = j;
      for (int it = 0; it < 4096; ++it) {
        a = mr_find(parent, a);
        b = mr_find(parent, b);
        if (a == b) break;
        if (a < b) {
          const int t = a;
          a = b;
          b = t;
        }
        if (atomicCAS(&parent[a], a, b) == a) break;
        if (it == 4095) atomicOr(status, snd::kStatusUnionTimeout);
      }
    }
  }
}

// float -> unsigned int with the same order (any sign)
__device__ __forceinline__ unsigned int snr_key(float x) {
  const unsigned int u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ unsigned long long pos_key(const snd_candidate_t& c) {
  return (static_cast<unsigned long long>(c.dm_index) << 44) | (static_cast<unsigned long long>(c.t) & ((1ull << 44) - 1));
}

__global__ void k_init_parent(int* parent, const uint32_t* count, int cap, unsigned int* best,
                              unsigned long long* tie) {
  const int n = min(static_cast<int>(*count), cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    parent[i] = i;
    best[i] = 0u;
    tie[i] = ~0ull;
  }
}

// pass 0: largest S/N per cluster; pass 1: among those, smallest (DM index, t)
__global__ void k_best(const snd_candidate_t* __restrict__ all, const uint32_t* __restrict__ count, int cap,
                       int* parent, unsigned int* best, unsigned long long* tie, int pass) {
  const int n = min(static_cast<int>(*count), cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int r = mr_find(parent, i);
    const unsigned int s = snr_key(all[i].snr);
    if (pass == 0) {
      atomicMax(&best[r], s);
    } else if (best[r] == s) {
      atomicMin(&tie[r], pos_key(all[i]));
    }
  }
}

// representatives, ranked by (t, DM index) directly into the output
__global__ void k_emit_sorted(const snd_candidate_t* __restrict__ all, const uint32_t* __restrict__ count, int cap,
                              int* parent, const unsigned int* best, const unsigned long long* tie,
                              snd_candidate_t* __restrict__ out, uint32_t* __restrict__ nout) {
  const int n = min(static_cast<int>(*count), cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int r = mr_find(parent, i);
    const snd_candidate_t c = all[i];
    if (best[r] != snr_key(c.snr) || tie[r] != pos_key(c)) continue;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const int rj = mr_find(parent, j);
      const snd_candidate_t cj = all[j];
      if (best[rj] != snr_key(cj.snr) || tie[rj] != pos_key(cj)) continue;
      rank += (cj.t < c.t) || (cj.t == c.t && cj.dm_index < c.dm_index);
    }
    out[rank] = c;
    atomicAdd(nout, 1u);
  }
}

int fail(MultiRate& m, int code) {
  if (!m.sticky) m.sticky = code;
  return code;
}

}  // namespace

extern "C" int snd_multirate_plan(const double* freqs_mhz, int32_t nchan, double dt_s, const double* dm_grid,
                                  int32_t ndm, int32_t branching, snd_mode_t mode, const snd_options_t* opts,
                                  int32_t s_max, snd_multirate_t* out) {
  if (out) *out = nullptr;
  if (!out || !freqs_mhz || !dm_grid || nchan < 2 || ndm < 1 || !(dt_s > 0.0) || s_max < 1 ||
      (s_max & (s_max - 1)) != 0 || s_max > 1024)
    return SND_ERR_ARG;
  snd_options_t o;
  if (opts) {
    o = *opts;
  } else {
    int rc = snd_options_init(mode, &o);
    if (rc) return rc;
  }
  MultiRate* m = nullptr;
  try {
    snd::alloc_point();
    m = new MultiRate();
  } catch (const std::bad_alloc&) {
    return SND_ERR_NOMEM;
  }
  try {
  m->nchan = nchan;
  m->ndm = ndm;
  m->dt = dt_s;
  m->dms.assign(dm_grid, dm_grid + ndm);
  double fmin = freqs_mhz[0], fmax = freqs_mhz[0];
  for (int c = 1; c < nchan; ++c) {
    fmin = std::min(fmin, freqs_mhz[c]);
    fmax = std::max(fmax, freqs_mhz[c]);
  }
  const double df = std::fabs(freqs_mhz[1] - freqs_mhz[0]);
  const double fc = 0.5 * (fmax + fmin);
  std::vector<int> S(ndm, 1);
  int smax_used = 1;
  for (int i = 0; i < ndm; ++i) {
    if (!std::isfinite(dm_grid[i]) || dm_grid[i] < 0.0) {
      delete m;
      return SND_ERR_DM;
    }
    const double tau = ((kKdm * dm_grid[i]) * df) / (fc * fc * fc);
    int s = 1;
    while (s * 2 <= s_max && static_cast<double>(s * 2) * dt_s <= tau) s *= 2;
    S[i] = s;
    smax_used = std::max(smax_used, s);
  }
  m->s_max = smax_used;
  if (o.max_chunk % smax_used != 0) {
    delete m;
    return SND_ERR_ARG;
  }
  m->max_chunk = o.max_chunk;
  for (int s = 1; s <= smax_used; s *= 2) {
    Band b;
    b.S = s;
    std::vector<double> sub;
    for (int i = 0; i < ndm; ++i)
      if (S[i] == s) {
        b.gidx.push_back(i);
        sub.push_back(dm_grid[i]);
      }
    if (sub.empty()) continue;
    snd_options_t ob = o;
    ob.max_chunk = o.max_chunk / s;
    const int rc = snd_plan_ex(freqs_mhz, nchan, dt_s * s, sub.data(), static_cast<int32_t>(sub.size()), branching,
                               mode, &ob, &b.plan);
    if (rc) {
      for (auto& x : m->bands) snd_destroy(x.plan);
      delete m;
      return rc;
    }
    m->bands.push_back(std::move(b));
  }
  // workspace: per band its plan's workspace, scrunch staging and DM map; then merge buffers
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes, 256);
    return at;
  };
  int cap_total = 0;
  for (auto& b : m->bands) {
    b.off_ws = take(snd_workspace_size(b.plan));
    b.off_staging = take(static_cast<size_t>(o.max_chunk / b.S) * nchan);
    b.off_map = take(sizeof(int32_t) * b.gidx.size());
    cap_total += o.cand_capacity;
  }
  m->cap = cap_total;
  m->off_all = take(sizeof(snd_candidate_t) * cap_total);
  m->off_parent = take(sizeof(int32_t) * cap_total);
  m->off_best = take(sizeof(uint32_t) * cap_total);
  m->off_tie = take(sizeof(unsigned long long) * cap_total);
  m->off_out = take(sizeof(snd_candidate_t) * cap_total);
  m->off_cnt = take(sizeof(uint32_t) * 4);
  m->off_dm = take(sizeof(double) * ndm);
  m->off_native = take(static_cast<size_t>(o.max_chunk) * nchan);
  m->ws_bytes = off;
  snd::alloc_point();  // the band tables are complete
  } catch (const std::bad_alloc&) {
    for (auto& x : m->bands) snd_destroy(x.plan);
    delete m;
    return SND_ERR_NOMEM;
  }
  *out = reinterpret_cast<snd_multirate_t>(m);
  return SND_OK;
}

extern "C" int snd_multirate_info(snd_multirate_t h, int32_t* nbands, int32_t* scrunch, int32_t* band_ndm, int32_t cap) {
  if (!h || !nbands) return SND_ERR_ARG;
  const MultiRate& m = *reinterpret_cast<MultiRate*>(h);
  *nbands = static_cast<int32_t>(m.bands.size());
  for (int i = 0; i < static_cast<int>(m.bands.size()) && i < cap; ++i) {
    if (scrunch) scrunch[i] = m.bands[i].S;
    if (band_ndm) band_ndm[i] = static_cast<int32_t>(m.bands[i].gidx.size());
  }
  return SND_OK;
}

extern "C" size_t snd_multirate_workspace_size(snd_multirate_t h) {
  return h ? reinterpret_cast<MultiRate*>(h)->ws_bytes : 0;
}

extern "C" int snd_multirate_bind_workspace(snd_multirate_t h, void* d_ws, size_t bytes, void* stream) {
  if (!h) return SND_ERR_ARG;
  MultiRate& m = *reinterpret_cast<MultiRate*>(h);
  if (!d_ws || bytes < m.ws_bytes || (reinterpret_cast<uintptr_t>(d_ws) & 255u)) return SND_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(d_ws);
  for (auto& b : m.bands) {
    const int rc = snd_bind_workspace(b.plan, base + b.off_ws, snd_workspace_size(b.plan), stream);
    if (rc) return rc;
    if (cudaMemcpyAsync(base + b.off_map, b.gidx.data(), sizeof(int32_t) * b.gidx.size(), cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
      return SND_ERR_CUDA;
  }
  if (cudaMemcpyAsync(base + m.off_dm, m.dms.data(), sizeof(double) * m.dms.size(), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemsetAsync(base + m.off_cnt, 0, sizeof(uint32_t) * 4, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)  // pageable uploads: finish before returning
    return SND_ERR_CUDA;
  m.ws = d_ws;
  m.bound = true;
  m.last_stream = s;
  m.sticky = 0;
  return SND_OK;
}

namespace {

// scrunch the chunk for every band with S > 1, then one step of all band plans (their trees
// grouped into shared launches), enqueued on s
int enqueue_bands(MultiRate& m, const uint8_t* d_chunk, int32_t nsamp, cudaStream_t s, cudaStream_t owner) {
  char* base = static_cast<char*>(m.ws);
  std::vector<Plan*> plans;
  std::vector<const uint8_t*> src;
  std::vector<int32_t> ns;
  for (auto& b : m.bands) {
    const uint8_t* in = d_chunk;
    if (b.S > 1) {
      uint8_t* st = reinterpret_cast<uint8_t*>(base + b.off_staging);
      const int nout = nsamp / b.S;
      const size_t total = static_cast<size_t>(nout) * m.nchan;
      const int blocks = static_cast<int>(std::min<size_t>((total + 255) / 256, 152 * 16));
      k_scrunch<<<blocks, 256, 0, s>>>(d_chunk, nout, m.nchan, b.S, st);
      if (cudaGetLastError() != cudaSuccess) return SND_ERR_CUDA;
      in = st;
    }
    Plan& p = *reinterpret_cast<Plan*>(b.plan);
    if (p.sticky) return p.sticky;
    plans.push_back(&p);
    src.push_back(in);
    ns.push_back(nsamp / b.S);
  }
  return snd::enqueue_plans(plans.data(), static_cast<int>(plans.size()), src.data(), ns.data(), s, owner);
}

int run_bands(MultiRate& m, const uint8_t* d_chunk, int32_t nsamp, cudaStream_t s) {
  const int rc = m.graph ? m.runner.run(s, [&](cudaStream_t cs) { return enqueue_bands(m, d_chunk, nsamp, cs, s); })
                         : enqueue_bands(m, d_chunk, nsamp, s, s);
  if (rc) return fail(m, rc);
  m.last_stream = s;
  return SND_OK;
}

int check_chunk(MultiRate& m, const void* chunk, int32_t nsamp) {
  if (m.sticky) return m.sticky;
  if (!m.bound) return SND_ERR_STATE;
  if (!chunk) return SND_ERR_ARG;
  if (nsamp < 1 || nsamp > m.max_chunk || nsamp % m.s_max) return SND_ERR_CHUNK;
  return SND_OK;
}

}  // namespace

extern "C" int snd_multirate_execute(snd_multirate_t h, const uint8_t* d_chunk, int32_t nsamp, void* stream) {
  if (!h) return SND_ERR_ARG;
  MultiRate& m = *reinterpret_cast<MultiRate*>(h);
  const int rc = check_chunk(m, d_chunk, nsamp);
  if (rc) return rc;
  return run_bands(m, d_chunk, nsamp, static_cast<cudaStream_t>(stream));
}

extern "C" int snd_multirate_execute_host(snd_multirate_t h, const uint8_t* h_chunk, int32_t nsamp, void* stream) {
  if (!h) return SND_ERR_ARG;
  MultiRate& m = *reinterpret_cast<MultiRate*>(h);
  const int rc = check_chunk(m, h_chunk, nsamp);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t* native = reinterpret_cast<uint8_t*>(static_cast<char*>(m.ws) + m.off_native);
  if (cudaMemcpyAsync(native, h_chunk, static_cast<size_t>(nsamp) * m.nchan, cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return fail(m, SND_ERR_CUDA);
  return run_bands(m, native, nsamp, s);
}

extern "C" int snd_multirate_set_graph(snd_multirate_t h, int32_t enable) {
  if (!h) return SND_ERR_ARG;
  reinterpret_cast<MultiRate*>(h)->graph = enable != 0;
  return SND_OK;
}

extern "C" int snd_multirate_band_plan(snd_multirate_t h, int32_t band, snd_plan_t* out) {
  if (out) *out = nullptr;
  if (!h || !out) return SND_ERR_ARG;
  MultiRate& m = *reinterpret_cast<MultiRate*>(h);
  if (band < 0 || band >= static_cast<int>(m.bands.size())) return SND_ERR_ARG;
  *out = m.bands[band].plan;
  return SND_OK;
}

extern "C" int snd_multirate_candidates(snd_multirate_t h, snd_candidate_t* host_out, int32_t cap, int32_t* n_out) {
  if (n_out) *n_out = 0;
  if (!h || !n_out || cap < 0 || (cap > 0 && !host_out)) return SND_ERR_ARG;
  MultiRate& m = *reinterpret_cast<MultiRate*>(h);
  if (!m.bound) return SND_ERR_STATE;
  if (m.sticky) return m.sticky;
  cudaStream_t s = m.last_stream;
  char* base = static_cast<char*>(m.ws);
  auto* all = reinterpret_cast<snd_candidate_t*>(base + m.off_all);
  auto* parent = reinterpret_cast<int*>(base + m.off_parent);
  auto* best = reinterpret_cast<unsigned int*>(base + m.off_best);
  auto* tie = reinterpret_cast<unsigned long long*>(base + m.off_tie);
  auto* outd = reinterpret_cast<snd_candidate_t*>(base + m.off_out);
  auto* cnt = reinterpret_cast<uint32_t*>(base + m.off_cnt);  // gathered, merged, merge status, band status
  const double* dm = reinterpret_cast<const double*>(base + m.off_dm);
  if (cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * 4, s) != cudaSuccess) return fail(m, SND_ERR_CUDA);
  for (auto& b : m.bands) {
    const Plan& p = *reinterpret_cast<Plan*>(b.plan);
    k_gather<<<64, 256, 0, s>>>(p.dp.cand, p.dp.counters, p.cand_cap, reinterpret_cast<int32_t*>(base + b.off_map),
                                b.S, all, cnt, m.cap, cnt + 2, cnt + 3);
    // the band list and its status word start afresh (kCntCands, kCntStatus are adjacent)
    if (cudaMemsetAsync(p.dp.counters + snd::kCntCands, 0, sizeof(uint32_t) * 2, s) != cudaSuccess)
      return fail(m, SND_ERR_CUDA);
  }
  const double tw = kMergeSeconds / m.dt;
  k_init_parent<<<64, 256, 0, s>>>(parent, cnt, m.cap, best, tie);
  k_link<<<64, 256, 0, s>>>(all, cnt, m.cap, dm, tw, parent, cnt + 2);
  k_best<<<64, 256, 0, s>>>(all, cnt, m.cap, parent, best, tie, 0);
  k_best<<<64, 256, 0, s>>>(all, cnt, m.cap, parent, best, tie, 1);
  k_emit_sorted<<<64, 256, 0, s>>>(all, cnt, m.cap, parent, best, tie, outd, cnt + 1);
  if (cudaGetLastError() != cudaSuccess) return fail(m, SND_ERR_CUDA);
  uint32_t hc[4];
  if (cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(m, SND_ERR_CUDA);
  const int n = static_cast<int>(hc[1]);
  const int take = std::min(n, cap);
  if (take > 0 && cudaMemcpy(host_out, outd, sizeof(snd_candidate_t) * take, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(m, SND_ERR_CUDA);
  *n_out = take;
  const uint32_t st = hc[2] | hc[3];
  if (st & (snd::kStatusTauTimeout | snd::kStatusUnionTimeout)) return SND_ERR_TIMEOUT;
  if (st & (snd::kStatusCellOverflow | snd::kStatusRunOverflow | snd::kStatusCandOverflow |
            snd::kStatusBlockCandOverflow | snd::kStatusBounds))
    return SND_ERR_OVERFLOW;
  return n > cap ? SND_ERR_OVERFLOW : SND_OK;
}

extern "C" void snd_multirate_destroy(snd_multirate_t h) {
  if (!h) return;
  MultiRate* m = reinterpret_cast<MultiRate*>(h);
  for (auto& b : m->bands) snd_destroy(b.plan);
  delete m;
}
