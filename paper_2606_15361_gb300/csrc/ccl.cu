// Candidate detection (Methods, "Candidate detection"): threshold mask -> square binary
// closing -> 8-connected labelling -> islands of at least N_min pixels -> one candidate per
// island at its peak pixel.
//
//  * Closing (side 2r+1): dilation with outside = 0, then erosion with outside = 1, each
//    done separably (rows, then DM columns) on the bit-packed mask, 32 samples per word.
//  * Labelling works on runs of set bits of the closed mask. Runs are counted and written
//    per row (deterministic order: row-major), runs of adjacent rows that touch under
//    8-connectivity (s_j <= e_i and s_i <= e_j, ends exclusive) are united in a lock-free
//    union-find whose root is the smallest run index, and island sizes are summed per root.
//  * Peak: each original-mask cell finds its run and raises its island's 64-bit key
//    (S/N float bits << 32 | ~cell index) with atomicMax: larger S/N wins, ties go to the
//    smaller cell index = smaller DM row, then smaller t.
//  * The block's candidates are ranked by (t, DM index) and appended to the plan's list.
// Every data-dependent loop is bounded; a bound that is hit sets a status bit instead of
// spinning.

#include <vector>

#include "snd_internal.h"

namespace snd {
namespace {

constexpr int kGridStride = 152 * 4;

__global__ void k_close_h(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int mw, int nb,
                          int r, int erode) {
  const int d = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int nbw = (nb + 31) >> 5;
  if (q >= nbw) return;
  const uint32_t outside = erode ? 0xFFFFFFFFu : 0u;
  const uint32_t tailvalid = (nb & 31) ? ((1u << (nb & 31)) - 1u) : 0xFFFFFFFFu;
  auto word = [&](int qq) -> uint32_t {
    if (qq < 0 || qq >= nbw) return outside;
    uint32_t w = in[static_cast<size_t>(d) * mw + qq];
    if (qq == nbw - 1) w = erode ? (w | ~tailvalid) : (w & tailvalid);
    return w;
  };
  const uint32_t a = word(q - 1), b = word(q), c = word(q + 1);
  uint32_t acc = b;
  for (int k = 1; k <= r; ++k) {
    const uint32_t right = __funnelshift_r(b, c, k);  // bit t <- bit t+k
    const uint32_t left = __funnelshift_l(a, b, k);   // bit t <- bit t-k
    acc = erode ? (acc & right & left) : (acc | right | left);
  }
  if (q == nbw - 1) acc &= tailvalid;
  out[static_cast<size_t>(d) * mw + q] = acc;
}

__global__ void k_close_v(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int ndm, int mw,
                          int nb, int r, int erode) {
  const int d = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int nbw = (nb + 31) >> 5;
  if (q >= nbw) return;
  uint32_t acc = erode ? 0xFFFFFFFFu : 0u;
  for (int j = -r; j <= r; ++j) {
    const int dd = d + j;
    if (dd < 0 || dd >= ndm) continue;  // outside: 1 for erosion, 0 for dilation (no-ops)
    const uint32_t w = in[static_cast<size_t>(dd) * mw + q];
    acc = erode ? (acc & w) : (acc | w);
  }
  if (q == nbw - 1 && (nb & 31)) acc &= (1u << (nb & 31)) - 1u;
  out[static_cast<size_t>(d) * mw + q] = acc;
}

// The four closing passes fused: a CTA owns a tile of kCloseTR rows x kCloseTQ words and
// stages the rows and words its two dilation + erosion passes reach (2r rows and two words
// each side) in shared memory. Each pass follows k_close_h / k_close_v exactly: outside
// the plane the dilation reads 0 and the erosion 1, bits past nb are cleared after every
// pass (and read as 1 by the horizontal erosion).
constexpr int kCloseTR = 32, kCloseTQ = 32, kCloseNQ = kCloseTQ + 4, kCloseThreads = 256;

__device__ __forceinline__ void close_tile(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int ndm, int mw,
                                           int nb, int r, int bx, int by, uint32_t* csm) {
  const int NR = kCloseTR + 4 * r;
  uint32_t* A = csm;                 // [NR][kCloseNQ]: input, then the dilated tile
  uint32_t* Bv = csm + NR * kCloseNQ;  // [NR][kCloseNQ]: horizontal pass results
  const int d0 = by * kCloseTR, q0 = bx * kCloseTQ;
  const int R0 = d0 - 2 * r, W0 = q0 - 2;
  const int nbw = (nb + 31) >> 5;
  const uint32_t tailvalid = (nb & 31) ? ((1u << (nb & 31)) - 1u) : 0xFFFFFFFFu;
  const int n = NR * kCloseNQ;
  const int tid = threadIdx.x;
  uint32_t any = 0u;
  // 1. input tile, dilation's outside value 0
  for (int idx = tid; idx < n; idx += kCloseThreads) {
    const int i = idx / kCloseNQ, k = idx - i * kCloseNQ;
    const int d = R0 + i, q = W0 + k;
    uint32_t w = 0u;
    if (d >= 0 && d < ndm && q >= 0 && q < nbw) {
      w = in[static_cast<size_t>(d) * mw + q];
      if (q == nbw - 1) w &= tailvalid;
    }
    A[idx] = w;
    any |= w;
  }
  // a tile whose staged input (halo included) is empty closes to an empty tile: most tiles of
  // a block far from any detection
  if (!__syncthreads_or(any != 0u)) {
    for (int idx = tid; idx < kCloseTR * kCloseTQ; idx += kCloseThreads) {
      const int d = d0 + idx / kCloseTQ, q = q0 + idx % kCloseTQ;
      if (d < ndm && q < nbw) out[static_cast<size_t>(d) * mw + q] = 0u;
    }
    return;
  }
  // 2. horizontal dilation, words 1 .. NQ-2
  for (int idx = tid; idx < n; idx += kCloseThreads) {
    const int i = idx / kCloseNQ, k = idx - i * kCloseNQ;
    if (k < 1 || k > kCloseNQ - 2) continue;
    const uint32_t a = A[idx - 1], b = A[idx], c = A[idx + 1];
    uint32_t acc = b;
    for (int kk = 1; kk <= r; ++kk) acc |= __funnelshift_r(b, c, kk) | __funnelshift_l(a, b, kk);
    if (W0 + k == nbw - 1) acc &= tailvalid;
    Bv[idx] = acc;
  }
  __syncthreads();
  // 3. vertical dilation into A, rows r .. NR-r-1, words 1 .. NQ-2
  for (int idx = tid; idx < n; idx += kCloseThreads) {
    const int i = idx / kCloseNQ, k = idx - i * kCloseNQ;
    if (i < r || i >= NR - r || k < 1 || k > kCloseNQ - 2) continue;
    const int d = R0 + i;
    uint32_t acc = 0u;
    for (int j = -r; j <= r; ++j) {
      const int dd = d + j;
      if (dd >= 0 && dd < ndm) acc |= Bv[idx + j * kCloseNQ];
    }
    if (W0 + k == nbw - 1) acc &= tailvalid;
    A[idx] = acc;
  }
  __syncthreads();
  // 4. horizontal erosion into Bv, rows r .. NR-r-1, words 2 .. NQ-3 (outside reads 1)
  for (int idx = tid; idx < n; idx += kCloseThreads) {
    const int i = idx / kCloseNQ, k = idx - i * kCloseNQ;
    if (i < r || i >= NR - r || k < 2 || k > kCloseNQ - 3) continue;
    auto word = [&](int kk) -> uint32_t {
      const int q = W0 + kk;
      if (q < 0 || q >= nbw) return 0xFFFFFFFFu;
      uint32_t w = A[i * kCloseNQ + kk];
      if (q == nbw - 1) w |= ~tailvalid;
      return w;
    };
    const uint32_t a = word(k - 1), b = word(k), c = word(k + 1);
    uint32_t acc = b;
    for (int kk = 1; kk <= r; ++kk) acc &= __funnelshift_r(b, c, kk) & __funnelshift_l(a, b, kk);
    if (W0 + k == nbw - 1) acc &= tailvalid;
    Bv[idx] = acc;
  }
  __syncthreads();
  // 5. vertical erosion to the output tile, rows 2r .. NR-2r-1, words 2 .. NQ-3
  for (int idx = tid; idx < n; idx += kCloseThreads) {
    const int i = idx / kCloseNQ, k = idx - i * kCloseNQ;
    if (i < 2 * r || i >= NR - 2 * r || k < 2 || k > kCloseNQ - 3) continue;
    const int d = R0 + i, q = W0 + k;
    if (d >= ndm || q >= nbw) continue;
    uint32_t acc = 0xFFFFFFFFu;
    for (int j = -r; j <= r; ++j) {
      const int dd = d + j;
      if (dd >= 0 && dd < ndm) acc &= Bv[idx + j * kCloseNQ];
    }
    if (q == nbw - 1) acc &= tailvalid;
    out[static_cast<size_t>(d) * mw + q] = acc;
  }
}

__global__ void __launch_bounds__(kCloseThreads) k_close(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                         int ndm, int mw, int nb, int r) {
  extern __shared__ uint32_t csm[];
  close_tile(in, out, ndm, mw, nb, r, blockIdx.x, blockIdx.y, csm);
}

// One warp per row: number of runs (run starts) of the closed mask.
__device__ __forceinline__ void run_count_row(const uint32_t* __restrict__ m, int ndm, int mw, int nb,
                                              int32_t* row_runs, const int warp, const int lane) {
  if (warp >= ndm) return;
  const int nbw = (nb + 31) >> 5;
  const uint32_t* row = m + static_cast<size_t>(warp) * mw;
  int cnt = 0;
  for (int q0 = 0; q0 < nbw; q0 += 32) {
    const int q = q0 + lane;
    const uint32_t w = q < nbw ? row[q] : 0u;
    const uint32_t prev = q > 0 && q - 1 < nbw ? row[q - 1] : 0u;
    cnt += __popc(w & ~((w << 1) | (prev >> 31)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, o);
  if (lane == 0) row_runs[warp] = cnt;
}

__global__ void k_run_count(const uint32_t* __restrict__ m, int ndm, int mw, int nb, int32_t* row_runs) {
  run_count_row(m, ndm, mw, nb, row_runs, (blockIdx.x * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31);
}

// One CTA of NT threads: exclusive scan of the per-row run counts; total -> counters[kCntRuns].
template <int NT>
__device__ __forceinline__ void scan_rows_cta(int32_t* row_runs, int ndm, uint32_t* counters, int run_cap) {
  __shared__ int part[64];
  const int tid = threadIdx.x;
  const int per = (ndm + NT - 1) / NT;
  const int lo = min(ndm, tid * per), hi = min(ndm, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += row_runs[i];
  // exclusive scan of the 1024 partial sums: within each warp, then over the 32 warp totals
  const int lane = tid & 31, wid = tid >> 5;
  int incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) part[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int t = lane < NT / 32 ? part[lane] : 0;
    int wincl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xFFFFFFFFu, wincl, o);
      if (lane >= o) wincl += u;
    }
    part[32 + lane] = wincl - t;
    if (lane == 31) {
      row_runs[ndm] = wincl;
      counters[kCntRuns] = static_cast<uint32_t>(wincl);
      if (wincl > run_cap) atomicOr(&counters[kCntStatus], kStatusRunOverflow);
    }
  }
  __syncthreads();
  int acc = part[32 + wid] + incl - s;
  for (int i = lo; i < hi; ++i) {
    const int v = row_runs[i];
    row_runs[i] = acc;
    acc += v;
  }
}

__global__ void k_scan_rows(int32_t* row_runs, int ndm, uint32_t* counters, int run_cap) {
  scan_rows_cta<1024>(row_runs, ndm, counters, run_cap);
}

// One warp per row: write runs [start, end) in order, initialise union-find state.
__device__ __forceinline__ void run_write_row(const uint32_t* __restrict__ m, int ndm, int mw, int nb,
                                              const int32_t* row_runs, int32_t* run_start, int32_t* run_end,
                                              int32_t* run_row, int32_t* parent, int32_t* npix,
                                              unsigned long long* peak, int32_t* pwidth, int run_cap, const int warp,
                                              const int lane) {
  if (warp >= ndm) return;
  if (row_runs[ndm] > run_cap) return;
  if (row_runs[warp + 1] == row_runs[warp]) return;  // a row without runs (most rows)
  const int nbw = (nb + 31) >> 5;
  const uint32_t* row = m + static_cast<size_t>(warp) * mw;
  int base_s = row_runs[warp], base_e = row_runs[warp];
  for (int q0 = 0; q0 < nbw; q0 += 32) {
    const int q = q0 + lane;
    const uint32_t w = q < nbw ? row[q] : 0u;
    const uint32_t prev = (q > 0 && q - 1 < nbw) ? row[q - 1] : 0u;
    const uint32_t next = (q + 1 < nbw) ? row[q + 1] : 0u;
    uint32_t st = w & ~((w << 1) | (prev >> 31));
    uint32_t en = w & ~((w >> 1) | (next << 31));
    const int ns = __popc(st), ne = __popc(en);
    int is = ns, ie = ne;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int us = __shfl_up_sync(0xFFFFFFFFu, is, o);
      const int ue = __shfl_up_sync(0xFFFFFFFFu, ie, o);
      if (lane >= o) {
        is += us;
        ie += ue;
      }
    }
    int ps = base_s + is - ns, pe = base_e + ie - ne;
    while (st) {
      const int b = __ffs(st) - 1;
      st &= st - 1;
      run_start[ps] = q * 32 + b;
      run_row[ps] = warp;
      parent[ps] = ps;
      npix[ps] = 0;
      peak[ps] = 0ull;
      pwidth[ps] = 0;
      ++ps;
    }
    while (en) {
      const int b = __ffs(en) - 1;
      en &= en - 1;
      run_end[pe++] = q * 32 + b + 1;
    }
    base_s += __shfl_sync(0xFFFFFFFFu, is, 31);
    base_e += __shfl_sync(0xFFFFFFFFu, ie, 31);
  }
}

__global__ void k_run_write(const uint32_t* __restrict__ m, int ndm, int mw, int nb, const int32_t* row_runs,
                            int32_t* run_start, int32_t* run_end, int32_t* run_row, int32_t* parent,
                            int32_t* npix, unsigned long long* peak, int32_t* pwidth, int run_cap) {
  run_write_row(m, ndm, mw, nb, row_runs, run_start, run_end, run_row, parent, npix, peak, pwidth, run_cap,
                (blockIdx.x * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31);
}

__device__ __forceinline__ int find_root(const int32_t* parent, int x, uint32_t* status, int lim) {
  const volatile int32_t* vp = parent;
  for (int it = 0; it < lim; ++it) {
    const int p = vp[x];
    if (p == x) return x;
    x = p;
  }
  atomicOr(status, kStatusUnionTimeout);
  return x;
}

__device__ __forceinline__ void unite(int32_t* parent, int a, int b, uint32_t* status, int lim) {
  for (int it = 0; it < (lim < 4096 ? lim : 4096); ++it) {
    a = find_root(parent, a, status, lim);
    b = find_root(parent, b, status, lim);
    if (a == b) return;
    if (a < b) {
      const int t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(&parent[a], a, b) == a) return;
  }
  atomicOr(status, kStatusUnionTimeout);
}

__device__ __forceinline__ int runs_total(const int32_t* row_runs, int ndm, int run_cap) {
  const int n = row_runs[ndm];
  return n > run_cap ? -1 : n;
}

// The remaining stages loop over their items i = i0, i0 + stride, ... (a grid-stride loop in
// the single-plan kernels, a loop over the whole cooperative grid in the many-beam kernel).
__device__ __forceinline__ void union_items(const int32_t* row_runs, int ndm, int run_cap, const int32_t* run_start,
                                            const int32_t* run_end, const int32_t* run_row, int32_t* parent,
                                            uint32_t* counters, int lim, int i0, int stride) {
  const int n = runs_total(row_runs, ndm, run_cap);
  for (int i = i0; i < n; i += stride) {
    const int d = run_row[i];
    if (d == 0) continue;
    const int s = run_start[i], e = run_end[i];
    int lo = row_runs[d - 1], hi = row_runs[d];
    // first run of the row above with end >= s
    int a = lo, b = hi;
    while (a < b) {
      const int mid = (a + b) >> 1;
      if (run_end[mid] >= s) b = mid; else a = mid + 1;
    }
    for (int j = a; j < hi && run_start[j] <= e; ++j) unite(parent, i, j, &counters[kCntStatus], lim);
  }
}

__global__ void k_union(const int32_t* row_runs, int ndm, int run_cap, const int32_t* run_start,
                        const int32_t* run_end, const int32_t* run_row, int32_t* parent, uint32_t* counters, int lim) {
  union_items(row_runs, ndm, run_cap, run_start, run_end, run_row, parent, counters, lim,
              blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__device__ __forceinline__ void flatten_items(const int32_t* row_runs, int ndm, int run_cap, const int32_t* run_start,
                                              const int32_t* run_end, int32_t* parent, int32_t* npix,
                                              uint32_t* counters, int lim, int i0, int stride) {
  const int n = runs_total(row_runs, ndm, run_cap);
  for (int i = i0; i < n; i += stride) {
    const int r = find_root(parent, i, &counters[kCntStatus], lim);
    parent[i] = r;
    atomicAdd(&npix[r], run_end[i] - run_start[i]);
  }
}

__global__ void k_flatten(const int32_t* row_runs, int ndm, int run_cap, const int32_t* run_start,
                          const int32_t* run_end, int32_t* parent, int32_t* npix, uint32_t* counters, int lim) {
  flatten_items(row_runs, ndm, run_cap, run_start, run_end, parent, npix, counters, lim,
                blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// Run of row d that contains column t, or -1.
__device__ __forceinline__ int run_of(const int32_t* row_runs, const int32_t* run_start, const int32_t* run_end,
                                      int d, int t) {
  const int lo = row_runs[d], hi = row_runs[d + 1];
  int a = lo - 1, b = hi - 1;  // last run with start <= t lies in [a, b]; a == lo - 1: none
  while (a < b) {
    const int mid = (a + b + 1) >> 1;
    if (run_start[mid] <= t) a = mid; else b = mid - 1;
  }
  if (a < lo || run_end[a] <= t) return -1;
  return a;
}

__device__ __forceinline__ void peak_items(const MfCell* cells, uint32_t* counters, int cell_cap, int nb,
                                           const int32_t* row_runs, int ndm, int run_cap, const int32_t* run_start,
                                           const int32_t* run_end, const int32_t* parent, unsigned long long* peak,
                                           int32_t* pwidth, int pass, int i0, int stride) {
  if (runs_total(row_runs, ndm, run_cap) < 0) return;
  const int nc = min(static_cast<int>(counters[kCntCells]), cell_cap);
  for (int i = i0; i < nc; i += stride) {
    const MfCell c = cells[i];
    const int d = static_cast<int>(c.cell / static_cast<uint32_t>(nb));
    const int t = static_cast<int>(c.cell - static_cast<uint32_t>(d) * static_cast<uint32_t>(nb));
    const int run = run_of(row_runs, run_start, run_end, d, t);
    if (run < 0) {
      atomicOr(&counters[kCntStatus], kStatusBounds);
      continue;
    }
    const int root = parent[run];
    const unsigned long long key =
        (static_cast<unsigned long long>(__float_as_uint(c.snr)) << 32) | (0xFFFFFFFFull - c.cell);
    if (pass == 0) {
      atomicMax(&peak[root], key);
    } else if (peak[root] == key) {
      pwidth[root] = c.width;
    }
  }
}

__global__ void k_peak(const MfCell* cells, uint32_t* counters, int cell_cap, int nb, const int32_t* row_runs,
                       int ndm, int run_cap, const int32_t* run_start, const int32_t* run_end,
                       const int32_t* parent, unsigned long long* peak, int32_t* pwidth, int pass) {
  peak_items(cells, counters, cell_cap, nb, row_runs, ndm, run_cap, run_start, run_end, parent, peak, pwidth, pass,
             blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__device__ __forceinline__ void emit_items(const int32_t* row_runs, int ndm, int run_cap, const int32_t* parent,
                                           const int32_t* npix, const unsigned long long* peak, const int32_t* pwidth,
                                           int nb, int n_min, long long f_prev, const float* dm_f32,
                                           snd_candidate_t* bcand, int cand_cap, uint32_t* counters, int i0,
                                           int stride) {
  const int n = runs_total(row_runs, ndm, run_cap);
  for (int i = i0; i < n; i += stride) {
    if (parent[i] != i || npix[i] < n_min || peak[i] == 0ull) continue;
    const uint32_t cell = 0xFFFFFFFFu - static_cast<uint32_t>(peak[i] & 0xFFFFFFFFull);
    const int d = static_cast<int>(cell / static_cast<uint32_t>(nb));
    const int t = static_cast<int>(cell - static_cast<uint32_t>(d) * static_cast<uint32_t>(nb));
    const uint32_t idx = atomicAdd(&counters[kCntBlockCands], 1u);
    if (idx >= static_cast<uint32_t>(cand_cap)) {
      atomicOr(&counters[kCntStatus], kStatusBlockCandOverflow);
      continue;
    }
    snd_candidate_t c;
    c.dm_index = d;
    c.dm = dm_f32[d];
    c.t = f_prev + t;
    c.snr = __uint_as_float(static_cast<uint32_t>(peak[i] >> 32));
    c.width = pwidth[i];
    c.npix = npix[i];
    c.reserved = 0;
    bcand[idx] = c;
  }
}

__global__ void k_emit(const int32_t* row_runs, int ndm, int run_cap, const int32_t* parent, const int32_t* npix,
                       const unsigned long long* peak, const int32_t* pwidth, int nb, int n_min,
                       long long f_prev, const float* dm_f32, snd_candidate_t* bcand, int cand_cap,
                       uint32_t* counters) {
  emit_items(row_runs, ndm, run_cap, parent, npix, peak, pwidth, nb, n_min, f_prev, dm_f32, bcand, cand_cap, counters,
             blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// Rank every block candidate by (t, dm_index) (keys are distinct: one peak pixel per island)
// and place it after the candidates already held.
__device__ __forceinline__ void rank_items(const snd_candidate_t* bcand, snd_candidate_t* cand, uint32_t* counters,
                                           int cand_cap, int i0, int stride) {
  const int n = min(static_cast<int>(counters[kCntBlockCands]), cand_cap);
  const int base = static_cast<int>(counters[kCntCands]);
  for (int i = i0; i < n; i += stride) {
    const snd_candidate_t ci = bcand[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const snd_candidate_t cj = bcand[j];
      rank += (cj.t < ci.t) || (cj.t == ci.t && cj.dm_index < ci.dm_index);
    }
    const int pos = base + rank;
    if (pos < cand_cap) {
      cand[pos] = ci;
    } else {
      atomicOr(&counters[kCntStatus], kStatusCandOverflow);
    }
  }
}

__global__ void k_rank_append(const snd_candidate_t* bcand, snd_candidate_t* cand, uint32_t* counters,
                              int cand_cap) {
  rank_items(bcand, cand, counters, cand_cap, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__device__ __forceinline__ void bump(uint32_t* counters, int cand_cap) {
  const int n = min(static_cast<int>(counters[kCntBlockCands]), cand_cap);
  const int tot = static_cast<int>(counters[kCntCands]) + n;
  counters[kCntCands] = static_cast<uint32_t>(min(tot, cand_cap));
}

__global__ void k_bump(uint32_t* counters, int cand_cap) { bump(counters, cand_cap); }

// ---------------------------------------------------------------------------------------
// Candidate stage of many plans in ONE cooperative launch: the stages above run one after
// another over all beams' blocks, separated by grid-wide barriers (every CTA is resident, as a
// cooperative launch guarantees). Each barrier is a counter + generation pair in device
// memory; its wait is bounded, and a wait that runs out marks every beam's status word and
// ends the kernel.
// ---------------------------------------------------------------------------------------
constexpr int kMaxCandBeams = 64;
constexpr long long kGridWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

struct CandBeam {
  const uint32_t* mask;
  uint32_t* mask3;
  int ndm, mw, nb, r, run_cap, cell_cap, cand_cap, n_min, lim;
  int32_t *row_runs, *run_start, *run_end, *run_row, *parent, *npix, *pwidth;
  unsigned long long* peak;
  const MfCell* cells;
  long long f_prev;
  const float* dm_f32;
  snd_candidate_t *bcand, *cand;
  uint32_t* counters;
};

struct CandMulti {
  int nbeams;
  int first_close[kMaxCandBeams];  // closing tiles of the beams before
  int first_rows[kMaxCandBeams];   // 8-row groups of the beams before
  int total_close, total_rows;
  unsigned int* gbar;              // [2]: arrivals, generation
  long long wait_cycles;           // bound of a barrier wait (clock cycles)
  CandBeam beam[kMaxCandBeams];
};

__device__ __forceinline__ int cbeam_of(const int* first, int n, int i) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ bool grid_barrier(const CandMulti& m) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = m.gbar + 1;
    const unsigned int g = *gen;
    __threadfence();
    if (atomicAdd(m.gbar, 1u) == gridDim.x - 1) {
      m.gbar[0] = 0;
      __threadfence();
      atomicAdd(m.gbar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > m.wait_cycles) {
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (!ok)
      for (int b = 0; b < m.nbeams; ++b) atomicOr(&m.beam[b].counters[kCntStatus], kStatusGridTimeout);
  }
  return __syncthreads_and(ok) != 0;
}

__global__ void __launch_bounds__(256) k_cand_multi(const __grid_constant__ CandMulti m) {
  extern __shared__ uint32_t csm[];
  const int nblk = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int gtid = bid * 256 + tid, gthreads = nblk * 256;
  // 1. closing (a plain copy for a 1 x 1 element)
  for (int v = bid; v < m.total_close; v += nblk) {
    const int b = cbeam_of(m.first_close, m.nbeams, v);
    const CandBeam& e = m.beam[b];
    const int local = v - m.first_close[b];
    const int nbw = (e.nb + 31) >> 5;
    const int tx = (nbw + kCloseTQ - 1) / kCloseTQ;
    const int bx = local % tx, by = local / tx;
    if (e.r > 0) {
      close_tile(e.mask, e.mask3, e.ndm, e.mw, e.nb, e.r, bx, by, csm);
    } else {
      for (int k = tid; k < kCloseTR * kCloseTQ; k += 256) {
        const int d = by * kCloseTR + k / kCloseTQ, q = bx * kCloseTQ + k % kCloseTQ;
        if (d < e.ndm && q < nbw) e.mask3[static_cast<size_t>(d) * e.mw + q] = e.mask[static_cast<size_t>(d) * e.mw + q];
      }
    }
    __syncthreads();
  }
  if (!grid_barrier(m)) return;
  // 2. runs per row
  for (int v = bid; v < m.total_rows; v += nblk) {
    const int b = cbeam_of(m.first_rows, m.nbeams, v);
    const CandBeam& e = m.beam[b];
    run_count_row(e.mask3, e.ndm, e.mw, e.nb, e.row_runs, (v - m.first_rows[b]) * 8 + warp, lane);
  }
  if (!grid_barrier(m)) return;
  // 3. scan of the run counts, one CTA per beam
  for (int b = bid; b < m.nbeams; b += nblk) {
    const CandBeam& e = m.beam[b];
    scan_rows_cta<256>(e.row_runs, e.ndm, e.counters, e.run_cap);
    __syncthreads();
  }
  if (!grid_barrier(m)) return;
  // 4. runs and union-find state
  for (int v = bid; v < m.total_rows; v += nblk) {
    const int b = cbeam_of(m.first_rows, m.nbeams, v);
    const CandBeam& e = m.beam[b];
    run_write_row(e.mask3, e.ndm, e.mw, e.nb, e.row_runs, e.run_start, e.run_end, e.run_row, e.parent, e.npix,
                  e.peak, e.pwidth, e.run_cap, (v - m.first_rows[b]) * 8 + warp, lane);
  }
  if (!grid_barrier(m)) return;
  // 5. - 10. over each beam's runs, cells and block candidates
  for (int b = 0; b < m.nbeams; ++b) {
    const CandBeam& e = m.beam[b];
    union_items(e.row_runs, e.ndm, e.run_cap, e.run_start, e.run_end, e.run_row, e.parent, e.counters, e.lim, gtid,
                gthreads);
  }
  if (!grid_barrier(m)) return;
  for (int b = 0; b < m.nbeams; ++b) {
    const CandBeam& e = m.beam[b];
    flatten_items(e.row_runs, e.ndm, e.run_cap, e.run_start, e.run_end, e.parent, e.npix, e.counters, e.lim, gtid,
                  gthreads);
  }
  if (!grid_barrier(m)) return;
  for (int pass = 0; pass < 2; ++pass) {
    for (int b = 0; b < m.nbeams; ++b) {
      const CandBeam& e = m.beam[b];
      peak_items(e.cells, e.counters, e.cell_cap, e.nb, e.row_runs, e.ndm, e.run_cap, e.run_start, e.run_end,
                 e.parent, e.peak, e.pwidth, pass, gtid, gthreads);
    }
    if (!grid_barrier(m)) return;
  }
  for (int b = 0; b < m.nbeams; ++b) {
    const CandBeam& e = m.beam[b];
    emit_items(e.row_runs, e.ndm, e.run_cap, e.parent, e.npix, e.peak, e.pwidth, e.nb, e.n_min, e.f_prev, e.dm_f32,
               e.bcand, e.cand_cap, e.counters, gtid, gthreads);
  }
  if (!grid_barrier(m)) return;
  for (int b = 0; b < m.nbeams; ++b) {
    const CandBeam& e = m.beam[b];
    rank_items(e.bcand, e.cand, e.counters, e.cand_cap, gtid, gthreads);
  }
  if (!grid_barrier(m)) return;
  for (int b = gtid; b < m.nbeams; b += gthreads) bump(m.beam[b].counters, m.beam[b].cand_cap);
}

// iteration bound of a union-find root walk (the plan's test limit, if set)
int union_limit(const Plan& p) {
  return p.loop_limit > 0 ? static_cast<int>(p.loop_limit < (1 << 20) ? p.loop_limit : (1 << 20)) : (1 << 20);
}

}  // namespace

cudaError_t launch_candidates(const Plan& p, int64_t f_prev, int nb, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  if (!(p.flags & kFlagReferenceTree)) {
    // one cooperative launch instead of the eleven stage launches below
    ChunkPos c{};
    c.f_prev = f_prev;
    c.nb = nb;
    const Plan* pp = &p;
    return launch_candidates_batch(&pp, &c, 1, s);
  }
  // the reference tree's plans: the closing as separate passes and one launch per stage
  const DevPtrs& dp = p.dp;
  const int r = p.closing / 2;
  const int nbw = (nb + 31) / 32;
  dim3 blk(128), grd((nbw + 127) / 128, p.ndm);
  if (r > 0 && (p.flags & kFlagReferenceTree)) {
    // reference path: the four separable passes as separate launches
    p.launches += 4;
    k_close_h<<<grd, blk, 0, s>>>(dp.mask, dp.mask2, p.mw, nb, r, 0);
    k_close_v<<<grd, blk, 0, s>>>(dp.mask2, dp.mask3, p.ndm, p.mw, nb, r, 0);
    k_close_h<<<grd, blk, 0, s>>>(dp.mask3, dp.mask2, p.mw, nb, r, 1);
    k_close_v<<<grd, blk, 0, s>>>(dp.mask2, dp.mask3, p.ndm, p.mw, nb, r, 1);
  } else if (r > 0) {
    p.launches += 1;
    const int smem = 2 * (kCloseTR + 4 * r) * kCloseNQ * static_cast<int>(sizeof(uint32_t));
    dim3 cg((nbw + kCloseTQ - 1) / kCloseTQ, (p.ndm + kCloseTR - 1) / kCloseTR);
    k_close<<<cg, kCloseThreads, smem, s>>>(dp.mask, dp.mask3, p.ndm, p.mw, nb, r);
  } else {
    cudaMemcpyAsync(dp.mask3, dp.mask, sizeof(uint32_t) * static_cast<size_t>(p.ndm) * p.mw,
                    cudaMemcpyDeviceToDevice, s);
  }
  const int wblocks = (p.ndm * 32 + 255) / 256;
  k_run_count<<<wblocks, 256, 0, s>>>(dp.mask3, p.ndm, p.mw, nb, dp.row_runs);
  k_scan_rows<<<1, 1024, 0, s>>>(dp.row_runs, p.ndm, dp.counters, p.run_cap);
  k_run_write<<<wblocks, 256, 0, s>>>(dp.mask3, p.ndm, p.mw, nb, dp.row_runs, dp.run_start, dp.run_end,
                                      dp.run_row, dp.parent, dp.npix, dp.peak, dp.pwidth, p.run_cap);
  const int lim = union_limit(p);
  k_union<<<kGridStride, 256, 0, s>>>(dp.row_runs, p.ndm, p.run_cap, dp.run_start, dp.run_end, dp.run_row,
                                      dp.parent, dp.counters, lim);
  k_flatten<<<kGridStride, 256, 0, s>>>(dp.row_runs, p.ndm, p.run_cap, dp.run_start, dp.run_end, dp.parent,
                                        dp.npix, dp.counters, lim);
  k_peak<<<kGridStride, 256, 0, s>>>(dp.cells, dp.counters, p.cell_cap, nb, dp.row_runs, p.ndm, p.run_cap,
                                     dp.run_start, dp.run_end, dp.parent, dp.peak, dp.pwidth, 0);
  k_peak<<<kGridStride, 256, 0, s>>>(dp.cells, dp.counters, p.cell_cap, nb, dp.row_runs, p.ndm, p.run_cap,
                                     dp.run_start, dp.run_end, dp.parent, dp.peak, dp.pwidth, 1);
  k_emit<<<kGridStride, 256, 0, s>>>(dp.row_runs, p.ndm, p.run_cap, dp.parent, dp.npix, dp.peak, dp.pwidth, nb,
                                     p.n_min, f_prev, dp.dm_f32, dp.bcand, p.cand_cap, dp.counters);
  k_rank_append<<<kGridStride, 256, 0, s>>>(dp.bcand, dp.cand, dp.counters, p.cand_cap);
  k_bump<<<1, 1, 0, s>>>(dp.counters, p.cand_cap);
  p.launches += 11;
  return cudaGetLastError();
}

// The candidate stages of several plans' blocks in one cooperative launch (plans on the
// reference closing path keep their own launches). The grid barrier's two words are slots
// kCntGridBar.. of the first plan's counters; the arrival count is cleared before the launch.
cudaError_t launch_candidates_batch(const Plan* const* plans, const ChunkPos* pos, int n, cudaStream_t s) {
  std::vector<int> batch;
  for (int i = 0; i < n; ++i) {
    if (pos[i].nb <= 0) continue;
    if (plans[i]->flags & kFlagReferenceTree) {
      const cudaError_t e = launch_candidates(*plans[i], pos[i].f_prev, pos[i].nb, s);
      if (e != cudaSuccess) return e;
    } else {
      batch.push_back(i);
    }
  }
  for (size_t i0 = 0; i0 < batch.size(); i0 += kMaxCandBeams) {
    CandMulti m{};
    int rmax = 0;
    for (size_t k = i0; k < batch.size() && m.nbeams < kMaxCandBeams; ++k) {
      const Plan& p = *plans[batch[k]];
      const ChunkPos& c = pos[batch[k]];
      const DevPtrs& dp = p.dp;
      CandBeam& e = m.beam[m.nbeams];
      e.mask = dp.mask;
      e.mask3 = dp.mask3;
      e.ndm = p.ndm;
      e.mw = p.mw;
      e.nb = c.nb;
      e.r = p.closing / 2;
      e.run_cap = p.run_cap;
      e.cell_cap = p.cell_cap;
      e.cand_cap = p.cand_cap;
      e.n_min = p.n_min;
      e.lim = union_limit(p);
      e.row_runs = dp.row_runs;
      e.run_start = dp.run_start;
      e.run_end = dp.run_end;
      e.run_row = dp.run_row;
      e.parent = dp.parent;
      e.npix = dp.npix;
      e.pwidth = dp.pwidth;
      e.peak = dp.peak;
      e.cells = dp.cells;
      e.f_prev = c.f_prev;
      e.dm_f32 = dp.dm_f32;
      e.bcand = dp.bcand;
      e.cand = dp.cand;
      e.counters = dp.counters;
      const int nbw = (c.nb + 31) / 32;
      m.first_close[m.nbeams] = m.total_close;
      m.first_rows[m.nbeams] = m.total_rows;
      m.total_close += ((nbw + kCloseTQ - 1) / kCloseTQ) * ((p.ndm + kCloseTR - 1) / kCloseTR);
      m.total_rows += (p.ndm + 7) / 8;
      rmax = rmax > e.r ? rmax : e.r;
      ++m.nbeams;
    }
    const Plan& owner = *plans[batch[i0]];
    m.gbar = owner.dp.counters + kCntGridBar;
    m.wait_cycles = owner.wait_limit > 0 ? owner.wait_limit : kGridWaitCycles;
    const int smem = 2 * (kCloseTR + 4 * rmax) * kCloseNQ * static_cast<int>(sizeof(uint32_t));
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cand_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cand_multi, 256, smem);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) e = cudaMemsetAsync(m.gbar, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    // one CTA per SM at most 2: the stages are latency bound, and fewer CTAs make cheaper barriers
    const int grid = nsm * (per_sm < 2 ? per_sm : 2);
    void* args[] = {&m};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_cand_multi), dim3(grid), dim3(256), args,
                                    static_cast<size_t>(smem), s);
    owner.launches += 1;
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace snd
