// DM-scaled boxcar matched filter (Methods, "Matched filtering").
//
// One CTA per DM row. The row segment [F_prev, E_new) of the plane ring (block start times
// [F_prev, F_new) plus the Wmax-1 samples their windows reach) is staged in shared memory,
// realigned so that F_prev sits on a 16-byte boundary; its exact integer sums give mu and
// sigma over the block's start times, and an in-place exclusive scan turns it into prefix
// sums so every boxcar is P[t+W] - P[t]. Scan and threshold work on groups of four
// consecutive samples per lane (one 128-bit shared access per group).
//
// Decision: a cell is in the mask iff max over the row's widths of
//   SNR(W) = (S_W - mu*W) / (sigma*sqrt(W))          (FP64, this operation order)
// reaches Theta. SNR(S) is monotone in the integer S, so thread 0 finds per width the
// smallest integer tau_W with SNR(tau_W) >= Theta by a bounded search around
// mu*W + Theta*sigma*sqrt(W); the per-cell test is then the exact integer compare
// S_W >= tau_W. Cells in the mask get their FP64 S/N maximum (ties -> smaller width)
// rounded to float and are appended to the block's cell list for peak selection.
// Mode A floors sigma at sigma_min; Mode C scores the integer root counts (S/N does not
// change under the 1/sqrt(N_f) scale).

#include <climits>
#include <cmath>
#include <vector>

#include "bulk.h"
#include "snd_internal.h"

namespace snd {
namespace {

struct MfArgs {
  const int32_t* plane;
  int Lp, ndm;
  long long f_prev, e_prev, e_new;
  int nb;  // start times in this block
  const uint16_t* width_mask;
  int binary;
  double theta, sigma_min;
  float out_scale;  // 1/sqrt(N_f) for the caller's float plane, else 0
  uint32_t* mask;
  int mw;
  MfCell* cells;
  int cell_cap;
  uint32_t* counters;
  void* plane_out;
  int nemit;
  int out_u8;       // caller's plane in uint8 (binary / graded roots are 0..255)
  int pf_rows;      // rows resident at once: row d prefetches row d + pf_rows into L2
  int tau_steps;    // bound of the threshold search, steps each way
  int nowrap;       // every prefix sum of the staged segment is below 2^31 (no wrap-around)
  int stat32;       // a lane's sums of y and y^2 over its groups fit in 32 bits
  long long wait_cycles;  // bound of the staging wait (clock cycles)
};

constexpr int kMfThreads = 256;
constexpr uint32_t kAllWidths = (1u << kNumWidthSlots) - 1u;

template <bool A, bool NW = false>
struct WidthSet {  // tag: every width slot of the row is in use (A) or not known to be; prefix
  static constexpr bool kAll = A;     // sums that never wrap (NW)
  static constexpr bool kNoWrap = NW;
};

__device__ __forceinline__ double snr_of(long long s, double mu_w, double den) {
  return __ddiv_rn(__dsub_rn(static_cast<double>(s), mu_w), den);
}

// One DM row d of one plan's block (the body of k_mf and of the many-beam k_mf_multi).
__device__ __forceinline__ void mf_row(const MfArgs& a, const int d) {
  // smem: 4 words of front pad, then y[0..4*G) with y 16-byte aligned, G = len/4 + 2 groups, and
  // one spare group
  extern __shared__ __align__(16) int32_t smem[];
  constexpr int NWARP = kMfThreads / 32;
  __shared__ long long red1[NWARP], red2[NWARP];
  __shared__ int tau[kNumWidthSlots];
  __shared__ double s_muw[kNumWidthSlots], s_den[kNumWidthSlots];
  __shared__ int s_ok;
  __shared__ uint32_t wsum[NWARP];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int len = static_cast<int>(a.e_new - a.f_prev);
  const int c0 = static_cast<int>(a.f_prev % a.Lp);
  const int r0 = c0 & 3;
  int32_t* y = smem + 4;  // y[i] = ring column c0 + i, zero from i = len on
  int4* Y4 = reinterpret_cast<int4*>(y);
  const int G = (len >> 2) + 2;  // groups staged: y[len] and one group past it
  const int nb = a.nb;
  // groups of the statistics passes: warp 0 also finds the row's thresholds in FP64 (a long
  // dependent chain), so the contiguous group segments go to warps 1..NWARP-1
  constexpr int NSEG = NWARP - 1;
  const int segg = ((G + NSEG * 32 - 1) / (NSEG * 32)) * 32;
  const int glo = wid == 0 ? 0 : min(G, (wid - 1) * segg), ghi = wid == 0 ? 0 : min(G, glo + segg);
  // 1. stage the row segment. Bulk path: the TMA engine copies ring columns c0 - r0 ... (16-byte
  //    aligned) as they are, and the statistics pass below shifts them by sh = r0 in place, so
  //    that y[i] = column c0 + i. Otherwise each thread loads and realigns its groups (sh = 0).
  __shared__ int4 bnd[NWARP];  // first staged group of each warp's segment, before the shift
  int sh = 0;
  const int32_t* src = a.plane + static_cast<size_t>(d) * a.Lp;
  const int ng = G + (r0 != 0 ? 1 : 0);  // groups copied by the bulk path
  if (4 * ng <= a.Lp) {
    // one thread issues the bulk copies (one, or two across the ring's wrap point) onto an
    // mbarrier; every thread waits for them (bounded)
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = smem_u32(&bar);
    if (tid == 0) {
      bar_init(b, 1);
      bar_init_fence();
    }
    __syncthreads();
    const int ca0 = c0 - r0;
    const int n1 = min(ng, (a.Lp - ca0) >> 2);  // groups before the wrap point
    if (tid == 0) {
      bar_expect(b, static_cast<uint32_t>(ng) * 16u);
      bulk_g2s(smem_u32(y), src + ca0, static_cast<uint32_t>(n1) * 16u, b);
      if (n1 < ng) bulk_g2s(smem_u32(y + 4 * n1), src, static_cast<uint32_t>(ng - n1) * 16u, b);
    }
    const bool ok = bar_wait(b, 0, a.wait_cycles);
    if (!__syncthreads_and(ok)) {
      // the wait gave up: report it, let the copies land (normal bound) before the CTA leaves
      if (tid == 0) {
        atomicOr(&a.counters[kCntStatus], kStatusMfTimeout);
        bar_wait(b, 0, kStageWaitCycles);
      }
      return;
    }
    sh = r0;
    if (lane == 0 && glo < ghi) bnd[wid] = Y4[glo];
  } else {
    // aligned group m of y takes global groups m and m+1 of the row (16-byte loads of columns
    // c0 - r0 + 4m ...; Lp % 4 == 0, so a group never straddles the ring's wrap point); four
    // groups per thread are loaded before any is stored, so their loads are in flight together
    constexpr int KB = 4;
    for (int m0 = tid; m0 < G; m0 += KB * kMfThreads) {
      int4 g0[KB], g1[KB];
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        const int m = m0 + k * kMfThreads;
        if (m >= G) break;
        int ca = c0 - r0 + 4 * m;
        if (ca >= a.Lp) ca -= a.Lp;
        int cb = ca + 4;
        if (cb >= a.Lp) cb -= a.Lp;
        g0[k] = __ldg(reinterpret_cast<const int4*>(src + ca));
        g1[k] = r0 != 0 ? __ldg(reinterpret_cast<const int4*>(src + cb)) : g0[k];
      }
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        const int m = m0 + k * kMfThreads;
        if (m >= G) break;
        int4 o = g0[k];
        if (r0 == 1) o = make_int4(g0[k].y, g0[k].z, g0[k].w, g1[k].x);
        else if (r0 == 2) o = make_int4(g0[k].z, g0[k].w, g1[k].x, g1[k].y);
        else if (r0 == 3) o = make_int4(g0[k].w, g1[k].x, g1[k].y, g1[k].z);
        const int i = 4 * m;
        if (i + 3 >= len) {
          if (i >= len) o.x = 0;
          if (i + 1 >= len) o.y = 0;
          if (i + 2 >= len) o.z = 0;
          if (i + 3 >= len) o.w = 0;
        }
        Y4[m] = o;
      }
    }
  }
  __syncthreads();
  // 2. one pass over each warp's segment: the shift by sh (bulk path) and the zero tail from
  //    y[len] on, the caller's plane (the newly emitted samples [E_prev, E_new)), the segment's
  //    total (for the scan) and the exact integer sums over the block's start times (y[i], i < nb)
  const int first = static_cast<int>(a.e_prev - a.f_prev);
  {
    uint32_t tot = 0;
    long long s1 = 0, s2 = 0;
    // a lane sums y and y^2 in 32 bits where its groups cannot overflow them (a.stat32), else
    // in 64 bits; the warp reduction is in 64 bits either way
    auto pass = [&](auto zero) {
      using Acc = decltype(zero);
      Acc a1 = 0, a2 = 0;
      for (int base = glo; base < ghi; base += 32) {
        const int g = base + lane;
        int4 v = make_int4(0, 0, 0, 0);
        if (g < ghi) {
          v = Y4[g];
          if (sh != 0) {
            // y group g = the last 4 - sh values of staged group g and the first sh of group g + 1
            // (the next warp's first group as it was before that warp shifted it)
            const int4 nx = (g + 1 == ghi && g + 1 < G) ? bnd[wid + 1] : Y4[g + 1];
            if (sh == 1) v = make_int4(v.y, v.z, v.w, nx.x);
            else if (sh == 2) v = make_int4(v.z, v.w, nx.x, nx.y);
            else v = make_int4(v.w, nx.x, nx.y, nx.z);
          }
          const int i = 4 * g;
          if (i + 3 >= len) {
            if (i >= len) v.x = 0;
            if (i + 1 >= len) v.y = 0;
            if (i + 2 >= len) v.z = 0;
            if (i + 3 >= len) v.w = 0;
          }
        }
        if (sh != 0) __syncwarp();  // every lane has read its next group before any is rewritten
        if (g < ghi && (sh != 0 || 4 * g + 3 >= len)) Y4[g] = v;
        if (g >= ghi) continue;
        const int i = 4 * g;
        if (a.plane_out && i + 3 >= first && i < first + a.nemit) {
          const int vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int k = i + e - first;
            if (k < 0 || k >= a.nemit) continue;
            const size_t o = static_cast<size_t>(d) * a.nemit + k;
            if (a.out_scale != 0.0f) static_cast<float*>(a.plane_out)[o] = static_cast<float>(vv[e]) * a.out_scale;
            else if (a.out_u8) static_cast<uint8_t*>(a.plane_out)[o] = static_cast<uint8_t>(vv[e]);
            else static_cast<int32_t*>(a.plane_out)[o] = vv[e];
          }
        }
        const uint32_t gs = static_cast<uint32_t>(v.x) + static_cast<uint32_t>(v.y) + static_cast<uint32_t>(v.z) +
                            static_cast<uint32_t>(v.w);
        tot += gs;
        const Acc vx = static_cast<Acc>(v.x), vy = static_cast<Acc>(v.y), vz = static_cast<Acc>(v.z),
                  vw = static_cast<Acc>(v.w);
        if (i + 3 < nb) {
          a1 += static_cast<Acc>(gs);
          a2 += (vx * vx + vy * vy) + (vz * vz + vw * vw);
        } else if (i < nb) {
          a1 += vx;
          a2 += vx * vx;
          if (i + 1 < nb) {
            a1 += vy;
            a2 += vy * vy;
          }
          if (i + 2 < nb) {
            a1 += vz;
            a2 += vz * vz;
          }
        }
      }
      s1 = static_cast<long long>(a1);
      s2 = static_cast<long long>(a2);
    };
    if (a.stat32) pass(0u); else pass(0ll);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tot += __shfl_xor_sync(0xFFFFFFFFu, tot, o);
      s1 += __shfl_down_sync(0xFFFFFFFFu, s1, o);
      s2 += __shfl_down_sync(0xFFFFFFFFu, s2, o);
    }
    if (lane == 0) {
      wsum[wid] = tot;
      red1[wid] = s1;
      red2[wid] = s2;
    }
  }
  __syncthreads();
  if (nb <= 0) return;
  const uint32_t wm = a.width_mask[d];
  if (wid == 0) {
    // row statistics (FP64, fixed order) and, lane j, the integer threshold of width 2^j
    long long t1 = 0, t2 = 0;
    for (int w = 0; w < NWARP; ++w) {
      t1 += red1[w];
      t2 += red2[w];
    }
    const double n = static_cast<double>(nb);
    const double mu = __ddiv_rn(static_cast<double>(t1), n);
    const double var = __dsub_rn(__ddiv_rn(static_cast<double>(t2), n), __dmul_rn(mu, mu));
    double sig = var > 0.0 ? __dsqrt_rn(var) : 0.0;
    if (a.binary && sig < a.sigma_min) sig = a.sigma_min;
    if (lane == 0) s_ok = sig > 0.0;
    if (sig > 0.0 && lane < kNumWidthSlots && ((wm >> lane) & 1)) {
      const double w = static_cast<double>(1 << lane);
      const double mu_w = __dmul_rn(mu, w);
      const double den = __dmul_rn(sig, __dsqrt_rn(w));
      s_muw[lane] = mu_w;
      s_den[lane] = den;
      double est = ceil(__dadd_rn(mu_w, __dmul_rn(a.theta, den)));
      if (est < 0.0) est = 0.0;
      if (est > 2147483000.0) est = 2147483000.0;
      long long sv = static_cast<long long>(est);
      int down = 0, up = 0;
      while (sv > 0 && down < a.tau_steps && snr_of(sv - 1, mu_w, den) >= a.theta) {
        --sv;
        ++down;
      }
      while (up < a.tau_steps && snr_of(sv, mu_w, den) < a.theta) {
        ++sv;
        ++up;
      }
      if (down == a.tau_steps || up == a.tau_steps) atomicOr(&a.counters[kCntStatus], kStatusTauTimeout);
      tau[lane] = static_cast<int>(sv);
    }
  }
  // 3. exclusive scan in place (uint32 wrap-around keeps window sums exact): a lane scans its
  //    group of four, the warp scans the group totals, the running carry starts at the sum of
  //    the segments before this warp's
  {
    uint32_t carry = 0;
    for (int w = 0; w < wid; ++w) carry += wsum[w];
    for (int base = glo; base < ghi; base += 32) {
      const int g = base + lane;
      const int4 v = (g < ghi) ? Y4[g] : make_int4(0, 0, 0, 0);
      const uint32_t a0 = static_cast<uint32_t>(v.x);
      const uint32_t a1 = a0 + static_cast<uint32_t>(v.y);
      const uint32_t a2 = a1 + static_cast<uint32_t>(v.z);
      const uint32_t a3 = a2 + static_cast<uint32_t>(v.w);
      uint32_t incl = a3;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += u;
      }
      const uint32_t ex = carry + incl - a3;
      if (g < ghi)
        Y4[g] = make_int4(static_cast<int32_t>(ex), static_cast<int32_t>(ex + a0), static_cast<int32_t>(ex + a1),
                          static_cast<int32_t>(ex + a2));
      carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
  }
  __syncthreads();
  // the row a CTA of the next wave will stage: its segment into L2 (bulk prefetches, one or two
  // across the wrap point) while this row is scored
  if (tid == 0 && d + a.pf_rows < a.ndm) {
    const int32_t* nsrc = a.plane + static_cast<size_t>(d + a.pf_rows) * a.Lp;
    const int gq = min(G + 1, a.Lp >> 2);  // 16-byte groups of the next row's staged columns
    const int n1 = min(gq, (a.Lp - (c0 - r0)) >> 2);
    bulk_prefetch_l2(nsrc + (c0 - r0), static_cast<uint32_t>(n1) * 16u);
    if (n1 < gq) bulk_prefetch_l2(nsrc, static_cast<uint32_t>(gq - n1) * 16u);
  }
  const int nbw = (nb + 31) >> 5;
  uint32_t* mrow = a.mask + static_cast<size_t>(d) * a.mw;
  if (!s_ok) {
    for (int q = tid; q < nbw; q += kMfThreads) mrow[q] = 0;
    return;
  }
  int tw[kNumWidthSlots];
#pragma unroll
  for (int j = 0; j < kNumWidthSlots; ++j) tw[j] = ((wm >> j) & 1) ? tau[j] : 0x7FFFFFFF;
  const uint32_t* P = reinterpret_cast<const uint32_t*>(y);
  const uint4* P4 = reinterpret_cast<const uint4*>(y);
  // 4. threshold: lane m of an iteration tests start times 4m..4m+3 against every width of the
  //    row (window ends P[4m + W ...] are group m + W/4 for W >= 4, groups m and m+1 below).
  //    A cell passes iff max over widths of S_W - tau_W >= 0; S_W < 2^31 and tau_W < 2^31, so
  //    the wrapped difference P[t+W] - P[t] - tau_W read as int32 is exact. Eight lanes'
  //    nibbles make one mask word.
  // hit nibble of start times 4m..4m+3 (bit e: start time 4m + e passes)
  // Without wrap-around (prefix sums below 2^31, the usual case) the test is rearranged as
  // max over W of (P[t+W] - tau_W) >= P[t]: one add-and-max per (start time, width), which
  // the compiler can issue as a single three-input integer instruction.
  auto group_hits = [&](int m, auto all) -> uint32_t {
    constexpr bool ALL = decltype(all)::kAll;
    constexpr bool NOWRAP = decltype(all)::kNoWrap;
    const uint4 p = P4[m];
    const uint4 q = P4[m + 1];
    int h0 = INT_MIN, h1 = INT_MIN, h2 = INT_MIN, h3 = INT_MIN;
    auto upd = [](int& h, uint32_t end, uint32_t start, int tj) {
      if constexpr (NOWRAP) {
        h = max(static_cast<int>(end) + (-tj), h);
      } else {
        h = max(h, static_cast<int>(end - start - static_cast<uint32_t>(tj)));
      }
    };
    if (ALL || (wm & 1u)) {
      upd(h0, p.y, p.x, tw[0]);
      upd(h1, p.z, p.y, tw[0]);
      upd(h2, p.w, p.z, tw[0]);
      upd(h3, q.x, p.w, tw[0]);
    }
    if (ALL || (wm & 2u)) {
      upd(h0, p.z, p.x, tw[1]);
      upd(h1, p.w, p.y, tw[1]);
      upd(h2, q.x, p.z, tw[1]);
      upd(h3, q.y, p.w, tw[1]);
    }
    if (ALL || (wm & 4u)) {
      upd(h0, q.x, p.x, tw[2]);
      upd(h1, q.y, p.y, tw[2]);
      upd(h2, q.z, p.z, tw[2]);
      upd(h3, q.w, p.w, tw[2]);
    }
    auto wide = [&](int j) {
      const uint4 e = P4[m + (1 << (j - 2))];
      upd(h0, e.x, p.x, tw[j]);
      upd(h1, e.y, p.y, tw[j]);
      upd(h2, e.z, p.z, tw[j]);
      upd(h3, e.w, p.w, tw[j]);
    };
#pragma unroll
    for (int j = 3; j < kNumWidthSlots; ++j)
      if (ALL || ((wm >> j) & 1u)) wide(j);
    if constexpr (NOWRAP)
      return (h0 >= static_cast<int>(p.x) ? 1u : 0u) | (h1 >= static_cast<int>(p.y) ? 2u : 0u) |
             (h2 >= static_cast<int>(p.z) ? 4u : 0u) | (h3 >= static_cast<int>(p.w) ? 8u : 0u);
    return (h0 >= 0 ? 1u : 0u) | (h1 >= 0 ? 2u : 0u) | (h2 >= 0 ? 4u : 0u) | (h3 >= 0 ? 8u : 0u);
  };
  const int ngt = (nb + 3) >> 2;
  for (int base = wid * 32; base < ngt; base += NWARP * 32) {
    const int m = base + lane;
    uint32_t nib = 0;
    if (m < ngt) {
      // rows with every width (most rows above a small DM) take a copy of the loop with no
      // width tests, so all window loads of the group can be in flight together
      if (a.nowrap)
        nib = (wm == kAllWidths) ? group_hits(m, WidthSet<true, true>{}) : group_hits(m, WidthSet<false, true>{});
      else
        nib = (wm == kAllWidths) ? group_hits(m, WidthSet<true>{}) : group_hits(m, WidthSet<false>{});
      const int rem = nb - 4 * m;  // start times of this group inside the block
      if (rem < 4) nib &= (1u << rem) - 1u;
    }
    uint32_t word = nib << (4 * (lane & 7));
    word |= __shfl_xor_sync(0xFFFFFFFFu, word, 1);
    word |= __shfl_xor_sync(0xFFFFFFFFu, word, 2);
    word |= __shfl_xor_sync(0xFFFFFFFFu, word, 4);
    const int qw = (base >> 3) + (lane >> 3);
    if ((lane & 7) == 0 && qw < nbw) mrow[qw] = word;
    while (nib) {
      const int e = __ffs(nib) - 1;
      nib &= nib - 1u;
      const int t = 4 * m + e;
      const uint32_t p0 = P[t];
      double best = -1.0e300;
      int bw = 0;
      for (int j = 0; j < kNumWidthSlots; ++j) {
        if (!((wm >> j) & 1)) continue;
        const long long S = static_cast<int>(P[t + (1 << j)] - p0);
        const double v = snr_of(S, s_muw[j], s_den[j]);
        if (v > best) {
          best = v;
          bw = 1 << j;
        }
      }
      const uint32_t idx = atomicAdd(&a.counters[kCntCells], 1u);
      if (idx < static_cast<uint32_t>(a.cell_cap)) {
        MfCell c;
        c.cell = static_cast<uint32_t>(d) * static_cast<uint32_t>(nb) + static_cast<uint32_t>(t);
        c.snr = __double2float_rn(best);
        c.width = bw;
        a.cells[idx] = c;
      } else {
        atomicOr(&a.counters[kCntStatus], kStatusCellOverflow);
      }
    }
  }
}

__global__ void __launch_bounds__(kMfThreads, 3) k_mf(const __grid_constant__ MfArgs a) { mf_row(a, blockIdx.x); }

constexpr int kMaxMfBeams = 64;

// Many plans' blocks in one launch: CTA i scores row i - first[b] of the last beam b with
// first[b] <= i.
struct MfMulti {
  int nbeams;
  int first[kMaxMfBeams];
  MfArgs beam[kMaxMfBeams];
};

__global__ void __launch_bounds__(kMfThreads, 3) k_mf_multi(const __grid_constant__ MfMulti m) {
  const int i = static_cast<int>(blockIdx.x);
  int lo = 0, hi = m.nbeams - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (m.first[mid] <= i) lo = mid; else hi = mid - 1;
  }
  mf_row(m.beam[lo], i - m.first[lo]);
}

// Arguments of one plan's block; *smem = the dynamic shared memory of its row staging.
// Returns false when the block has nothing to do.
bool mf_args(const Plan& p, int64_t e_prev, int64_t e_new, int64_t f_prev, int64_t f_new, void* d_plane_out,
             MfArgs& a, int* smem) {
  const int nb = static_cast<int>(f_new - f_prev);
  const int nemit = static_cast<int>(e_new - e_prev);
  if (nb <= 0 && (d_plane_out == nullptr || nemit <= 0)) return false;
  a = MfArgs{};
  a.plane = p.dp.plane;
  a.Lp = p.Lp;
  a.ndm = p.ndm;
  a.f_prev = f_prev;
  a.e_prev = e_prev;
  a.e_new = e_new;
  a.nb = nb;
  a.width_mask = p.dp.width_mask;
  a.binary = p.mode == SND_MODE_BINARY;
  a.theta = p.det_theta;
  a.sigma_min = p.sigma_min;
  a.out_scale = (p.mode == SND_MODE_FLOAT) ? static_cast<float>(1.0 / std::sqrt(static_cast<double>(p.nchan))) : 0.0f;
  a.mask = p.dp.mask;
  a.mw = p.mw;
  a.cells = p.dp.cells;
  a.cell_cap = p.cell_cap;
  a.counters = p.dp.counters;
  a.plane_out = nemit > 0 ? d_plane_out : nullptr;
  a.nemit = nemit;
  a.out_u8 = p.plane_u8;
  a.tau_steps = p.loop_limit > 0 ? static_cast<int>(p.loop_limit < 64 ? p.loop_limit : 64) : 64;
  const int len = static_cast<int>(e_new - f_prev);
  *smem = ((len >> 2) + 4) * 16;  // front pad (4 words), len/4 + 2 aligned groups and one more for the
                                  // bulk copy of a segment that starts off a 16-byte boundary
  {
    // largest root value of the mode times the staged samples bounds every prefix sum
    const double vmax = p.mode == SND_MODE_BINARY ? 1.0 : (p.mode == SND_MODE_GRADED ? p.N : p.nchan);
    a.nowrap = vmax * (len + 8.0) < 2147483647.0 ? 1 : 0;
    // samples a lane of the statistics pass sums (its groups of the seven-warp segments)
    const int groups = (len >> 2) + 2;
    const double per_lane = 4.0 * ((groups + 7 * 32 - 1) / (7 * 32));
    a.stat32 = per_lane * vmax * vmax < 4294967295.0 ? 1 : 0;
  }
  a.wait_cycles = p.wait_limit > 0 ? p.wait_limit : kStageWaitCycles;
  return true;
}

// rows resident at once on the GPU for a kernel with `smem` bytes per CTA
template <typename K>
cudaError_t resident_rows(K kern, int smem, int fallback, int* out) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMfThreads, smem);
  *out = per_sm > 0 ? nsm * per_sm : fallback;
  return e;
}

}  // namespace

cudaError_t launch_mf(const Plan& p, int64_t e_prev, int64_t e_new, int64_t f_prev, int64_t f_new,
                      void* d_plane_out, cudaStream_t s) {
  MfArgs a;
  int smem = 0;
  if (!mf_args(p, e_prev, e_new, f_prev, f_new, d_plane_out, a, &smem)) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_mf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = resident_rows(k_mf, smem, p.ndm, &a.pf_rows);
  if (e != cudaSuccess) return e;
  k_mf<<<p.ndm, kMfThreads, smem, s>>>(a);
  p.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_mf_batch(const Plan* const* plans, const ChunkPos* pos, int n, cudaStream_t s) {
  // Blocks are grouped by the CTAs per SM their row staging allows (shared memory up to about
  // 72 KB: three, 110 KB: two, more: one), so a long-chunk beam does not lower the occupancy of
  // every other beam's rows: at most three launches (more only past 64 beams per group).
  auto cls = [](int smem) { return smem <= 72 * 1024 ? 0 : (smem <= 110 * 1024 ? 1 : 2); };
  std::vector<MfArgs> args(n);
  std::vector<int> sm(n, 0), live(n, 0);
  for (int i = 0; i < n; ++i)
    live[i] = mf_args(*plans[i], pos[i].e_prev, pos[i].e_new, pos[i].f_prev, pos[i].f_new, nullptr, args[i], &sm[i]);
  for (int c = 0; c < 3; ++c) {
    for (int i0 = 0; i0 < n;) {
      MfMulti m{};
      int smem = 0, ctas = 0;
      const Plan* owner = nullptr;
      int i = i0;
      for (; i < n && m.nbeams < kMaxMfBeams; ++i) {
        if (!live[i] || cls(sm[i]) != c) continue;
        m.beam[m.nbeams] = args[i];
        m.first[m.nbeams] = ctas;
        ctas += plans[i]->ndm;
        smem = smem > sm[i] ? smem : sm[i];
        if (!owner) owner = plans[i];
        ++m.nbeams;
      }
      i0 = i;
      if (m.nbeams == 0) continue;
      cudaError_t e = cudaFuncSetAttribute(k_mf_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      int pf = 0;
      if (e == cudaSuccess) e = resident_rows(k_mf_multi, smem, ctas, &pf);
      if (e != cudaSuccess) return e;
      for (int b = 0; b < m.nbeams; ++b) m.beam[b].pf_rows = pf;
      k_mf_multi<<<ctas, kMfThreads, smem, s>>>(m);
      owner->launches += 1;
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace snd
