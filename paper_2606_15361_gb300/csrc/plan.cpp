// Host side of the SND library: options, plan construction, statistics, error strings.
//
// Plan construction follows Methods, "The Spiking Neural Dedispersion algorithm":
// integer delays per channel and trial DM, leaf clusters of C contiguous channels,
// B-ary levels above them, and enumeration of the distinct integer-delay patterns of
// every node. The GPU evaluates the tree from the leaf patterns (see tree.cu); the
// deeper-level pattern counts are kept as plan statistics (neuron counts, additions per
// DM-sample, Eq. hist_mem).
//
// This file must be compiled without floating-point contraction (-ffp-contract=off):
// the delay rounding and the width rule are FP64 decisions with a fixed operation order.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <unordered_map>
#include <vector>

#include "snd_internal.h"

using snd::Plan;

namespace {

constexpr double kDm = 4.148808e3;  // MHz^2 s pc^-1 cm^3

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct VecHash {
  size_t operator()(const std::vector<int32_t>& v) const {
    uint64_t h = 1469598103934665603ull;
    for (int32_t x : v) {
      h ^= static_cast<uint32_t>(x);
      h *= 1099511628211ull;
    }
    return static_cast<size_t>(h ^ (h >> 29));
  }
};

int choose_tree_geometry(Plan& p);
int choose_tree_geometry_w(Plan& p, int warps);
int choose_ztree_geometry(Plan& p);
void choose_direct_geometry(Plan& p);

}  // namespace

namespace snd {

// Host allocation failure injection (snd_debug_fail_host_alloc): the allocation point that
// finds the countdown at zero throws std::bad_alloc, as a failed allocation would, and
// disarms it; -1 = disarmed.
std::atomic<int> g_fail_alloc{-1};

void alloc_point() {
  int v = g_fail_alloc.load();
  while (v >= 0) {
    if (g_fail_alloc.compare_exchange_weak(v, v == 0 ? -1 : v - 1)) {
      if (v == 0) throw std::bad_alloc();
      return;
    }
  }
}

}  // namespace snd

extern "C" int snd_debug_fail_host_alloc(int32_t after) {
  snd::g_fail_alloc.store(after < 0 ? -1 : after);
  return SND_OK;
}

extern "C" int snd_options_init(snd_mode_t mode, snd_options_t* o) {
  if (!o) return SND_ERR_ARG;
  if (mode != SND_MODE_BINARY && mode != SND_MODE_GRADED && mode != SND_MODE_FLOAT && mode != SND_MODE_ZFLOAT)
    return SND_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  // Supplementary Table S1 operating points; C = 4 from its SND-tree block.
  o->cluster_size = 4;
  o->k_leaf = 2;
  o->k_internal = 2;
  o->graded_cap = 255;
  o->enc_theta = (mode == SND_MODE_GRADED) ? 0.75 : 1.5;
  o->det_theta = 7.0;
  o->sigma_min = 0.20;
  o->mf_alpha = 0.1;  // Methods, "Matched filtering"
  o->closing_size = 9;
  o->n_min_pixels = 10;
  o->max_chunk = 32768;
  o->cand_capacity = 65536;
  o->cell_capacity = 1 << 20;
  o->run_capacity = 1 << 21;
  o->flags = 0;
  return SND_OK;
}

namespace snd {

int build_plan(Plan& p) {
  const int nchan = p.nchan, ndm = p.ndm, C = p.C, B = p.B;
  alloc_point();  // the delay table
  // --- delays (Methods, "Incoherent dedispersion") ---
  std::vector<double> inv2(nchan);
  for (int c = 0; c < nchan; ++c) inv2[c] = 1.0 / (p.freqs[c] * p.freqs[c]);
  p.ref_chan = 0;
  p.min_chan = 0;
  for (int c = 1; c < nchan; ++c) {
    if (p.freqs[c] > p.freqs[p.ref_chan]) p.ref_chan = c;
    if (p.freqs[c] < p.freqs[p.min_chan]) p.min_chan = c;
  }
  p.delays.assign(static_cast<size_t>(ndm) * nchan, 0);
  int64_t dmax = 0;
  for (int d = 0; d < ndm; ++d) {
    const double kd = kDm * p.dms[d];
    for (int c = 0; c < nchan; ++c) {
      const double x = (kd * (inv2[c] - inv2[p.ref_chan])) / p.dt;
      const double r = std::floor(x + 0.5);
      if (!(r >= 0.0) || r > 1.0e9) return SND_ERR_DM;
      p.delays[static_cast<size_t>(d) * nchan + c] = static_cast<int32_t>(r);
      dmax = std::max<int64_t>(dmax, static_cast<int64_t>(r));
    }
  }
  p.D = static_cast<int>(dmax);

  // --- boxcar widths (Methods, "Matched filtering") ---
  p.width_mask.assign(ndm, 0);
  p.wmax = 1;
  for (int d = 0; d < ndm; ++d) {
    const double sweep = ((kDm * p.dms[d]) * (inv2[p.min_chan] - inv2[p.ref_chan])) / p.dt;
    const double lim = p.mf_alpha * sweep;
    uint16_t m = 0x000F;  // 1, 2, 4, 8
    for (int j = 4; j < kNumWidthSlots; ++j)
      if (static_cast<double>(1 << j) <= lim) m |= static_cast<uint16_t>(1u << j);
    p.width_mask[d] = m;
    for (int j = 0; j < kNumWidthSlots; ++j)
      if (m & (1u << j)) p.wmax = std::max(p.wmax, 1 << j);
  }

  // --- tree levels (Methods, "Leaf clusters" / "Tree levels") ---
  p.level_nodes.clear();
  p.level_nodes.push_back((nchan + C - 1) / C);
  while (p.level_nodes.back() > 1) p.level_nodes.push_back((p.level_nodes.back() + B - 1) / B);
  p.nlev = static_cast<int>(p.level_nodes.size());
  if (p.nlev > kMaxLevels) return SND_ERR_UNSUPPORTED;
  p.nleaves = p.level_nodes[0];
  const int NL = p.nleaves;

  // channel range and reference channel of every node, level by level
  std::vector<std::vector<int>> node_lo(p.nlev), node_hi(p.nlev), node_ref(p.nlev);
  for (int l = 0; l < p.nlev; ++l) {
    const int n = p.level_nodes[l];
    node_lo[l].resize(n);
    node_hi[l].resize(n);
    node_ref[l].resize(n);
    for (int i = 0; i < n; ++i) {
      int lo, hi;
      if (l == 0) {
        lo = i * C;
        hi = std::min(nchan, lo + C);
      } else {
        lo = node_lo[l - 1][i * B];
        hi = node_hi[l - 1][std::min(p.level_nodes[l - 1], (i + 1) * B) - 1];
      }
      node_lo[l][i] = lo;
      node_hi[l][i] = hi;
      int r = lo;
      for (int c = lo + 1; c < hi; ++c)
        if (p.freqs[c] > p.freqs[r]) r = c;
      node_ref[l][i] = r;
    }
  }

  // --- leaf patterns: distinct relative delays delta_c(d) - delta_ref(d) per leaf ---
  alloc_point();
  p.leaf_pid.assign(static_cast<size_t>(ndm) * NL, 0);
  std::vector<int32_t> leaf_loc(static_cast<size_t>(ndm) * NL, 0);  // id local to the leaf
  p.pat_rel.clear();
  p.npat = 0;
  std::vector<int> leaf_npat(NL, 0);
  int64_t din = 0;
  {
    std::vector<int32_t> key(C);
    for (int k = 0; k < NL; ++k) {
      std::unordered_map<std::vector<int32_t>, int, VecHash> ids;
      const int base = p.npat;
      const int lo = node_lo[0][k], hi = node_hi[0][k], r = node_ref[0][k];
      for (int d = 0; d < ndm; ++d) {
        const int32_t* row = &p.delays[static_cast<size_t>(d) * nchan];
        std::fill(key.begin(), key.end(), 0);
        for (int c = lo; c < hi; ++c) {
          key[c - lo] = row[c] - row[r];
          din = std::max<int64_t>(din, key[c - lo]);
        }
        auto it = ids.find(key);
        int id;
        if (it == ids.end()) {
          id = p.npat++;
          ids.emplace(key, id);
          p.pat_rel.insert(p.pat_rel.end(), key.begin(), key.end());
          leaf_npat[k]++;
        } else {
          id = it->second;
        }
        p.leaf_pid[static_cast<size_t>(d) * NL + k] = id;
        leaf_loc[static_cast<size_t>(d) * NL + k] = id - base;
      }
    }
  }

  // --- statistics: distinct patterns at every level, additions, Eq. hist_mem ---
  alloc_point();
  {
    p.level_unique.assign(p.nlev, 0);
    double adds = 0.0;
    const int bits_out = (p.mode == SND_MODE_BINARY)   ? 1
                         : (p.mode == SND_MODE_GRADED) ? 8
                         : (p.mode == SND_MODE_ZFLOAT && (p.flags & SND_FLAG_FP16_PARTIALS)) ? 16
                                                       : 32;
    double hist_bits_bytes = std::ceil(static_cast<double>(nchan) * static_cast<double>(din) / 8.0);
    // node pattern ids of the level below, [ndm][n]
    std::vector<int32_t> below(leaf_loc);
    std::vector<int> below_count(leaf_npat);
    for (int k = 0; k < NL; ++k) {
      p.level_unique[0] += leaf_npat[k];
      adds += static_cast<double>(leaf_npat[k]) * (node_hi[0][k] - node_lo[0][k] - 1);
    }
    for (int l = 0; l < p.nlev; ++l) {
      const int n = p.level_nodes[l];
      // ring depth d_{n,m}: largest shift the parent requests from node n in pattern m
      if (l + 1 < p.nlev) {
        for (int i = 0; i < n; ++i) {
          const int par = i / B;
          std::vector<int64_t> depth(below_count[i], 0);
          for (int d = 0; d < ndm; ++d) {
            const int32_t* row = &p.delays[static_cast<size_t>(d) * nchan];
            const int64_t sh = row[node_ref[l][i]] - row[node_ref[l + 1][par]];
            int32_t m = below[static_cast<size_t>(d) * n + i];
            depth[m] = std::max(depth[m], sh);
          }
          for (int64_t dd : depth)
            hist_bits_bytes += std::ceil(static_cast<double>(dd) * bits_out / 8.0);
        }
      }
      if (l + 1 >= p.nlev) break;
      const int np = p.level_nodes[l + 1];
      std::vector<int32_t> cur(static_cast<size_t>(ndm) * np, 0);
      std::vector<int> cur_count(np, 0);
      for (int j = 0; j < np; ++j) {
        const int c0 = j * B, c1 = std::min(n, (j + 1) * B);
        std::unordered_map<std::vector<int32_t>, int, VecHash> ids;
        std::vector<int32_t> key(2 * (c1 - c0));
        for (int d = 0; d < ndm; ++d) {
          const int32_t* row = &p.delays[static_cast<size_t>(d) * nchan];
          for (int i = c0; i < c1; ++i) {
            key[2 * (i - c0)] = below[static_cast<size_t>(d) * n + i];
            key[2 * (i - c0) + 1] = row[node_ref[l][i]] - row[node_ref[l + 1][j]];
          }
          auto it = ids.find(key);
          int id;
          if (it == ids.end()) {
            id = cur_count[j]++;
            ids.emplace(key, id);
          } else {
            id = it->second;
          }
          cur[static_cast<size_t>(d) * np + j] = id;
        }
        p.level_unique[l + 1] += cur_count[j];
        adds += static_cast<double>(cur_count[j]) * (c1 - c0 - 1);
      }
      below.swap(cur);
      below_count.swap(cur_count);
    }
    p.adds_per_dm_sample = adds / ndm;
    p.hist_mem_bytes = static_cast<int64_t>(hist_bits_bytes);
  }

  // --- DM tiles: distinct leaf patterns per (tile, leaf), per-DM index and shift, for the
  // bit-sliced tree; the labelled-payload tree has tiles of its own (and no bit ring use) ---
  alloc_point();  // the kernel tables
  int rc = (p.mode == SND_MODE_ZFLOAT) ? choose_ztree_geometry(p) : choose_tree_geometry(p);
  if (p.mode != SND_MODE_ZFLOAT) {
    choose_direct_geometry(p);
    if (p.direct) rc = SND_OK;  // the leaf-sharing kernel may not fit; the direct one does
  }
  if (rc) return rc;

  // --- ring, plane ring and workspace layout ---
  const TreeGeom& g = p.geom;
  const int maxw_chunk = (p.max_chunk + 31) / 32;
  // words reachable from one emitted block: delay + chunk + tile padding + funnel partner
  p.R = (p.D >> 5) + maxw_chunk + std::max(g.cspan, p.dgeom.cspan) + 8;
  p.R = static_cast<int>(align_up(static_cast<size_t>(p.R), 4));  // 16-byte aligned bulk copies of ring rows
  p.Lp = static_cast<int>(align_up(static_cast<size_t>(p.wmax) - 1 + p.max_chunk + 96, 32));
  p.mw = (p.Lp + 31) / 32;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  p.off.ring = take(sizeof(uint32_t) * static_cast<size_t>(nchan) * 2 * p.R);
  p.off.hist = take(sizeof(uint32_t) * static_cast<size_t>(nchan) * 256);
  p.off.levels = take(sizeof(int32_t) * nchan);
  p.off.plane = take(sizeof(int32_t) * static_cast<size_t>(ndm) * p.Lp);
  p.off.mask = take(sizeof(uint32_t) * static_cast<size_t>(ndm) * p.mw);
  p.off.mask2 = take(sizeof(uint32_t) * static_cast<size_t>(ndm) * p.mw);
  p.off.mask3 = take(sizeof(uint32_t) * static_cast<size_t>(ndm) * p.mw);
  p.off.cells = take(sizeof(MfCell) * static_cast<size_t>(p.cell_cap));
  p.off.counters = take(sizeof(uint32_t) * kCntSlots);
  p.off.row_runs = take(sizeof(int32_t) * (static_cast<size_t>(ndm) + 1));
  p.off.run_start = take(sizeof(int32_t) * static_cast<size_t>(p.run_cap));
  p.off.run_end = take(sizeof(int32_t) * static_cast<size_t>(p.run_cap));
  p.off.run_row = take(sizeof(int32_t) * static_cast<size_t>(p.run_cap));
  p.off.parent = take(sizeof(int32_t) * static_cast<size_t>(p.run_cap));
  p.off.npix = take(sizeof(int32_t) * static_cast<size_t>(p.run_cap));
  p.off.peak = take(sizeof(unsigned long long) * static_cast<size_t>(p.run_cap));
  p.off.pwidth = take(sizeof(int32_t) * static_cast<size_t>(p.run_cap));
  p.off.bcand = take(sizeof(snd_candidate_t) * static_cast<size_t>(p.cand_cap));
  p.off.cand = take(sizeof(snd_candidate_t) * static_cast<size_t>(p.cand_cap));
  p.off.staging = take(static_cast<size_t>(p.max_chunk) * nchan);
  p.off.staging2 = take(static_cast<size_t>(p.max_chunk) * nchan);
  p.off.width_mask = take(sizeof(uint16_t) * ndm);
  p.off.dm_f32 = take(sizeof(float) * ndm);
  p.off.tp_off = take(sizeof(int32_t) * p.tp_off.size());
  p.off.gepk = take(sizeof(uint32_t) * std::max<size_t>(1, p.gepk.size()));
  p.off.gleaf = take(sizeof(int32_t) * std::max<size_t>(1, p.gleaf.size()));
  p.off.gmeta = take(sizeof(uint32_t) * p.gmeta.size());
  p.off.tile_wb = take(sizeof(int32_t) * p.tile_wb.size());
  p.off.delays = take(sizeof(int32_t) * p.delays.size());
  p.off.dmeta = take(sizeof(uint16_t) * std::max<size_t>(8, p.dmeta.size()));
  p.off.dbase = take(sizeof(int32_t) * std::max<size_t>(4, p.dbase.size()));
  p.off.level_fires = take(sizeof(unsigned long long) * snd::kMaxLevels);
  if (p.mode == SND_MODE_ZFLOAT) {
    const size_t es = p.zgeom.fp16 ? 2 : 4;
    p.off.zring = take(es * static_cast<size_t>(nchan) * p.zgeom.Rz);
    p.off.ztab = take(es * static_cast<size_t>(nchan) * 256);
    p.off.zwb = take(sizeof(int32_t) * p.zwb.size());
    p.off.zcarry = take(sizeof(int32_t) * p.zcarry.size());
  }
  p.ws_bytes = o;
  return SND_OK;
}

}  // namespace snd

namespace {

// Tree kernel geometry: the kernel shape of tree_shape(), or, when a DM tile of that many
// trial DMs spans delays too wide for shared memory (coarse DM grids), the same kernel with
// fewer warps (fewer DMs per tile) until it fits.
int choose_tree_geometry(Plan& p) {
  const snd::TreeShape sh = snd::tree_shape(p.mode, p.nlev, p.KL > p.KI ? p.KL : p.KI);
  int rc = SND_ERR_UNSUPPORTED;
  for (int w = sh.warps; w >= 4; w /= 2) {
    rc = choose_tree_geometry_w(p, w);
    if (rc != SND_ERR_UNSUPPORTED) break;
  }
  return rc;
}

// Geometry for `warps` warps: DMs per CTA, output words per CTA, the per-(tile, leaf) lists
// of distinct leaf patterns, the staged window sizes, and how many leaves (a multiple of B)
// are staged per shared-memory round so that a CTA fits the shared-memory budget.
int choose_tree_geometry_w(Plan& p, int warps) {
  snd::TreeGeom& g = p.geom;
  const int ndm = p.ndm, NL = p.nleaves, nchan = p.nchan;
  const snd::TreeShape sh = snd::tree_shape(p.mode, p.nlev, p.KL > p.KI ? p.KL : p.KI);
  g.warps = warps;
  g.dpw = sh.dpw;
  g.kw = sh.kw;
  g.dms_per_cta = warps * sh.dpw;
  g.tile_words = 32 * g.kw;
  g.planes = (p.mode == SND_MODE_BINARY) ? 1 : 3;
  g.ndm_tiles = (ndm + g.dms_per_cta - 1) / g.dms_per_cta;

  p.tp_off.assign(static_cast<size_t>(g.ndm_tiles) * NL + 1, 0);
  p.tp_pid.clear();
  p.tp_smin.clear();
  p.tp_leaf.clear();
  p.dl_lp.assign(static_cast<size_t>(ndm) * NL, 0);
  p.dl_sh.assign(static_cast<size_t>(ndm) * NL, 0);
  p.tile_wb.assign(static_cast<size_t>(g.ndm_tiles) * nchan, 0);
  int64_t sspread = 0, cspread = 0;
  std::vector<int> npat_tl(static_cast<size_t>(g.ndm_tiles) * NL, 0);
  for (int t = 0; t < g.ndm_tiles; ++t) {
    const int d0 = t * g.dms_per_cta, d1 = std::min(ndm, d0 + g.dms_per_cta);
    for (int c = 0; c < nchan; ++c) {
      int32_t lo = p.delays[static_cast<size_t>(d0) * nchan + c], hi = lo;
      for (int d = d0 + 1; d < d1; ++d) {
        lo = std::min(lo, p.delays[static_cast<size_t>(d) * nchan + c]);
        hi = std::max(hi, p.delays[static_cast<size_t>(d) * nchan + c]);
      }
      p.tile_wb[static_cast<size_t>(t) * nchan + c] = std::max(lo - 31, 0) >> 5;
      cspread = std::max<int64_t>(cspread, static_cast<int64_t>(hi) - lo);
    }
    for (int k = 0; k < NL; ++k) {
      // reference channel of the leaf: highest frequency among its channels
      int r = k * p.C;
      for (int c = k * p.C + 1; c < std::min(nchan, (k + 1) * p.C); ++c)
        if (p.freqs[c] > p.freqs[r]) r = c;
      const size_t at = static_cast<size_t>(t) * NL + k;
      p.tp_off[at] = static_cast<int32_t>(p.tp_pid.size());
      std::vector<int32_t> pids, smin, smax;
      for (int d = d0; d < d1; ++d) {
        const int32_t pid = p.leaf_pid[static_cast<size_t>(d) * NL + k];
        const int32_t s = p.delays[static_cast<size_t>(d) * nchan + r];
        int idx = -1;
        for (size_t i = 0; i < pids.size(); ++i)
          if (pids[i] == pid) idx = static_cast<int>(i);
        if (idx < 0) {
          idx = static_cast<int>(pids.size());
          pids.push_back(pid);
          smin.push_back(s);
          smax.push_back(s);
        } else {
          smin[idx] = std::min(smin[idx], s);
          smax[idx] = std::max(smax[idx], s);
        }
        p.dl_lp[static_cast<size_t>(d) * NL + k] = static_cast<uint8_t>(idx);
        p.dl_sh[static_cast<size_t>(d) * NL + k] = s;
      }
      for (size_t i = 0; i < pids.size(); ++i) {
        p.tp_pid.push_back(pids[i]);
        p.tp_smin.push_back(smin[i]);
        p.tp_leaf.push_back(k);
        sspread = std::max<int64_t>(sspread, static_cast<int64_t>(smax[i]) - smin[i]);
      }
      npat_tl[at] = static_cast<int>(pids.size());
    }
  }
  p.tp_off.back() = static_cast<int32_t>(p.tp_pid.size());
  // series word j covers leaf samples [32*(smin>>5) + 32 j, +32): a DM with shift s reads
  // words (s>>5)-(smin>>5) + w and +1 for w < tile_words
  g.span = g.tile_words + static_cast<int>(sspread >> 5) + 2;
  // channel c of entry (smin, rel) is read at window words ((32(smin>>5)+rel)>>5) - wb_c + j (+1)
  g.cspan = g.span + static_cast<int>((cspread + 31) >> 5) + 2;

  auto smem_for = [&](int G, int* mp_out) {
    int mp = 0;
    for (int t = 0; t < g.ndm_tiles; ++t)
      for (int k0 = 0; k0 < NL; k0 += G) {
        int s = 0;
        for (int k = k0; k < std::min(NL, k0 + G); ++k) s += npat_tl[static_cast<size_t>(t) * NL + k];
        mp = std::max(mp, s);
      }
    *mp_out = mp;
    // series as word pairs + two staging buffers (windows, meta, entry offsets and leaves) +
    // the tile's window base per channel
    const int64_t buf = (static_cast<int64_t>(G) * p.C * g.cspan + static_cast<int64_t>(g.dms_per_cta) * G +
                         static_cast<int64_t>(mp) * (p.C + 1) + 3) & ~int64_t(3);
    const int64_t words = 2 * static_cast<int64_t>(mp) * g.planes * g.span + 2 * buf + nchan;
    return words * 4;
  };
  // binary trees run two CTAs per SM (about 100 KB each); graded and float trees one, which
  // may take twice that so a group holds more leaves (fewer rounds of staging and barriers)
  const int64_t budget = (p.mode == SND_MODE_BINARY ? 100 : 200) * 1024;
  const int unit = (p.nlev == 1) ? 1 : std::min(p.B, NL);
  int G = unit, mp = 0;
  int64_t bytes = smem_for(G, &mp);
  for (int m = 2; unit * m <= NL + unit - 1 && unit * (m - 1) < NL; ++m) {
    int mp2 = 0;
    const int64_t b2 = smem_for(unit * m, &mp2);
    if (b2 > budget) break;
    G = unit * m;
    mp = mp2;
    bytes = b2;
  }
  g.group_leaves = G;
  g.max_pat_group = mp;
  g.smem_bytes = static_cast<int>(bytes);
  if (bytes > 220 * 1024) return SND_ERR_UNSUPPORTED;

  // Precomputed staging offsets, so a CTA only copies tables:
  //  gepk[entry][ci]: channel ci of entry (smin, rel) is read at staged-window word
  //    ((32*(smin>>5) + rel) >> 5) - wb_c (+ j, + 1) with bit shift rel & 31;
  //  gleaf[entry]: its leaf relative to the first leaf of its group;
  //  gmeta[d][k]: DM d gathers leaf k from series word ((e*planes*span + j0) << 5 | s & 31),
  //    e = the entry's index within its group, j0 = (s>>5) - (smin>>5), s = the leaf shift.
  const size_t ntp = p.tp_pid.size();
  p.gepk.assign(ntp * p.C, 0);
  p.gleaf.assign(ntp, 0);
  for (int t = 0; t < g.ndm_tiles; ++t)
    for (int k = 0; k < NL; ++k)
      for (int32_t e = p.tp_off[static_cast<size_t>(t) * NL + k]; e < p.tp_off[static_cast<size_t>(t) * NL + k + 1];
           ++e) {
        const int pid = p.tp_pid[e], smin = p.tp_smin[e];
        p.gleaf[e] = k - (k / G) * G;
        for (int ci = 0; ci < p.C; ++ci) {
          const int c = k * p.C + ci;
          if (c >= nchan) continue;
          const int q = 32 * (smin >> 5) + p.pat_rel[static_cast<size_t>(pid) * p.C + ci];
          const int eoff = (q >> 5) - p.tile_wb[static_cast<size_t>(t) * nchan + c];
          p.gepk[e * p.C + ci] = (static_cast<uint32_t>(eoff) << 5) | static_cast<uint32_t>(q & 31);
        }
      }
  p.gmeta.assign(static_cast<size_t>(ndm) * NL, 0);
  for (int d = 0; d < ndm; ++d) {
    const int t = d / g.dms_per_cta;
    for (int k = 0; k < NL; ++k) {
      const size_t at = static_cast<size_t>(d) * NL + k;
      const int g0 = (k / G) * G;
      const int ebase = p.tp_off[static_cast<size_t>(t) * NL + g0];
      const int eg = p.tp_off[static_cast<size_t>(t) * NL + k] + p.dl_lp[at];  // global entry index
      const int s = p.dl_sh[at];
      const int j0 = (s >> 5) - (p.tp_smin[eg] >> 5);
      p.gmeta[at] = (static_cast<uint32_t>((eg - ebase) * g.planes * g.span + j0) << 5) | static_cast<uint32_t>(s & 31);
    }
  }
  return SND_OK;
}

// Direct tree kernel (tree_direct.cu): whether it applies to the plan, its instantiation and
// tile shape, and its tables. A CTA covers 32 consecutive trial DMs (lanes) and warps x kw
// output words; channels are staged 64 at a time. Per (DM tile, channel) the first staged ring
// word is base4 = (min over the tile of delta >> 5) rounded down to a multiple of 4 (16-byte
// aligned bulk copies), and per (tile, channel, DM) the 16-bit entry (delta >> 5) - base4 << 5 |
// delta & 31 gives the DM's window word and funnel shift.
void choose_direct_geometry(Plan& p) {
  snd::DirectGeom& g = p.dgeom;
  g = snd::DirectGeom{};
  p.direct = false;
  p.dmeta.clear();
  p.dbase.clear();
  if (p.mode == SND_MODE_ZFLOAT || (p.flags & (SND_FLAG_REFERENCE_TREE | SND_FLAG_LEAF_SHARING))) return;
  const int nchan = p.nchan, ndm = p.ndm;
  if (nchan % 64 != 0 || nchan >= 8192) return;
  int inst = snd::kDirNone, kw = 4;
  if (p.mode == SND_MODE_FLOAT) {
    inst = nchan < 2048 ? snd::kDirFloat11 : snd::kDirFloat13;
  } else if (p.mode == SND_MODE_GRADED) {
    // the exact level: the first level whose (full) nodes hold more than N channels; below it
    // every node value is its plain channel sum
    int sub = p.nlev - 1;
    int64_t width = p.C;
    for (int l = 0; l < p.nlev; ++l, width *= p.B) {
      if (std::min<int64_t>(width, nchan) > p.N) {
        sub = l;
        break;
      }
    }
    int64_t sub_ch = p.C;
    for (int l = 0; l < sub; ++l) sub_ch *= p.B;
    if (sub == p.nlev - 1) sub_ch = nchan;
    if (sub_ch % 64 != 0 || nchan % sub_ch != 0) return;
    int planes = 0;
    while ((int64_t(1) << planes) <= sub_ch) ++planes;
    const int up = p.nlev - 1 - sub;
    if (up == 0) {
      inst = planes <= 11 ? snd::kDirGraded11U0 : snd::kDirGraded13U0;
    } else if (planes <= 9 && up == 1) {
      inst = snd::kDirGraded9U1;
    } else if (planes <= 9 && up == 2) {
      inst = snd::kDirGraded9U2;
      kw = 2;
    } else {
      return;
    }
    g.sub_lev = sub;
    g.sub_groups = static_cast<int>(sub_ch / 64);
  } else {
    if (p.C != 4 || p.KL < 1 || p.KL > 4 || p.KI < 1 || p.KI > 2 || p.nlev < 2) return;
    const int up = p.nlev - 1;
    // regular trees (B = 2, 4 or 8): the levels inside a 16-leaf group as fixed logic; per-level
    // fire counts take the general state
    const int uin = p.B == 2 ? 4 : (p.B == 4 ? 2 : 1);
    const bool reg = (p.B == 2 || p.B == 4 || p.B == 8) && !(p.flags & SND_FLAG_LEVEL_RATES) && up >= uin &&
                     up - uin <= (p.B == 8 ? 3 : 4);
    if (reg) {
      if (p.B == 2)
        inst = p.KI == 1 ? snd::kDirBinReg2K1 : snd::kDirBinReg2K2;
      else if (p.B == 4)
        inst = p.KI == 1 ? snd::kDirBinReg4K1 : snd::kDirBinReg4K2;
      else
        inst = p.KI == 1 ? snd::kDirBinReg8K1 : snd::kDirBinReg8K2;
    } else if (up <= 4) {
      inst = snd::kDirBinary4;
    } else if (up <= 8) {
      inst = snd::kDirBinary8;
    } else if (up <= 12) {
      inst = snd::kDirBinary12;
      kw = 2;
    } else {
      return;
    }
  }
  g.kw = kw;
  g.warps = p.tree_warps ? p.tree_warps : 8;
  g.tile_words = g.warps * kw;
  int span_kw = kw;  // words per warp the staged windows must cover
  if ((p.flags & SND_FLAG_LEVEL_RATES) && p.mode != SND_MODE_BINARY) {
    // the binary counting pass (K_L = K_I = 1) on the same tables
    const int up = p.nlev - 1;
    if (p.C != 4 || up < 1 || up > 12) return;
    g.rates_inst = up <= 4 ? snd::kDirBinary4 : (up <= 8 ? snd::kDirBinary8 : snd::kDirBinary12);
    g.rates_kw = up <= 8 ? 4 : 2;
    span_kw = std::max(kw, g.rates_kw);
  }
  g.ndm_tiles = (ndm + 31) / 32;
  p.dbase.assign(static_cast<size_t>(g.ndm_tiles) * nchan, 0);
  int64_t omax = 0;
  for (int t = 0; t < g.ndm_tiles; ++t)
    for (int c = 0; c < nchan; ++c) {
      int32_t lo = INT32_MAX, hi = 0;
      for (int d = t * 32; d < std::min(ndm, t * 32 + 32); ++d) {
        const int32_t v = p.delays[static_cast<size_t>(d) * nchan + c];
        lo = std::min(lo, v);
        hi = std::max(hi, v);
      }
      const int32_t b4 = (lo >> 5) & ~3;
      p.dbase[static_cast<size_t>(t) * nchan + c] = b4;
      omax = std::max<int64_t>(omax, (hi >> 5) - b4);
    }
  if (omax > 2047) return;
  g.cspan = static_cast<int>(align_up(static_cast<size_t>(4 + omax + g.warps * span_kw), 4));
  // stage 128 channels per round (half the barriers) when they fit two CTAs per SM
  auto smem_for = [&](int sg) { return (2 * 64 * sg * static_cast<int64_t>(g.cspan) + 64 * sg * 32 + nchan) * 4; };
  if (p.tree_round == 64)
    g.sgroups = 1;
  else if (p.tree_round == 128)
    g.sgroups = nchan % 128 == 0 ? 2 : 1;
  else
    g.sgroups = (nchan % 128 == 0 && smem_for(2) <= 100 * 1024) ? 2 : 1;
  const int64_t smem = smem_for(g.sgroups);
  if (smem > 200 * 1024) return;
  g.smem_bytes = static_cast<int>(smem);
  p.dmeta.assign(static_cast<size_t>(g.ndm_tiles) * nchan * 32, 0);
  for (int t = 0; t < g.ndm_tiles; ++t)
    for (int c = 0; c < nchan; ++c) {
      const int32_t b4 = p.dbase[static_cast<size_t>(t) * nchan + c];
      for (int l = 0; l < 32; ++l) {
        const int d = std::min(ndm - 1, t * 32 + l);
        const int32_t v = p.delays[static_cast<size_t>(d) * nchan + c];
        p.dmeta[(static_cast<size_t>(t) * nchan + c) * 32 + l] =
            static_cast<uint16_t>((((v >> 5) - b4) << 5) | (v & 31));
      }
    }
  g.inst = inst;
  p.direct = true;
}

// Labelled-payload tree geometry: DMs per CTA, samples per CTA (32 lanes x samples per
// lane, in pairs; fewer samples for deeper trees so the per-level partial sums stay in registers), the
// first staged sample of each channel per DM tile (its smallest delay over the tile) and the
// widest staged window, leaves staged per shared-memory round, and the payload ring length.
int choose_ztree_geometry(Plan& p) {
  snd::ZGeom& z = p.zgeom;
  const int ndm = p.ndm, nchan = p.nchan, NL = p.nleaves;
  if (p.nlev > 16) return SND_ERR_UNSUPPORTED;
  z.fp16 = (p.flags & SND_FLAG_FP16_PARTIALS) ? 1 : 0;
  z.unit = (p.flags & SND_FLAG_UNIT_PAYLOAD) ? 1 : 0;
  z.maxl = p.nlev <= 4 ? 4 : (p.nlev <= 8 ? 8 : 16);
  z.spt = z.maxl == 4 ? 8 : (z.maxl == 8 ? 4 : 2);
  z.dms_per_cta = 16;
  z.tile_samples = 32 * z.spt;
  z.ndm_tiles = (ndm + z.dms_per_cta - 1) / z.dms_per_cta;
  p.zwb.assign(static_cast<size_t>(z.ndm_tiles) * nchan, 0);
  int64_t spread = 0;
  for (int t = 0; t < z.ndm_tiles; ++t) {
    const int d0 = t * z.dms_per_cta, d1 = std::min(ndm, d0 + z.dms_per_cta);
    for (int c = 0; c < nchan; ++c) {
      int32_t lo = p.delays[static_cast<size_t>(d0) * nchan + c], hi = lo;
      for (int d = d0 + 1; d < d1; ++d) {
        lo = std::min(lo, p.delays[static_cast<size_t>(d) * nchan + c]);
        hi = std::max(hi, p.delays[static_cast<size_t>(d) * nchan + c]);
      }
      p.zwb[static_cast<size_t>(t) * nchan + c] = lo;
      spread = std::max<int64_t>(spread, static_cast<int64_t>(hi) - lo);
    }
  }
  if (spread > (1 << 20)) return SND_ERR_UNSUPPORTED;
  const int es = z.fp16 ? 2 : 4;
  z.win = static_cast<int>(align_up(static_cast<size_t>(z.tile_samples + spread), 8));
  // per staged channel and buffer (two buffers: one filled while the other is read): its
  // window with a 16-byte alignment slack and one spare chunk, and the tile's DM offsets
  const int64_t wz = z.win + 2 * (16 / es);
  const int64_t per_chan = wz * es + 4 * z.dms_per_cta;
  const int64_t budget = 52 * 1024;
  int G = static_cast<int>(budget / (per_chan * p.C));
  if (G < 1) {
    G = 1;
    if (2 * per_chan * p.C > 200 * 1024) return SND_ERR_UNSUPPORTED;
  }
  z.group_leaves = std::min(G, NL);
  const int gc = z.group_leaves * p.C;
  z.smem_bytes = static_cast<int>(2 * (static_cast<size_t>(gc) * wz * es + static_cast<size_t>(4) * z.dms_per_cta * gc));
  // carry depth of each leaf: how many consecutive levels, from the leaves' parents up, it
  // finishes (while the node is the last child of its parent: the B-th or the ragged last)
  p.zcarry.assign(NL, 0);
  for (int k = 0; k < NL; ++k) {
    int i = k, depth = 0;
    for (int l = 0; l + 1 < p.nlev; ++l) {
      if (!((i % p.B == p.B - 1) || (i == p.level_nodes[l] - 1))) break;
      ++depth;
      i /= p.B;
    }
    p.zcarry[k] = depth;
  }
  // every emitted sample reads [E_prev, T_new): at most D + max_chunk samples back
  z.Rz = static_cast<int>(align_up(static_cast<size_t>(p.D) + p.max_chunk + 64, 8));
  return SND_OK;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

extern "C" int snd_plan_ex(const double* freqs_mhz, int32_t nchan, double dt_s,
                           const double* dm_grid, int32_t ndm, int32_t branching, snd_mode_t mode,
                           const snd_options_t* opts, snd_plan_t* out) {
  if (out) *out = nullptr;
  if (!out || !freqs_mhz || !dm_grid || nchan < 1 || ndm < 1 || branching < 2 || branching > 64)
    return SND_ERR_ARG;
  if (mode != SND_MODE_BINARY && mode != SND_MODE_GRADED && mode != SND_MODE_FLOAT && mode != SND_MODE_ZFLOAT)
    return SND_ERR_ARG;
  if (!finite_pos(dt_s)) return SND_ERR_ARG;
  if (nchan > 65536 || ndm > 65536) return SND_ERR_UNSUPPORTED;
  snd_options_t o;
  if (opts) {
    o = *opts;
  } else {
    snd_options_init(mode, &o);
  }
  if (o.flags & ~(SND_FLAG_REFERENCE_TREE | SND_FLAG_FP16_PARTIALS | SND_FLAG_LEAF_SHARING | SND_FLAG_UNIT_PAYLOAD |
                  SND_FLAG_LEVEL_RATES))
    return SND_ERR_ARG;
  if ((o.flags & SND_FLAG_LEVEL_RATES) && (mode == SND_MODE_ZFLOAT || (o.flags & SND_FLAG_REFERENCE_TREE)))
    return SND_ERR_UNSUPPORTED;
  if ((o.flags & (SND_FLAG_FP16_PARTIALS | SND_FLAG_UNIT_PAYLOAD)) && mode != SND_MODE_ZFLOAT) return SND_ERR_ARG;
  if ((o.flags & SND_FLAG_REFERENCE_TREE) && mode == SND_MODE_ZFLOAT) return SND_ERR_UNSUPPORTED;
  if (o.cluster_size < 1 || o.cluster_size > 7) return SND_ERR_UNSUPPORTED;
  if (mode == SND_MODE_BINARY && (o.k_leaf < 1 || o.k_leaf > 8 || o.k_internal < 1 || o.k_internal > 8))
    return SND_ERR_UNSUPPORTED;
  if (mode == SND_MODE_GRADED && (o.graded_cap < 1 || o.graded_cap > 255)) return SND_ERR_UNSUPPORTED;
  if (!std::isfinite(o.enc_theta) || !finite_pos(o.det_theta) || !std::isfinite(o.sigma_min) ||
      o.sigma_min < 0.0 || !std::isfinite(o.mf_alpha) || o.mf_alpha < 0.0)
    return SND_ERR_ARG;
  if (o.closing_size < 1 || o.closing_size > 31 || (o.closing_size & 1) == 0) return SND_ERR_ARG;
  if (o.plane_dtype < 0 || o.plane_dtype > 1 ||
      (o.plane_dtype == 1 && mode != SND_MODE_BINARY && mode != SND_MODE_GRADED))
    return SND_ERR_ARG;
  if ((o.tree_warps != 0 && o.tree_warps != 2 && o.tree_warps != 4 && o.tree_warps != 8) ||
      (o.tree_round != 0 && o.tree_round != 64 && o.tree_round != 128))
    return SND_ERR_ARG;
  if (o.n_min_pixels < 1 || o.max_chunk < 1 || o.max_chunk > (1 << 22) || o.cand_capacity < 1 ||
      o.cell_capacity < 1 || o.run_capacity < 1)
    return SND_ERR_ARG;
  for (int c = 0; c < nchan; ++c)
    if (!finite_pos(freqs_mhz[c])) return SND_ERR_FREQ_ORDER;
  {
    std::vector<double> f(freqs_mhz, freqs_mhz + nchan);
    std::sort(f.begin(), f.end());
    for (int c = 1; c < nchan; ++c)
      if (f[c] == f[c - 1]) return SND_ERR_FREQ_ORDER;
  }
  for (int d = 0; d < ndm; ++d)
    if (!std::isfinite(dm_grid[d]) || dm_grid[d] < 0.0) return SND_ERR_DM;

  Plan* p = nullptr;
  try {
    snd::alloc_point();
    p = new Plan();
  } catch (const std::bad_alloc&) {
    return SND_ERR_NOMEM;
  }
  try {
    p->nchan = nchan;
    p->ndm = ndm;
    p->mode = mode;
    p->B = branching;
    p->C = o.cluster_size;
    p->KL = o.k_leaf;
    p->KI = o.k_internal;
    p->N = o.graded_cap;
    p->dt = dt_s;
    p->enc_theta = o.enc_theta;
    p->det_theta = o.det_theta;
    p->sigma_min = o.sigma_min;
    p->mf_alpha = o.mf_alpha;
    p->closing = o.closing_size;
    p->n_min = o.n_min_pixels;
    p->max_chunk = o.max_chunk;
    p->cand_cap = o.cand_capacity;
    p->cell_cap = o.cell_capacity;
    p->run_cap = o.run_capacity;
    p->flags = o.flags;
    p->plane_u8 = o.plane_dtype;
    p->tree_warps = o.tree_warps;
    p->tree_round = o.tree_round;
    p->freqs.assign(freqs_mhz, freqs_mhz + nchan);
    p->dms.assign(dm_grid, dm_grid + ndm);
    int rc = snd::build_plan(*p);
    if (!rc && (p->flags & SND_FLAG_LEVEL_RATES) &&
        (!p->direct || p->C != 4 || (p->mode != SND_MODE_BINARY && p->dgeom.rates_inst == snd::kDirNone)))
      rc = SND_ERR_UNSUPPORTED;  // the fire counts come from the direct kernel's binary tree
    if (rc) {
      delete p;
      return rc;
    }
    // the matched filter stages one row segment (Wmax - 1 + chunk samples) in shared memory;
    // cell indices (row * nb + t) must fit 32 bits
    if ((static_cast<int64_t>(p->wmax) + p->max_chunk) * 4 + 4096 > 227 * 1024 ||
        static_cast<int64_t>(ndm) * p->Lp >= (int64_t(1) << 32)) {
      delete p;
      return SND_ERR_UNSUPPORTED;
    }
  } catch (const std::bad_alloc&) {
    delete p;
    return SND_ERR_NOMEM;
  } catch (...) {
    delete p;
    return SND_ERR_ARG;
  }
  *out = reinterpret_cast<snd_plan_t>(p);
  return SND_OK;
}

extern "C" int snd_plan(const double* freqs_mhz, int32_t nchan, double dt_s, const double* dm_grid,
                        int32_t ndm, int32_t branching, snd_mode_t mode, snd_plan_t* out) {
  return snd_plan_ex(freqs_mhz, nchan, dt_s, dm_grid, ndm, branching, mode, nullptr, out);
}

extern "C" size_t snd_workspace_size(snd_plan_t plan) {
  if (!plan) return 0;
  return reinterpret_cast<Plan*>(plan)->ws_bytes;
}

extern "C" int snd_plan_stats(snd_plan_t plan, snd_plan_stats_t* s) {
  if (!plan || !s) return SND_ERR_ARG;
  const Plan& p = *reinterpret_cast<Plan*>(plan);
  std::memset(s, 0, sizeof(*s));
  s->nchan = p.nchan;
  s->ndm = p.ndm;
  s->mode = p.mode;
  s->branching = p.B;
  s->cluster_size = p.C;
  s->max_delay = p.D;
  s->nlevels = p.nlev;
  for (int l = 0; l < p.nlev && l < 24; ++l) {
    s->nodes_per_level[l] = p.level_nodes[l];
    s->unique_per_level[l] = p.level_unique[l];
  }
  s->adds_per_dm_sample = p.adds_per_dm_sample;
  s->wmax = p.wmax;
  s->ring_words = p.R;
  s->hist_mem_bytes = p.hist_mem_bytes;
  s->workspace_bytes = p.ws_bytes;
  s->samples_in = p.T;
  s->emitted = p.E;
  s->scored = p.F;
  s->candidates_pending = p.pending_host;
  s->tree_tile_dms = p.geom.dms_per_cta;
  s->tree_tile_words = p.geom.tile_words;
  s->tree_group_leaves = p.geom.group_leaves;
  s->tree_smem_bytes = p.geom.smem_bytes;
  if (p.mode == SND_MODE_ZFLOAT) {
    s->tree_tile_dms = p.zgeom.dms_per_cta;
    s->tree_tile_words = p.zgeom.tile_samples / 32;
    s->tree_group_leaves = p.zgeom.group_leaves;
    s->tree_smem_bytes = p.zgeom.smem_bytes;
  }
  s->max_patterns_per_group = p.geom.max_pat_group;
  s->kernel_launches = p.launches;
  s->device_status = static_cast<int32_t>(p.last_status);
  s->tree_kernel = (p.mode == SND_MODE_ZFLOAT) ? 3 : (p.flags & SND_FLAG_REFERENCE_TREE) ? 2 : p.direct ? 1 : 0;
  if (p.direct) {
    s->tree_tile_dms = 32;
    s->tree_tile_words = p.dgeom.tile_words;
    s->tree_group_leaves = 64 / p.C;
    s->tree_smem_bytes = p.dgeom.smem_bytes;
  }
  return SND_OK;
}

extern "C" int snd_delay_table(snd_plan_t plan, int32_t* host_out, int64_t n) {
  if (!plan || !host_out) return SND_ERR_ARG;
  const Plan& p = *reinterpret_cast<Plan*>(plan);
  if (n < static_cast<int64_t>(p.delays.size())) return SND_ERR_ARG;
  std::memcpy(host_out, p.delays.data(), p.delays.size() * sizeof(int32_t));
  return SND_OK;
}

extern "C" void snd_destroy(snd_plan_t plan) {
  if (!plan) return;
  delete reinterpret_cast<Plan*>(plan);
}

extern "C" const char* snd_error_string(int status) {
  switch (status) {
    case SND_OK: return "ok";
    case SND_ERR_ARG: return "invalid argument";
    case SND_ERR_FREQ_ORDER: return "channel frequencies must be finite, positive and distinct";
    case SND_ERR_DM: return "trial DMs must be finite and non-negative";
    case SND_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case SND_ERR_CHUNK: return "chunk length outside 1..max_chunk";
    case SND_ERR_CUDA: return "CUDA runtime error";
    case SND_ERR_STATE: return "call not valid in the plan's current state";
    case SND_ERR_TIMEOUT: return "bounded device loop gave up";
    case SND_ERR_OVERFLOW: return "device list capacity overflowed";
    case SND_ERR_NOMEM: return "host allocation failed";
    case SND_ERR_UNSUPPORTED: return "configuration not supported by the GPU kernels";
    default: return "unknown status";
  }
}
