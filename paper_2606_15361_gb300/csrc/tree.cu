// SND delay-and-add tree on the GPU (Methods, "The Spiking Neural Dedispersion algorithm",
// "Tree activation modes").
//
// Semantics, per trial DM d and output time t (a_c = x_c(t + delta_c(d))):
//   leaf (C contiguous channels): s = sum a_c ; node of B children: s = sum of child values
//   Mode A: v = 1[s >= K_L] at leaves, 1[s >= K_I] above; Mode B: v = min(s, N) at every
//   node; Mode C: v = s. The plane holds the root value (Mode C: the integer root count,
//   scaled by 1/sqrt(N_f) only when written to the caller's float plane).
// Every inter-node shift is a difference of the globally rounded delays, so each channel
// is read at exactly t + delta_c(d) and the whole tree of one DM is evaluated at one
// output time ("absolute time" form): no shifts above the leaves.
//
// GPU design (k_tree):
//  * 32 output samples per 32-bit word, one bit plane per value bit (bit-sliced), so one
//    logic instruction advances 32 samples. Binary nodes keep a thermometer code of the
//    child count, graded nodes a saturating 8-plane counter, float a plain counter.
//  * A CTA owns DT consecutive trial DMs (one warp each, lanes = consecutive words, so all
//    shared-memory gathers are conflict-free) and 32*KW output words.
//  * Leaf sharing (the paper's unique leaf neurons): within the CTA's DM tile each leaf has
//    only a few distinct integer-delay patterns. Phase 1 evaluates each distinct
//    (leaf, pattern) series once into shared memory, reading the L2-resident bit ring;
//    phase 2 has every DM gather its leaf values from those series at its own leaf shift
//    (one funnel shift per plane and word) and push them up its tree.
//  * Leaves are processed in groups sized to the shared-memory budget; the per-DM tree
//    state (one accumulator per open level) stays in registers across groups.

#include <cuda_pipeline.h>

#include <vector>

#include "snd_internal.h"

namespace snd {
namespace {

struct TreeArgs {
  const uint32_t* ring;
  int R, nchan, ndm, nleaves;
  int C, B, KL, KI, N, nlev;
  int level_nodes[kMaxLevels];
  const int32_t* tp_off;   // [ndm_tiles * nleaves + 1] first (tile, leaf) entry of each leaf
  const uint32_t* gepk;    // [entries][C] window word offset << 5 | bit shift of each entry channel
  const int32_t* gleaf;    // [entries] leaf of each entry, relative to its group's first leaf
  const uint32_t* gmeta;   // [ndm][nleaves] series word offset << 5 | bit shift of (DM, leaf)
  const int32_t* tile_wb;  // [ndm_tiles][nchan] first staged ring word of each channel, relative to the tile
  int G, span, cspan, maxpat;
  int tile_words;   // output words per CTA (<= 32*KW)
  int plain1;       // graded: the cap cannot bind inside a level-1 node
  int span_extra;   // leaf-series words beyond tile_words
  long long word0;  // absolute index of the first output word
  int nwords;       // output words of this call
  int32_t* plane;
  int Lp;
};

constexpr int kMaxBatchBeams = 64;

struct TreeMulti {
  int nbeams;
  int first[kMaxBatchBeams];  // first CTA of each beam
  int ntx[kMaxBatchBeams];    // time tiles of each beam
  TreeArgs beam[kMaxBatchBeams];
};

__device__ __forceinline__ uint32_t funnel(uint32_t lo, uint32_t hi, int sh) {
  return __funnelshift_r(lo, hi, sh);
}

// a[0..ND) += b[0..NS), ripple carry; returns the carry out of the top plane.
template <int ND, int NS>
__device__ __forceinline__ uint32_t add_planes(uint32_t* a, const uint32_t* b) {
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const uint32_t x = a[i], y = b[i];
    a[i] = x ^ y ^ c;
    c = (x & y) | (c & (x ^ y));
  }
#pragma unroll
  for (int i = NS; i < ND; ++i) {
    const uint32_t x = a[i];
    a[i] = x ^ c;
    c = x & c;
  }
  return c;
}

// Clamp a bit-sliced NP-plane value to n (lanes where value > n, or over = 1, become n).
template <int NP>
__device__ __forceinline__ void clamp_planes(uint32_t* a, uint32_t over, int n) {
  uint32_t gt = 0, eq = 0xFFFFFFFFu;
#pragma unroll
  for (int p = NP - 1; p >= 0; --p) {
    if ((n >> p) & 1) {
      eq &= a[p];
    } else {
      gt |= eq & a[p];
      eq &= ~a[p];
    }
  }
  gt |= over;
#pragma unroll
  for (int p = 0; p < NP; ++p) a[p] = ((n >> p) & 1) ? (a[p] | gt) : (a[p] & ~gt);
}

// In-register transpose of a 32x32 bit matrix: bit c of m[r] <-> bit r of m[c].
__device__ __forceinline__ void transpose32(uint32_t* m) {
  uint32_t mask = 0x0000FFFFu;
#pragma unroll
  for (int j = 16; j != 0; j >>= 1, mask ^= (mask << j)) {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      if (k & j) continue;
      const uint32_t t = ((m[k] >> j) ^ m[k + j]) & mask;
      m[k + j] ^= t;
      m[k] ^= t << j;
    }
  }
}

// Write the 32 samples of one output word (value planes -> int32) to a 128-byte-aligned slot.
template <int NP>
__device__ __forceinline__ void store_word(int32_t* dst, const uint32_t* planes) {
  uint32_t m[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) m[i] = (i < NP) ? planes[i < NP ? i : 0] : 0u;
  transpose32(m);
  int4* d4 = reinterpret_cast<int4*>(dst);
#pragma unroll
  for (int i = 0; i < 8; ++i)
    d4[i] = make_int4(static_cast<int>(m[4 * i]), static_cast<int>(m[4 * i + 1]),
                      static_cast<int>(m[4 * i + 2]), static_cast<int>(m[4 * i + 3]));
}

__device__ __forceinline__ void store_bits(int32_t* dst, uint32_t v) {
  int4* d4 = reinterpret_cast<int4*>(dst);
#pragma unroll
  for (int i = 0; i < 8; ++i)
    d4[i] = make_int4((v >> (4 * i)) & 1, (v >> (4 * i + 1)) & 1, (v >> (4 * i + 2)) & 1,
                      (v >> (4 * i + 3)) & 1);
}

constexpr int kBinary = SND_MODE_BINARY, kGraded = SND_MODE_GRADED, kFloat = SND_MODE_FLOAT;

// Bit-sliced count of up to 7 one-bit inputs (3 planes). NC is the compile-time channel
// bound: NC = 4 for clusters of exactly four channels, 8 for the generic (predicated) path.
template <int NC>
__device__ __forceinline__ void count7(const uint32_t* x, int cs, uint32_t* c) {
  c[0] = c[1] = c[2] = 0;
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    if (NC != 8 || i < cs) {
      const uint32_t k0 = c[0] & x[i];
      c[0] ^= x[i];
      const uint32_t k1 = c[1] & k0;
      c[1] ^= k0;
      c[2] |= k1;
    }
  }
}

// Per-warp tree state: DPW trial DMs x KW words per lane. Level 1 is accumulated per node
// (all of its leaves in one go); levels >= 2 keep one accumulator per open node.
template <int MODE, int MAXL, int KW, int TH, int DPW>
struct Tree;

// Mode A: thermometer codes, acc[..][i] = 1[count >= i+1].
template <int MAXL, int KW, int TH, int DPW>
struct Tree<kBinary, MAXL, KW, TH, DPW> {
  static constexpr int kLeafPlanes = 1;
  uint32_t acc[MAXL][DPW][KW][TH];
  uint32_t root[DPW][KW];
  uint32_t ksel[TH];  // one-hot masks selecting the K_I plane (keeps acc in registers)
  int cnt[MAXL], node[MAXL], fan[MAXL];

  __device__ __forceinline__ void init(const TreeArgs& a) {
#pragma unroll
    for (int i = 0; i < TH; ++i) ksel[i] = (i == a.KI - 1) ? 0xFFFFFFFFu : 0u;
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
#pragma unroll
      for (int d = 0; d < DPW; ++d)
#pragma unroll
        for (int j = 0; j < KW; ++j)
#pragma unroll
          for (int i = 0; i < TH; ++i) acc[l][d][j][i] = 0;
      cnt[l] = 0;
      node[l] = 0;
      fan[l] = (l >= 2 && l < a.nlev) ? min(a.B, a.level_nodes[l - 1]) : 1;
    }
#pragma unroll
    for (int d = 0; d < DPW; ++d)
#pragma unroll
      for (int j = 0; j < KW; ++j) root[d][j] = 0;
  }
  // leaf: quorum K_L over the cluster's channel bits
  template <int NC>
  __device__ __forceinline__ static void leaf(const TreeArgs& a, const uint32_t* x, int cs, uint32_t* out) {
    uint32_t t[TH];  // TH >= K_L
#pragma unroll
    for (int i = 0; i < TH; ++i) t[i] = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (NC != 8 || c < cs) {
#pragma unroll
        for (int i = TH - 1; i > 0; --i) t[i] |= t[i - 1] & x[c];
        t[0] |= x[c];
      }
    }
    uint32_t r = 0;
#pragma unroll
    for (int i = 0; i < TH; ++i) r |= t[i] & ((i == a.KL - 1) ? 0xFFFFFFFFu : 0u);
    out[0] = r;
  }
  // level-1 node accumulator for one DM
  struct Node {
    uint32_t t[KW][TH];
  };
  __device__ __forceinline__ static void node_clear(Node& n) {
#pragma unroll
    for (int j = 0; j < KW; ++j)
#pragma unroll
      for (int i = 0; i < TH; ++i) n.t[j][i] = 0;
  }
  __device__ __forceinline__ static void node_add(Node& n, int j, const uint32_t* v) {
#pragma unroll
    for (int i = TH - 1; i > 0; --i) n.t[j][i] |= n.t[j][i - 1] & v[0];
    n.t[j][0] |= v[0];
  }
  __device__ __forceinline__ uint32_t select_k(const uint32_t* t) const {
    uint32_t r = 0;
#pragma unroll
    for (int i = 0; i < TH; ++i) r |= t[i] & ksel[i];
    return r;
  }
  // all DMs of the warp finished level-1 node n: push their values up
  __device__ __forceinline__ void push_nodes(const TreeArgs& a, Node (&nd)[DPW]) {
    uint32_t cur[DPW][KW];
#pragma unroll
    for (int d = 0; d < DPW; ++d)
#pragma unroll
      for (int j = 0; j < KW; ++j) cur[d][j] = select_k(nd[d].t[j]);
    if (a.nlev == 2) {
#pragma unroll
      for (int d = 0; d < DPW; ++d)
#pragma unroll
        for (int j = 0; j < KW; ++j) root[d][j] = cur[d][j];
      return;
    }
#pragma unroll
    for (int l = 2; l < MAXL; ++l) {
      if (l >= a.nlev) break;
#pragma unroll
      for (int d = 0; d < DPW; ++d)
#pragma unroll
        for (int j = 0; j < KW; ++j) {
#pragma unroll
          for (int i = TH - 1; i > 0; --i) acc[l][d][j][i] |= acc[l][d][j][i - 1] & cur[d][j];
          acc[l][d][j][0] |= cur[d][j];
        }
      if (++cnt[l] < fan[l]) break;
#pragma unroll
      for (int d = 0; d < DPW; ++d)
#pragma unroll
        for (int j = 0; j < KW; ++j) {
          cur[d][j] = select_k(acc[l][d][j]);
#pragma unroll
          for (int i = 0; i < TH; ++i) acc[l][d][j][i] = 0;
        }
      cnt[l] = 0;
      ++node[l];
      fan[l] = min(a.B, a.level_nodes[l - 1] - a.B * node[l]);
      if (l == a.nlev - 1) {
#pragma unroll
        for (int d = 0; d < DPW; ++d)
#pragma unroll
          for (int j = 0; j < KW; ++j) root[d][j] = cur[d][j];
      }
    }
  }
  __device__ __forceinline__ void set_root_leaf(int d, int j, const uint32_t* v) { root[d][j] = v[0]; }
  __device__ __forceinline__ void finish() {}
  __device__ __forceinline__ void store(int32_t* dst, int d, int j) const { store_bits(dst, root[d][j]); }
};

// Mode B: saturating 8-plane counters, min(sum, N) at every node.
template <int MAXL, int KW, int TH, int DPW>
struct Tree<kGraded, MAXL, KW, TH, DPW> {
  static constexpr int kLeafPlanes = 3;
  uint32_t acc[MAXL][DPW][KW][8];
  uint32_t root[DPW][KW][8];
  int cnt[MAXL], node[MAXL], fan[MAXL];

  __device__ __forceinline__ void init(const TreeArgs& a) {
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
#pragma unroll
      for (int d = 0; d < DPW; ++d)
#pragma unroll
        for (int j = 0; j < KW; ++j)
#pragma unroll
          for (int p = 0; p < 8; ++p) acc[l][d][j][p] = 0;
      cnt[l] = 0;
      node[l] = 0;
      fan[l] = (l >= 2 && l < a.nlev) ? min(a.B, a.level_nodes[l - 1]) : 1;
    }
#pragma unroll
    for (int d = 0; d < DPW; ++d)
#pragma unroll
      for (int j = 0; j < KW; ++j)
#pragma unroll
        for (int p = 0; p < 8; ++p) root[d][j][p] = 0;
  }
  template <int NC>
  __device__ __forceinline__ static void leaf(const TreeArgs& a, const uint32_t* x, int cs, uint32_t* out) {
    count7<NC>(x, cs, out);
    if (a.N < 7) clamp_planes<3>(out, 0u, a.N);
  }
  struct Node {
    uint32_t p[KW][8];
  };
  __device__ __forceinline__ static void node_clear(Node& n) {
#pragma unroll
    for (int j = 0; j < KW; ++j)
#pragma unroll
      for (int p = 0; p < 8; ++p) n.p[j][p] = 0;
  }
  // level-1 node: add a 3-plane leaf value. When B*min(C,N) <= min(N, 63) the cap cannot
  // bind inside a level-1 node and the sum fits 6 planes (plain add); otherwise saturate.
  __device__ __forceinline__ static void node_add_sat(Node& n, int j, const uint32_t* v, int N, bool plain) {
    if (plain) {
      add_planes<6, 3>(n.p[j], v);
      return;
    }
    const uint32_t over = add_planes<8, 3>(n.p[j], v);
    if (N == 255) {
#pragma unroll
      for (int p = 0; p < 8; ++p) n.p[j][p] |= over;
    } else {
      clamp_planes<8>(n.p[j], over, N);
    }
  }
  __device__ __forceinline__ static void add_sat8(uint32_t* acc, const uint32_t* v, int N) {
    const uint32_t over = add_planes<8, 8>(acc, v);
    if (N == 255) {
#pragma unroll
      for (int p = 0; p < 8; ++p) acc[p] |= over;
    } else {
      clamp_planes<8>(acc, over, N);
    }
  }
  __device__ __forceinline__ void push_nodes(const TreeArgs& a, Node (&nd)[DPW]) {
    if (a.nlev == 2) {
#pragma unroll
      for (int d = 0; d < DPW; ++d)
#pragma unroll
        for (int j = 0; j < KW; ++j)
#pragma unroll
          for (int p = 0; p < 8; ++p) root[d][j][p] = nd[d].p[j][p];
      return;
    }
    uint32_t cur[DPW][KW][8];
#pragma unroll
    for (int d = 0; d < DPW; ++d)
#pragma unroll
      for (int j = 0; j < KW; ++j)
#pragma unroll
        for (int p = 0; p < 8; ++p) cur[d][j][p] = nd[d].p[j][p];
#pragma unroll
    for (int l = 2; l < MAXL; ++l) {
      if (l >= a.nlev) break;
#pragma unroll
      for (int d = 0; d < DPW; ++d)
#pragma unroll
        for (int j = 0; j < KW; ++j) add_sat8(acc[l][d][j], cur[d][j], a.N);
      if (++cnt[l] < fan[l]) break;
#pragma unroll
      for (int d = 0; d < DPW; ++d)
#pragma unroll
        for (int j = 0; j < KW; ++j)
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            cur[d][j][p] = acc[l][d][j][p];
            acc[l][d][j][p] = 0;
          }
      cnt[l] = 0;
      ++node[l];
      fan[l] = min(a.B, a.level_nodes[l - 1] - a.B * node[l]);
      if (l == a.nlev - 1) {
#pragma unroll
        for (int d = 0; d < DPW; ++d)
#pragma unroll
          for (int j = 0; j < KW; ++j)
#pragma unroll
            for (int p = 0; p < 8; ++p) root[d][j][p] = cur[d][j][p];
      }
    }
  }
  __device__ __forceinline__ void set_root_leaf(int d, int j, const uint32_t* v) {
#pragma unroll
    for (int p = 0; p < 8; ++p) root[d][j][p] = (p < 3) ? v[p < 3 ? p : 0] : 0u;
  }
  __device__ __forceinline__ void finish() {}
  __device__ __forceinline__ void store(int32_t* dst, int d, int j) const { store_word<8>(dst, root[d][j]); }
};

// Mode C: no node rule, so the root count is the sum of all leaf counts: node sums of up to
// eight leaves (6 planes) are added into a 16-plane counter per (DM, word).
template <int MAXL, int KW, int TH, int DPW>
struct Tree<kFloat, MAXL, KW, TH, DPW> {
  static constexpr int kLeafPlanes = 3;
  uint32_t root[DPW][KW][16];
  __device__ __forceinline__ void init(const TreeArgs&) {
#pragma unroll
    for (int d = 0; d < DPW; ++d)
#pragma unroll
      for (int j = 0; j < KW; ++j)
#pragma unroll
        for (int p = 0; p < 16; ++p) root[d][j][p] = 0;
  }
  template <int NC>
  __device__ __forceinline__ static void leaf(const TreeArgs&, const uint32_t* x, int cs, uint32_t* out) {
    count7<NC>(x, cs, out);
  }
  struct Node {};  // float needs no per-node state
  __device__ __forceinline__ void add_node(int d, int j, const uint32_t* s6) { add_planes<16, 6>(root[d][j], s6); }
  __device__ __forceinline__ void finish() {}
  __device__ __forceinline__ void store(int32_t* dst, int d, int j) const { store_word<16>(dst, root[d][j]); }
};

// z[0..N] = x[0..N) + y[0..N) (ripple carry; N+1 planes out)
template <int N>
__device__ __forceinline__ void add2(const uint32_t* x, const uint32_t* y, uint32_t* z) {
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const uint32_t a = x[i], b = y[i];
    z[i] = a ^ b ^ c;
    c = (a & b) | (c & (a ^ b));
  }
  z[N] = c;
}

// Sum of eight 3-plane values by a pairwise adder tree (3+3 -> 4, 4+4 -> 5, 5+5 -> 6 planes):
// about 50 logic operations instead of ~96 for eight sequential adds into a 6-plane counter.
__device__ __forceinline__ void sum8(const uint32_t (&v)[8][3], uint32_t* out6) {
  uint32_t a[4][4], b[2][5];
#pragma unroll
  for (int i = 0; i < 4; ++i) add2<3>(v[2 * i], v[2 * i + 1], a[i]);
#pragma unroll
  for (int i = 0; i < 2; ++i) add2<4>(a[2 * i], a[2 * i + 1], b[i]);
  add2<5>(b[0], b[1], out6);
}

// k_tree: CTA = NW warps x DPW trial DMs each (DT = NW*DPW consecutive DMs) x tile_words
// output words. Per group of G leaves (a multiple of B, so level-1 nodes never straddle):
//   1. stage the group's channel windows from the mirrored bit ring into shared memory;
//   2. phase 1: one warp per distinct (leaf, pattern) entry, lanes over words: evaluate the
//      leaf's series once (the paper's unique leaf neuron for this DM tile);
//   3. phase 2: every warp gathers, for each of its DMs and each level-1 node of the group,
//      the node's leaf values at the DM's own leaf shifts (one funnel shift per plane and
//      word) and pushes the finished node values up the tree.
// One CTA of the tree: time tile bx (tile_words output words) of DM tile `tile`.
template <int MODE, int MAXL, int KW, int TH, int DPW, int CT>
__device__ __forceinline__ void tree_cta(const TreeArgs& a, int bx, int tile) {
  using T = Tree<MODE, MAXL, KW, TH, DPW>;
  constexpr int PL = T::kLeafPlanes;
  constexpr int NC = CT ? CT : 8;  // channels per leaf iterated at compile time
  extern __shared__ __align__(16) uint32_t sm[];
  const int NW = blockDim.y;
  const int DT = NW * DPW;
  const int lane = threadIdx.x, wd = threadIdx.y;
  const int tid = wd * 32 + lane, nthr = 32 * NW;
  const long long aw0 = a.word0 + static_cast<long long>(bx) * a.tile_words;
  const int awp = static_cast<int>(aw0 % a.R);
  const int NL = a.nleaves, C = a.C, G = a.G, span = a.span, cspan = a.cspan;
  // words this CTA emits: the chunk's last time tile may hold fewer than tile_words (a chunk
  // whose emitted range is not word-aligned spans one word more than its length / 32), and
  // its series, staged windows and phase-2 words shrink with it
  const int tw_eff = min(a.tile_words, static_cast<int>(a.nwords - static_cast<long long>(bx) * a.tile_words));
  const int span_eff = min(span, tw_eff + a.span_extra);
  const int cspan_eff = min(cspan, tw_eff + (cspan - a.tile_words) + 1);

  // leaf series are stored as word pairs (w[j], w[j+1]) so a gather is one 64-bit load
  // shared memory: leaf series (word pairs) + two staging buffers, each holding one group's
  // channel windows, per-(DM, leaf) offsets and per-entry channel offsets/leaves; the next
  // group's buffer is filled with cp.async while the current group computes
  uint2* ser = reinterpret_cast<uint2*>(sm);                                 // maxpat*PL*span pairs
  const int win_w = G * C * cspan, meta_w = DT * G, epk_w = a.maxpat * C;
  const int buf_w = (win_w + meta_w + epk_w + a.maxpat + 3) & ~3;
  uint32_t* bufs = sm + 2 * a.maxpat * PL * span;
  // window base word of every channel for this DM tile, read once per CTA
  int* swb = reinterpret_cast<int*>(bufs + 2 * buf_w);
  for (int c = tid; c < a.nchan; c += nthr) swb[c] = a.tile_wb[tile * a.nchan + c];
  __syncthreads();

  T st;
  st.init(a);
  const bool plain1 = a.plain1 != 0;

  auto prefetch = [&](int g0, int b) {
    const int g1 = min(NL, g0 + G);
    const int ng = g1 - g0;
    const int c_lo = g0 * C, c_hi = min(a.nchan, g1 * C);
    const int ebase = a.tp_off[tile * NL + g0];
    const int ne = a.tp_off[tile * NL + g1] - ebase;
    uint32_t* win = bufs + b * buf_w;
    uint32_t* meta = win + win_w;
    uint32_t* epk = meta + meta_w;
    uint32_t* eleaf = epk + epk_w;
    for (int cl = wd; cl < c_hi - c_lo; cl += NW) {
      const int c = c_lo + cl;
      const uint32_t* row = a.ring + static_cast<size_t>(c) * 2 * a.R + awp + swb[c];
      for (int j = lane; j < cspan_eff; j += 32) __pipeline_memcpy_async(win + cl * cspan + j, row + j, 4);
    }
    for (int dl = wd; dl < DT; dl += NW) {
      const uint32_t* src = a.gmeta + static_cast<size_t>(min(tile * DT + dl, a.ndm - 1)) * NL + g0;
      for (int kl = lane; kl < ng; kl += 32) __pipeline_memcpy_async(meta + dl * G + kl, src + kl, 4);
    }
    for (int i = tid; i < ne * C; i += nthr)
      __pipeline_memcpy_async(epk + i, a.gepk + static_cast<size_t>(ebase) * C + i, 4);
    for (int i = tid; i < ne; i += nthr) __pipeline_memcpy_async(eleaf + i, a.gleaf + ebase + i, 4);
    __pipeline_commit();
  };

  prefetch(0, 0);
  for (int g0 = 0, gi = 0; g0 < NL; g0 += G, ++gi) {
    const int g1 = min(NL, g0 + G);
    const int ng = g1 - g0;
    const int ebase = a.tp_off[tile * NL + g0];
    const int ne = a.tp_off[tile * NL + g1] - ebase;
    const int b = gi & 1;
    if (g1 < NL) {
      prefetch(g1, b ^ 1);
      __pipeline_wait_prior(1);
    } else {
      __pipeline_wait_prior(0);
    }
    const uint32_t* win = bufs + b * buf_w;
    const uint32_t* meta = win + win_w;
    const uint32_t* epk = meta + meta_w;
    const int* eleaf = reinterpret_cast<const int*>(epk + epk_w);
    (void)ng;
    __syncthreads();
    // 2. phase 1: distinct (leaf, pattern) series. Full 32-word chunks: one entry per warp,
    //    lanes over words. The short remainders (span_eff mod 32 words) of several entries
    //    share one warp pass, lane l taking word l mod tl of entry l / tl of the pass.
    const int main_w = span_eff & ~31, tl = span_eff & 31;
    uint32_t pk[NC];
    const uint32_t* wch[NC];
    int cs = 0;
    uint2* out = ser;
    auto entry = [&](int e) {  // channel offsets and series of entry e
      const int kl = eleaf[e];
      cs = CT ? CT : min(C, a.nchan - (g0 + kl) * C);
#pragma unroll
      for (int ci = 0; ci < NC; ++ci) {
        pk[ci] = (CT || ci < cs) ? epk[e * C + ci] : 0u;
        wch[ci] = win + (kl * C + ci) * cspan + (pk[ci] >> 5);
      }
      out = ser + e * PL * span;
    };
    auto series_word = [&](int j) {  // word j of the current entry's series, as word pairs
      uint32_t x[NC];
#pragma unroll
      for (int ci = 0; ci < NC; ++ci)
        x[ci] = (CT || ci < cs) ? funnel(wch[ci][j], wch[ci][j + 1], pk[ci] & 31) : 0u;
      uint32_t v[PL];
      T::template leaf<NC>(a, x, cs, v);
#pragma unroll
      for (int p = 0; p < PL; ++p) {
        out[p * span + j].x = v[p];
        if (j > 0) out[p * span + j - 1].y = v[p];
      }
    };
    for (int e = wd; e < ne; e += NW) {
      entry(e);
      for (int j = lane; j < main_w; j += 32) series_word(j);
    }
    if (tl > 0) {
      const int epi = 32 / tl;  // entries per pass
      const int el = lane / tl, jl = lane - el * tl;
      for (int e0 = wd * epi; e0 < ne; e0 += NW * epi) {
        const int e = e0 + el;
        if (el < epi && e < ne) {
          entry(e);
          series_word(main_w + jl);
        }
      }
    }
    __syncthreads();
    // 3. phase 2
    if constexpr (MODE != kBinary) {
      if (MODE == kGraded && a.nlev == 1) {
        // a single leaf is the root
#pragma unroll
        for (int d = 0; d < DPW; ++d) {
          const uint32_t m = meta[(wd * DPW + d) * G];
          const uint2* base = ser + (m >> 5);
#pragma unroll
          for (int jw = 0; jw < KW; ++jw) {
            uint32_t v[PL];
#pragma unroll
            for (int p = 0; p < PL; ++p) {
              const uint2 q = base[p * span + lane + 32 * jw];
              v[p] = funnel(q.x, q.y, m & 31);
            }
            if constexpr (MODE == kGraded) st.set_root_leaf(d, jw, v);
          }
        }
      } else {
        // float groups leaves by eight (its result does not depend on the tree); graded
        // follows the level-1 nodes of B leaves
        const int nstep = (MODE == kFloat) ? 8 : a.B;
        const bool plain = (MODE == kFloat) || plain1;
        for (int k0 = g0; k0 < g1; k0 += nstep) {
          const int n = min(g1, k0 + nstep) - k0;
          typename T::Node nd[DPW];
#pragma unroll
          for (int d = 0; d < DPW; ++d) {
            const uint32_t* mrow = meta + (wd * DPW + d) * G + (k0 - g0);
#pragma unroll
            for (int jw = 0; jw < KW; ++jw) {
              const int w = lane + 32 * jw;
              uint32_t s8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
              const bool live = 32 * jw < tw_eff;  // words [32 jw, 32 jw + 32) are emitted here
              if (!live) {
              } else if (plain && n == 8) {
                uint32_t v[8][3];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                  const uint32_t m = mrow[i];
                  const uint2* base = ser + (m >> 5);
#pragma unroll
                  for (int p = 0; p < 3; ++p) {
                    const uint2 q = base[p * span + w];
                    v[i][p] = funnel(q.x, q.y, m & 31);
                  }
                }
                sum8(v, s8);
              } else {
                for (int i = 0; i < n; ++i) {
                  const uint32_t m = mrow[i];
                  const uint2* base = ser + (m >> 5);
                  uint32_t v[3];
#pragma unroll
                  for (int p = 0; p < 3; ++p) {
                    const uint2 q = base[p * span + w];
                    v[p] = funnel(q.x, q.y, m & 31);
                  }
                  if (plain) {
                    add_planes<6, 3>(s8, v);
                  } else {
                    const uint32_t over = add_planes<8, 3>(s8, v);
                    if constexpr (MODE == kGraded) {
                      if (a.N == 255) {
#pragma unroll
                        for (int p = 0; p < 8; ++p) s8[p] |= over;
                      } else {
                        clamp_planes<8>(s8, over, a.N);
                      }
                    }
                  }
                }
              }
              if constexpr (MODE == kFloat) {
                if (live) st.add_node(d, jw, s8);
              } else {
#pragma unroll
                for (int p = 0; p < 8; ++p) nd[d].p[jw][p] = s8[p];
              }
            }
          }
          if constexpr (MODE == kGraded) st.push_nodes(a, nd);
        }
      }
    } else {
      if (a.nlev == 1) {
        // a single leaf is the root
#pragma unroll
        for (int d = 0; d < DPW; ++d) {
          const uint32_t m = meta[(wd * DPW + d) * G];
          const uint2* base = ser + (m >> 5);
#pragma unroll
          for (int jw = 0; jw < KW; ++jw) {
            const int w = lane + 32 * jw;
            uint32_t v[PL];
#pragma unroll
            for (int p = 0; p < PL; ++p) {
              const uint2 q = base[p * span + w];
              v[p] = funnel(q.x, q.y, m & 31);
            }
            st.set_root_leaf(d, jw, v);
          }
        }
      } else {
        for (int k0 = g0; k0 < g1; k0 += a.B) {
          const int k1 = min(g1, k0 + a.B);
          typename T::Node nd[DPW];
#pragma unroll
          for (int d = 0; d < DPW; ++d) {
            T::node_clear(nd[d]);
            for (int k = k0; k < k1; ++k) {
              const uint32_t m = meta[(wd * DPW + d) * G + (k - g0)];
              const uint2* base = ser + (m >> 5);
              const int sh = m & 31;
#pragma unroll
              for (int jw = 0; jw < KW; ++jw) {
                if (32 * jw >= tw_eff) continue;  // no emitted word in this lane slot
                const int w = lane + 32 * jw;
                uint32_t v[PL];
#pragma unroll
                for (int p = 0; p < PL; ++p) {
                  const uint2 q = base[p * span + w];
                  v[p] = funnel(q.x, q.y, sh);
                }
                if constexpr (MODE == kBinary) {
                  T::node_add(nd[d], jw, v);
                } else {
                  T::node_add_sat(nd[d], jw, v, a.N, plain1);
                }
              }
            }
          }
          st.push_nodes(a, nd);
        }
      }
    }
    __syncthreads();
  }
  st.finish();
  const int lw = a.Lp >> 5;
#pragma unroll
  for (int d = 0; d < DPW; ++d) {
    const int drow = tile * DT + wd * DPW + d;
    if (drow >= a.ndm) continue;
#pragma unroll
    for (int jw = 0; jw < KW; ++jw) {
      const int w = lane + 32 * jw;
      const long long aw = aw0 + w;
      if (w >= a.tile_words || aw - a.word0 >= a.nwords) continue;
      const int col = static_cast<int>(aw % lw) * 32;
      st.store(a.plane + static_cast<size_t>(drow) * a.Lp + col, d, jw);
    }
  }
}

#define SND_TREE_BOUNDS                                                                   \
  __launch_bounds__((MODE != kBinary && DPW == 1 && MAXL == 4 && KW == 1) ? 1024 : 512, \
                    (MODE == kBinary && TH == 2) ? 2 : 1)

template <int MODE, int MAXL, int KW, int TH, int DPW, int CT>
__global__ void SND_TREE_BOUNDS k_tree(const __grid_constant__ TreeArgs a) {
  tree_cta<MODE, MAXL, KW, TH, DPW, CT>(a, blockIdx.x, blockIdx.y);
}

// Several beams (plans with the same kernel instantiation) in one launch: CTA i belongs to
// the last beam with first[b] <= i; within a beam, CTAs run time tile fastest.
template <int MODE, int MAXL, int KW, int TH, int DPW, int CT>
__global__ void SND_TREE_BOUNDS k_tree_multi(const __grid_constant__ TreeMulti m) {
  const int i = static_cast<int>(blockIdx.x);
  int lo = 0, hi = m.nbeams - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (m.first[mid] <= i) lo = mid; else hi = mid - 1;
  }
  const int local = i - m.first[lo];
  tree_cta<MODE, MAXL, KW, TH, DPW, CT>(m.beam[lo], local % m.ntx[lo], local / m.ntx[lo]);
}

// Scalar verification kernel: one thread per (DM, output sample), the tree walked leaf by
// leaf with integer counts straight from the full delay table. Slow; selected by
// SND_FLAG_REFERENCE_TREE to cross-check k_tree.
struct RefArgs {
  const uint32_t* ring;
  int R, nchan, ndm, nleaves;
  int C, B, KL, KI, N, nlev, mode;
  int level_nodes[kMaxLevels];
  const int32_t* delays;
  long long e_prev, e_new;
  int32_t* plane;
  int Lp;
};

__global__ void k_tree_ref(RefArgs a) {
  const int d = blockIdx.y;
  const long long t = a.e_prev + static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= a.e_new) return;
  const int32_t* dl = a.delays + static_cast<size_t>(d) * a.nchan;
  int acc[kMaxLevels], cnt[kMaxLevels], node[kMaxLevels];
  for (int l = 0; l < kMaxLevels; ++l) acc[l] = cnt[l] = node[l] = 0;
  int root = 0;
  for (int k = 0; k < a.nleaves; ++k) {
    const int c0 = k * a.C, c1 = min(a.nchan, c0 + a.C);
    int s = 0;
    for (int c = c0; c < c1; ++c) {
      const long long smp = t + dl[c];
      const uint32_t w = a.ring[static_cast<size_t>(c) * 2 * a.R + static_cast<int>((smp >> 5) % a.R)];
      s += (w >> (smp & 31)) & 1;
    }
    int v = (a.mode == kBinary) ? (s >= a.KL) : (a.mode == kGraded ? min(s, a.N) : s);
    if (a.nlev == 1) {
      root = v;
      continue;
    }
    for (int l = 1; l < a.nlev; ++l) {
      acc[l] += v;
      const int fan = min(a.B, a.level_nodes[l - 1] - a.B * node[l]);
      if (++cnt[l] < fan) break;
      const int sum = acc[l];
      acc[l] = 0;
      cnt[l] = 0;
      ++node[l];
      v = (a.mode == kBinary) ? (sum >= a.KI) : (a.mode == kGraded ? min(sum, a.N) : sum);
      if (l == a.nlev - 1) root = v;
    }
  }
  a.plane[static_cast<size_t>(d) * a.Lp + static_cast<int>(t % a.Lp)] = root;
}

template <int MODE, int MAXL, int KW, int TH, int DPW>
cudaError_t run_tree(const TreeArgs& a, dim3 grid, dim3 block, int smem, cudaStream_t s) {
  auto kern = (a.C == 4 && a.nchan % 4 == 0) ? k_tree<MODE, MAXL, KW, TH, DPW, 4> : k_tree<MODE, MAXL, KW, TH, DPW, 0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  kern<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <int MODE, int MAXL, int KW, int TH, int DPW>
cudaError_t run_tree_multi(const TreeMulti& m, int ct4, int nctas, dim3 block, int smem, cudaStream_t s) {
  auto kern = ct4 ? k_tree_multi<MODE, MAXL, KW, TH, DPW, 4> : k_tree_multi<MODE, MAXL, KW, TH, DPW, 0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  kern<<<nctas, block, smem, s>>>(m);
  return cudaGetLastError();
}

struct GoSingle {
  const TreeArgs* a;
  dim3 grid, block;
  int smem;
  cudaStream_t s;
  template <int MODE, int MAXL, int KW, int TH, int DPW>
  cudaError_t go() { return run_tree<MODE, MAXL, KW, TH, DPW>(*a, grid, block, smem, s); }
};

struct GoMulti {
  const TreeMulti* m;
  int ct4, ctas;
  dim3 block;
  int smem;
  cudaStream_t s;
  template <int MODE, int MAXL, int KW, int TH, int DPW>
  cudaError_t go() { return run_tree_multi<MODE, MAXL, KW, TH, DPW>(*m, ct4, ctas, block, smem, s); }
};

// The k_tree instantiation a plan uses, following tree_shape(): the accumulators of every
// open level stay in registers. 0..9 below; +16 when the 4-channel leaf path applies.
int tree_inst(const Plan& p) {
  const int kmax = p.KL > p.KI ? p.KL : p.KI;
  const int maxl = p.nlev <= 4 ? 4 : (p.nlev <= 8 ? 8 : 16);
  const int ml = maxl == 4 ? 0 : (maxl == 8 ? 1 : 2);
  int id;
  if (p.mode == SND_MODE_BINARY) {
    id = (kmax <= 2 ? 0 : 3) + ml;
  } else if (p.mode == SND_MODE_GRADED) {
    id = 6 + ml;
  } else {
    id = 9;
  }
  return id + ((p.C == 4 && p.nchan % 4 == 0) ? 16 : 0);
}

template <typename F>
cudaError_t dispatch_inst(int id, F&& f) {
  switch (id & 15) {
    case 0: return f.template go<kBinary, 4, 2, 2, 2>();
    case 1: return f.template go<kBinary, 8, 1, 2, 2>();
    case 2: return f.template go<kBinary, 16, 1, 2, 1>();
    case 3: return f.template go<kBinary, 4, 1, 8, 1>();
    case 4: return f.template go<kBinary, 8, 1, 8, 1>();
    case 5: return f.template go<kBinary, 16, 1, 8, 1>();
    case 6: return f.template go<kGraded, 4, 2, 1, 1>();
    case 7: return f.template go<kGraded, 8, 1, 1, 1>();
    case 8: return f.template go<kGraded, 16, 1, 1, 1>();
    default: return f.template go<kFloat, 4, 2, 1, 1>();
  }
}

// Kernel arguments of one plan for output samples [e_prev, e_new); *ntx = time tiles.
void tree_args(const Plan& p, int64_t e_prev, int64_t e_new, TreeArgs& a, int* ntx) {
  const DevPtrs& dp = p.dp;
  a = TreeArgs{};
  a.ring = dp.ring;
  a.R = p.R;
  a.nchan = p.nchan;
  a.ndm = p.ndm;
  a.nleaves = p.nleaves;
  a.C = p.C;
  a.B = p.B;
  a.KL = p.KL;
  a.KI = p.KI;
  a.N = p.N;
  a.nlev = p.nlev;
  for (int l = 0; l < kMaxLevels; ++l) a.level_nodes[l] = l < p.nlev ? p.level_nodes[l] : 1;
  a.tp_off = dp.tp_off;
  a.gepk = dp.gepk;
  a.gleaf = dp.gleaf;
  a.gmeta = dp.gmeta;
  a.tile_wb = dp.tile_wb;
  const TreeGeom& g = p.geom;
  a.G = g.group_leaves;
  a.span = g.span;
  a.cspan = g.cspan;
  a.maxpat = g.max_pat_group;
  a.span_extra = g.span - g.tile_words;
  {
    const int lmax = p.B * (p.C < p.N ? p.C : p.N);
    a.plain1 = (lmax <= p.N && lmax <= 63) ? 1 : 0;
  }
  a.word0 = e_prev >> 5;
  a.nwords = static_cast<int>(((e_new - 1) >> 5) - (e_prev >> 5) + 1);
  // the fewest tiles of at most tile_words, either spread evenly or (graded and float) full
  // with one short tail tile, whichever costs less: per tile, 32-word chunks of leaf series
  // (phase 1, tile + span_extra words), 32-word phase-2 slots and a fixed part, weighted
  // about 4 : 9 : 2 as measured on the 1024-channel float tree. Binary trees (two CTAs per
  // SM, cheaper one-plane series) measured faster with even tiles.
  const int ntiles = (a.nwords + g.tile_words - 1) / g.tile_words;
  auto tile_cost = [&](int t) { return 4 * ((t + a.span_extra + 31) / 32) + 9 * ((t + 31) / 32) + 2; };
  auto cost = [&](int tw) {
    int c = 0;
    for (int i = 0, left = a.nwords; i < ntiles; ++i, left -= tw) c += tile_cost(left < tw ? left : tw);
    return c;
  };
  const int even = (a.nwords + ntiles - 1) / ntiles;
  a.tile_words = (p.mode != SND_MODE_BINARY && cost(g.tile_words) < cost(even)) ? g.tile_words : even;
  a.plane = dp.plane;
  a.Lp = p.Lp;
  *ntx = ntiles;
}

}  // namespace

// Kernel shape for a mode and tree depth: {warps per CTA, DMs per warp, words per lane}.
// Chosen so the per-thread accumulators (levels x DMs x words x planes) stay in registers.
TreeShape tree_shape(int mode, int nlev, int kmax) {
  const int maxl = nlev <= 4 ? 4 : (nlev <= 8 ? 8 : 16);
  if (mode == SND_MODE_BINARY) {
    const int regs = maxl * (kmax <= 2 ? 2 : 8);  // accumulator words per (DM, word)
    if (regs * 4 <= 48) return {16, 2, 2};
    if (regs * 2 <= 48) return {16, 2, 1};
    return {16, 1, 1};
  }
  // graded / float: 32 warps x 1 DM (1024 threads, <= 64 registers) keeps 32-DM tiles at
  // twice the warps per SM of 16 warps x 2 DMs
  if (mode == SND_MODE_GRADED) {
    if (maxl <= 4) return {16, 1, 2};
    return {16, 1, 1};
  }
  return {16, 1, 2};
}

cudaError_t launch_tree(const Plan& p, int64_t e_prev, int64_t e_new, cudaStream_t s) {
  if (e_new <= e_prev) return cudaSuccess;
  const DevPtrs& dp = p.dp;
  if (p.flags & kFlagReferenceTree) {
    RefArgs r{};
    r.ring = dp.ring;
    r.R = p.R;
    r.nchan = p.nchan;
    r.ndm = p.ndm;
    r.nleaves = p.nleaves;
    r.C = p.C;
    r.B = p.B;
    r.KL = p.KL;
    r.KI = p.KI;
    r.N = p.N;
    r.nlev = p.nlev;
    r.mode = p.mode;
    for (int l = 0; l < kMaxLevels; ++l) r.level_nodes[l] = l < p.nlev ? p.level_nodes[l] : 1;
    r.delays = dp.delays;
    r.e_prev = e_prev;
    r.e_new = e_new;
    r.plane = dp.plane;
    r.Lp = p.Lp;
    const long long n = e_new - e_prev;
    dim3 grid(static_cast<unsigned>((n + 255) / 256), p.ndm);
    k_tree_ref<<<grid, 256, 0, s>>>(r);
    p.launches += 1;
    return cudaGetLastError();
  }
  if (p.direct) return launch_tree_direct(p, e_prev, e_new, s);
  TreeArgs a;
  int ntx = 0;
  tree_args(p, e_prev, e_new, a, &ntx);
  const TreeGeom& g = p.geom;
  const dim3 block(32, g.warps), grid(ntx, g.ndm_tiles);
  const int smem = g.smem_bytes;
  p.launches += 1;
  GoSingle go{&a, grid, block, smem, s};
  return dispatch_inst(tree_inst(p), go);
}

// Trees of several plans in as few launches as possible: plans that share a kernel
// instantiation and block shape run in one launch (k_tree_multi, up to 64 beams each).
cudaError_t launch_tree_batch(const Plan* const* plans, const int64_t* e_prev, const int64_t* e_new, int n,
                              cudaStream_t s) {
  {
    // plans on the direct kernel go through its own grouped launches
    std::vector<const Plan*> dp;
    std::vector<int64_t> dep, den;
    for (int i = 0; i < n; ++i)
      if (plans[i]->direct) {
        dp.push_back(plans[i]);
        dep.push_back(e_prev[i]);
        den.push_back(e_new[i]);
      }
    if (!dp.empty()) {
      const cudaError_t e = launch_tree_direct_batch(dp.data(), dep.data(), den.data(), static_cast<int>(dp.size()), s);
      if (e != cudaSuccess) return e;
    }
  }
  std::vector<int> done(n, 0);
  for (int i = 0; i < n; ++i) done[i] = plans[i]->direct ? 1 : 0;
  for (int i = 0; i < n; ++i) {
    if (done[i]) continue;
    const int key = tree_inst(*plans[i]);
    const int warps = plans[i]->geom.warps;
    TreeMulti m{};
    int smem = 0, ctas = 0;
    const Plan* owner = nullptr;
    for (int j = i; j < n && m.nbeams < kMaxBatchBeams; ++j) {
      if (done[j] || tree_inst(*plans[j]) != key || plans[j]->geom.warps != warps) continue;
      done[j] = 1;
      if (e_new[j] <= e_prev[j]) continue;
      int ntx = 0;
      tree_args(*plans[j], e_prev[j], e_new[j], m.beam[m.nbeams], &ntx);
      m.first[m.nbeams] = ctas;
      m.ntx[m.nbeams] = ntx;
      ctas += ntx * plans[j]->geom.ndm_tiles;
      smem = smem > plans[j]->geom.smem_bytes ? smem : plans[j]->geom.smem_bytes;
      plans[j]->launches += (owner == nullptr) ? 1 : 0;
      owner = plans[j];
      ++m.nbeams;
    }
    if (m.nbeams == 0) continue;
    GoMulti go{&m, (key & 16) ? 1 : 0, ctas, dim3(32, warps), smem, s};
    const cudaError_t e = dispatch_inst(key, go);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace snd
