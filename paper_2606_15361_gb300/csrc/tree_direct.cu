// SND tree, direct form (Methods, "The Spiking Neural Dedispersion algorithm", "Tree
// activation modes"), for one GB300 CTA per (32 trial DMs x tile of output words).
//
// What is computed is the tree of the paper, node rule by node rule; only the order of the
// exact integer additions differs from a level-by-level walk:
//  * Mode C (float): no node rule, so the root is the sum of all channel bits. Every channel's
//    bit is added straight into a bit-sliced counter (carry-save full adders, 2 logic ops per
//    channel and word), which is the same integer.
//  * Mode B (graded): min(s, N) can only bind at a node whose channel count exceeds N. Below
//    the first such level ("exact level") every node value is its plain channel sum, so each
//    exact-level node is counted directly over its channels, clipped to N, and the few levels
//    above it are evaluated node by node with saturating 8-plane adders (the cap at every node,
//    the root included).
//  * Mode A (binary): every node thresholds, so the tree is walked leaf by leaf: a leaf is the
//    quorum of its C = 4 channel bits (>= K_L), and every node above keeps a two-plane
//    thermometer of its child count for the quorum K_I <= 2.
// Every channel is read at t + delta_c(d) (the shifts telescope), as in the leaf-sharing
// kernel (tree.cu), so both give the oracle's planes bit for bit.
//
// GPU mapping:
//  * lanes are 32 consecutive trial DMs; a warp owns KW consecutive 32-sample words of the
//    CTA's time tile (warp w: words w*KW ..), so per channel a lane reads one 16-bit offset
//    and then KW+1 consecutive window words (a sliding funnel-shift window). The 32 DMs of a
//    tile read one channel at offsets that differ by less than 32 words, so the reads hit
//    distinct banks (or broadcast) without conflicts.
//  * channels are staged 64 or 128 at a time (a round): every warp issues TMA bulk copies
//    (cp.async.bulk) of its share of the round's channel windows from the L2-resident bit
//    ring, and warp 0 the round's offset table, onto a double-buffered mbarrier pipeline, so
//    the next round lands while the current one is added. Waits are bounded; a wait that runs
//    out sets a status bit and ends the CTA.
//  * the counter planes stay in registers across groups; the root is turned into int32
//    samples by a 32x32 bit transpose and written with 128-bit stores.

#include <vector>

#include "bulk.h"
#include "snd_internal.h"

namespace snd {
namespace {

constexpr int kDG = 64;                          // channels per adder group (one carry out)
constexpr long long kDirWaitCycles = kStageWaitCycles;

struct DirArgs {
  const uint32_t* ring;
  int R, nchan, ndm;
  int B, KL, KI, N, nlev;
  int level_nodes[kMaxLevels];
  int sub_groups;          // graded: staged groups per exact-level node
  int sub_lev;             // graded: the exact level
  const uint16_t* meta;    // [ndm_tiles][nchan][32]: (word offset << 5) | bit shift
  const int32_t* base4;    // [ndm_tiles][nchan]: first staged ring word (relative, multiple of 4)
  int cspan;               // staged words per channel (multiple of 4)
  int sgroups;             // adder groups of kDG channels staged per round (1 or 2)
  int tile_words;          // NW * KW output words per CTA
  long long word0;         // absolute index of the first output word
  int nwords;              // output words of this call
  int32_t* plane;
  int Lp;
  uint32_t* status;
  long long wait_cycles;   // bound of a staging wait (clock cycles)
  long long e_prev, e_new; // emitted samples of this call
  int store;               // write the root plane (0: a fire-count pass only)
  unsigned long long* level_fires;  // binary: per-level counts of firing node-samples (null: off)
};

constexpr int kMaxDirBeams = 64;

struct DirMulti {
  int nbeams;
  int total;               // work items of all beams
  unsigned int* queue;     // next work item (zero at launch)
  int first[kMaxDirBeams];
  int ntx[kMaxDirBeams];
  DirArgs beam[kMaxDirBeams];
};

// s += a + b in carry-save form: s keeps the sum bit, the carry (weight x2) is returned
__device__ __forceinline__ uint32_t fa(uint32_t& s, uint32_t a, uint32_t b) {
  const uint32_t x = s;
  s = x ^ a ^ b;
  return (x & a) | (b & (x ^ a));
}

// Counter planes P[0..NPL) += 2^L bits fetched for channels c0 .. c0 + 2^L: a balanced tree
// of full adders; the single carry out (weight 2^L) is returned in cout.
template <int L, int KW, int NPL, typename F>
__device__ __forceinline__ void hs_block(uint32_t (&P)[NPL][KW], uint32_t (&cout)[KW], int c0, F& fetch) {
  if constexpr (L == 1) {
    uint32_t a[KW], b[KW];
    fetch(c0, a);
    fetch(c0 + 1, b);
#pragma unroll
    for (int j = 0; j < KW; ++j) cout[j] = fa(P[0][j], a[j], b[j]);
  } else {
    uint32_t ca[KW], cb[KW];
    hs_block<L - 1, KW, NPL>(P, ca, c0, fetch);
    hs_block<L - 1, KW, NPL>(P, cb, c0 + (1 << (L - 1)), fetch);
#pragma unroll
    for (int j = 0; j < KW; ++j) cout[j] = fa(P[L - 1][j], ca[j], cb[j]);
  }
}

// Add one group of 64 channels into P (planes 0..5 by the adder tree, the weight-64 carry
// rippled up from plane 6).
template <int KW, int NPL, typename F>
__device__ __forceinline__ void add_group(uint32_t (&P)[NPL][KW], F& fetch) {
  uint32_t c[KW];
  hs_block<6, KW, NPL>(P, c, 0, fetch);
#pragma unroll
  for (int p = 6; p < NPL; ++p)
#pragma unroll
    for (int j = 0; j < KW; ++j) {
      const uint32_t t = P[p][j] & c[j];
      P[p][j] ^= c[j];
      c[j] = t;
    }
}

// min(s, N) of an NP-plane count as 8 planes (N <= 255)
template <int NP>
__device__ __forceinline__ void cap8(const uint32_t* s, int N, uint32_t* out) {
  uint32_t gt = 0, eq = 0xFFFFFFFFu;
#pragma unroll
  for (int p = NP - 1; p >= 0; --p) {
    if ((N >> p) & 1) {
      eq &= s[p];
    } else {
      gt |= eq & s[p];
      eq &= ~s[p];
    }
  }
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const uint32_t sp = p < NP ? s[p < NP ? p : 0] : 0u;
    out[p] = ((N >> p) & 1) ? (sp | gt) : (sp & ~gt);
  }
}

// acc = min(acc + v, N) on 8 planes (acc, v <= N <= 255)
__device__ __forceinline__ void add_sat8(uint32_t* acc, const uint32_t* v, int N) {
  uint32_t c = 0;
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const uint32_t x = acc[p], y = v[p];
    acc[p] = x ^ y ^ c;
    c = (x & y) | (c & (x ^ y));
  }
  uint32_t s9[9];
#pragma unroll
  for (int p = 0; p < 8; ++p) s9[p] = acc[p];
  s9[8] = c;
  cap8<9>(s9, N, acc);
}

// 32x32 bit transpose: bit c of m[r] <-> bit r of m[c]
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

template <int NP>
__device__ __forceinline__ void store_planes(int32_t* dst, const uint32_t* planes) {
  uint32_t m[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) m[i] = (i < NP) ? planes[i < NP ? i : 0] : 0u;
  transpose32(m);
  int4* d4 = reinterpret_cast<int4*>(dst);
#pragma unroll
  for (int i = 0; i < 8; ++i)
    d4[i] = make_int4(static_cast<int>(m[4 * i]), static_cast<int>(m[4 * i + 1]), static_cast<int>(m[4 * i + 2]),
                      static_cast<int>(m[4 * i + 3]));
}

__device__ __forceinline__ void store_bits(int32_t* dst, uint32_t v) {
  int4* d4 = reinterpret_cast<int4*>(dst);
#pragma unroll
  for (int i = 0; i < 8; ++i)
    d4[i] = make_int4((v >> (4 * i)) & 1, (v >> (4 * i + 1)) & 1, (v >> (4 * i + 2)) & 1, (v >> (4 * i + 3)) & 1);
}

constexpr int kBinary = SND_MODE_BINARY, kGraded = SND_MODE_GRADED, kFloat = SND_MODE_FLOAT;

// Per-lane tree state of each mode. NPL: counter planes; MAXU: levels kept above the counted
// level (graded: above the exact level; binary: above the leaves).
template <int MODE, int KW, int NPL, int MAXU>
struct DState;

template <int KW, int NPL, int MAXU>
struct DState<kFloat, KW, NPL, MAXU> {
  uint32_t P[NPL][KW];
  __device__ __forceinline__ void set_counting(const DirArgs&, long long, bool) {}
  __device__ __forceinline__ void flush(const DirArgs&, int) {}
  __device__ __forceinline__ void init(const DirArgs&) {
#pragma unroll
    for (int p = 0; p < NPL; ++p)
#pragma unroll
      for (int j = 0; j < KW; ++j) P[p][j] = 0;
  }
  template <typename F>
  __device__ __forceinline__ void group(const DirArgs&, int, F& fetch) {
    add_group<KW, NPL>(P, fetch);
  }
  __device__ __forceinline__ void store(int32_t* row, int j) const {
    uint32_t pl[NPL];
#pragma unroll
    for (int p = 0; p < NPL; ++p) pl[p] = P[p][j];
    store_planes<NPL>(row, pl);
  }
};

template <int KW, int NPL, int MAXU>
struct DState<kGraded, KW, NPL, MAXU> {
  static_assert(NPL >= 8, "the root is kept in the counter planes");
  uint32_t P[NPL][KW];  // count of the open exact-level node; at the end, the root's 8 planes
  __device__ __forceinline__ void set_counting(const DirArgs&, long long, bool) {}
  __device__ __forceinline__ void flush(const DirArgs&, int) {}
  uint32_t acc[MAXU > 0 ? MAXU : 1][KW][8];
  int cnt[MAXU > 0 ? MAXU : 1], node[MAXU > 0 ? MAXU : 1], fan[MAXU > 0 ? MAXU : 1];
  __device__ __forceinline__ void clearP() {
#pragma unroll
    for (int p = 0; p < NPL; ++p)
#pragma unroll
      for (int j = 0; j < KW; ++j) P[p][j] = 0;
  }
  __device__ __forceinline__ void set_root(const uint32_t (&v)[KW][8]) {
#pragma unroll
    for (int j = 0; j < KW; ++j)
#pragma unroll
      for (int p = 0; p < 8; ++p) P[p][j] = v[j][p];
  }
  __device__ __forceinline__ void init(const DirArgs& a) {
    clearP();
#pragma unroll
    for (int u = 0; u < (MAXU > 0 ? MAXU : 1); ++u) {
#pragma unroll
      for (int j = 0; j < KW; ++j)
#pragma unroll
        for (int p = 0; p < 8; ++p) acc[u][j][p] = 0;
      const int l = a.sub_lev + 1 + u;  // level of the node accumulated in acc[u]
      cnt[u] = 0;
      node[u] = 0;
      fan[u] = (l < a.nlev) ? min(a.B, a.level_nodes[l - 1]) : 1;
    }
  }
  template <typename F>
  __device__ __forceinline__ void group(const DirArgs& a, int g, F& fetch) {
    add_group<KW, NPL>(P, fetch);
    if ((g + 1) % a.sub_groups != 0) return;
    // an exact-level node is complete: its value min(count, N) goes up the capped levels
    uint32_t cur[KW][8];
#pragma unroll
    for (int j = 0; j < KW; ++j) {
      uint32_t s[NPL];
#pragma unroll
      for (int p = 0; p < NPL; ++p) s[p] = P[p][j];
      cap8<NPL>(s, a.N, cur[j]);
    }
    clearP();
    if (MAXU == 0 || a.sub_lev == a.nlev - 1) {
      set_root(cur);
      return;
    }
#pragma unroll
    for (int u = 0; u < (MAXU > 0 ? MAXU : 1); ++u) {
      const int l = a.sub_lev + 1 + u;
      if (l >= a.nlev) break;
#pragma unroll
      for (int j = 0; j < KW; ++j) add_sat8(acc[u][j], cur[j], a.N);
      if (++cnt[u] < fan[u]) break;
#pragma unroll
      for (int j = 0; j < KW; ++j)
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          cur[j][p] = acc[u][j][p];
          acc[u][j][p] = 0;
        }
      cnt[u] = 0;
      ++node[u];
      fan[u] = min(a.B, a.level_nodes[l - 1] - a.B * node[u]);
      if (l == a.nlev - 1) set_root(cur);
    }
  }
  __device__ __forceinline__ void store(int32_t* row, int j) const {
    uint32_t pl[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) pl[p] = P[p][j];
    store_planes<8>(row, pl);
  }
};

template <int KW, int NPL, int MAXU>
struct DState<kBinary, KW, NPL, MAXU> {
  uint32_t t0[MAXU][KW], t1[MAXU][KW];  // thermometer of the open node of every level >= 1
  uint32_t root[KW];
  int cnt[MAXU], node[MAXU], fan[MAXU];
  uint32_t ki2;  // all-ones when K_I = 2 (else K_I = 1)
  // per-level fire counts (level 0 = leaves) over this lane's emitted samples, when counting
  bool counting;
  uint32_t vmask[KW];
  unsigned fires[MAXU + 1];
  __device__ __forceinline__ void set_counting(const DirArgs& a, long long aw_first, bool row_ok) {
    counting = a.level_fires != nullptr;
#pragma unroll
    for (int u = 0; u <= MAXU; ++u) fires[u] = 0;
#pragma unroll
    for (int j = 0; j < KW; ++j) {
      // bits of word aw_first + j whose samples lie in [e_prev, e_new)
      const long long s0 = (aw_first + j) * 32;
      const long long lo = a.e_prev > s0 ? a.e_prev - s0 : 0, hi = a.e_new - s0 < 32 ? a.e_new - s0 : 32;
      uint32_t m = 0;
      if (row_ok && hi > lo) m = (hi - lo >= 32 ? 0xFFFFFFFFu : ((1u << (hi - lo)) - 1u)) << lo;
      vmask[j] = m;
    }
  }
  __device__ __forceinline__ void count(int level, const uint32_t (&v)[KW]) {
#pragma unroll
    for (int j = 0; j < KW; ++j) fires[level] += __popc(v[j] & vmask[j]);
  }
  __device__ __forceinline__ void init(const DirArgs& a) {
    ki2 = a.KI >= 2 ? 0xFFFFFFFFu : 0u;
#pragma unroll
    for (int u = 0; u < MAXU; ++u) {
#pragma unroll
      for (int j = 0; j < KW; ++j) t0[u][j] = t1[u][j] = 0;
      const int l = 1 + u;
      cnt[u] = 0;
      node[u] = 0;
      fan[u] = (l < a.nlev) ? min(a.B, a.level_nodes[l - 1]) : 1;
    }
#pragma unroll
    for (int j = 0; j < KW; ++j) root[j] = 0;
  }
  // push a finished leaf's bits up the tree
  __device__ __forceinline__ void push(const DirArgs& a, uint32_t (&v)[KW]) {
#pragma unroll
    for (int u = 0; u < MAXU; ++u) {
      const int l = 1 + u;
      if (l >= a.nlev) break;
#pragma unroll
      for (int j = 0; j < KW; ++j) {
        t1[u][j] |= t0[u][j] & v[j];
        t0[u][j] |= v[j];
      }
      if (++cnt[u] < fan[u]) return;
#pragma unroll
      for (int j = 0; j < KW; ++j) {
        v[j] = (t1[u][j] & ki2) | (t0[u][j] & ~ki2);
        t0[u][j] = t1[u][j] = 0;
      }
      cnt[u] = 0;
      ++node[u];
      fan[u] = min(a.B, a.level_nodes[l - 1] - a.B * node[u]);
      if (counting) count(l, v);
      if (l == a.nlev - 1) {
#pragma unroll
        for (int j = 0; j < KW; ++j) root[j] = v[j];
      }
    }
  }
  // the lanes' counts summed per warp, added to the plan's per-level totals
  __device__ __forceinline__ void flush(const DirArgs& a, int lane) {
    if (!counting) return;
#pragma unroll
    for (int u = 0; u <= MAXU; ++u) {
      if (u >= a.nlev) break;
      unsigned c = fires[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
      if (lane == 0 && c) atomicAdd(a.level_fires + u, static_cast<unsigned long long>(c));
    }
  }
  // the 16 leaves of a staged group, each the quorum >= KL of its four channel bits
  template <int KL, typename F>
  __device__ __forceinline__ void leaves(const DirArgs& a, F& fetch) {
#pragma unroll 4
    for (int k = 0; k < kDG / 4; ++k) {
      uint32_t x0[KW], x1[KW], x2[KW], x3[KW], v[KW];
      fetch(4 * k, x0);
      fetch(4 * k + 1, x1);
      fetch(4 * k + 2, x2);
      fetch(4 * k + 3, x3);
#pragma unroll
      for (int j = 0; j < KW; ++j) {
        const uint32_t a0 = x0[j], a1 = x1[j], a2 = x2[j], a3 = x3[j];
        if constexpr (KL == 1) {
          v[j] = a0 | a1 | a2 | a3;
        } else if constexpr (KL == 2) {
          const uint32_t m3 = (a0 & a1) | (a2 & (a0 | a1));  // >= 2 of a0..a2
          v[j] = m3 | ((a0 | a1 | a2) & a3);
        } else if constexpr (KL == 3) {
          const uint32_t m3 = (a0 & a1) | (a2 & (a0 | a1));
          v[j] = (a0 & a1 & a2) | (m3 & a3);
        } else {
          v[j] = a0 & a1 & a2 & a3;
        }
      }
      if (counting) count(0, v);
      push(a, v);
    }
  }
  template <typename F>
  __device__ __forceinline__ void group(const DirArgs& a, int, F& fetch) {
    switch (a.KL) {
      case 1: leaves<1>(a, fetch); break;
      case 2: leaves<2>(a, fetch); break;
      case 3: leaves<3>(a, fetch); break;
      default: leaves<4>(a, fetch); break;
    }
  }
  __device__ __forceinline__ void store(int32_t* row, int j) const { store_bits(row, root[j]); }
};

// Mode A on a regular tree: B = 2, 4 or 8 (MODE = kBinReg + 10 B + K_I), C = 4, and each level
// groups B consecutive nodes of the one below (the last node of a level may have fewer). The
// levels whose nodes lie inside one staged group of 64 channels (16 leaves: up to level 4 for
// B = 2, level 2 for B = 4, level 1 for B = 8) are evaluated per group as a fixed tree of logic operations, with
// no per-leaf bookkeeping; only the levels above them keep an open node (its two-plane
// thermometer) from group to group. The same node rules, so the same planes, as the general
// binary state above.
constexpr int kBinReg = 100;

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <int MODE, int KW, int NPL, int MAXU>
struct DState {
  static constexpr int BB = (MODE - kBinReg) / 10, KI = (MODE - kBinReg) % 10;
  static_assert(BB == 2 || BB == 4 || BB == 8, "regular binary tree: B = 2, 4 or 8");
  static_assert(KI == 1 || KI == 2, "K_I = 1 or 2");
  static constexpr int UIN = BB == 2 ? 4 : (BB == 4 ? 2 : 1);  // highest level inside a group of 16 leaves
  static constexpr int SPAN = ipow(BB, UIN);       // leaves under one such node
  static constexpr int NTOP = 16 / SPAN;           // such nodes per group
  uint32_t t0[MAXU][KW], t1[MAXU][KW];  // thermometer of the open node of every level > UIN
  uint32_t root[KW];
  int cnt[MAXU], node_i[MAXU], fan[MAXU];
  __device__ __forceinline__ void set_counting(const DirArgs&, long long, bool) {}
  __device__ __forceinline__ void flush(const DirArgs&, int) {}
  __device__ __forceinline__ void init(const DirArgs& a) {
#pragma unroll
    for (int u = 0; u < MAXU; ++u) {
#pragma unroll
      for (int j = 0; j < KW; ++j) t0[u][j] = t1[u][j] = 0;
      const int l = UIN + 1 + u;
      cnt[u] = 0;
      node_i[u] = 0;
      fan[u] = (l < a.nlev) ? min(a.B, a.level_nodes[l - 1]) : 1;
    }
#pragma unroll
    for (int j = 0; j < KW; ++j) root[j] = 0;
  }
  // leaf L0: the quorum >= KL of its four channel bits
  template <int KL, int L0, typename F>
  __device__ __forceinline__ void leaf(F& fetch, uint32_t (&v)[KW]) {
    uint32_t x0[KW], x1[KW], x2[KW], x3[KW];
    fetch(4 * L0, x0);
    fetch(4 * L0 + 1, x1);
    fetch(4 * L0 + 2, x2);
    fetch(4 * L0 + 3, x3);
#pragma unroll
    for (int j = 0; j < KW; ++j) {
      const uint32_t a0 = x0[j], a1 = x1[j], a2 = x2[j], a3 = x3[j];
      if constexpr (KL == 1) {
        v[j] = a0 | a1 | a2 | a3;
      } else if constexpr (KL == 2) {
        const uint32_t m3 = (a0 & a1) | (a2 & (a0 | a1));  // >= 2 of a0..a2
        v[j] = m3 | ((a0 | a1 | a2) & a3);
      } else if constexpr (KL == 3) {
        const uint32_t m3 = (a0 & a1) | (a2 & (a0 | a1));
        v[j] = (a0 & a1 & a2) | (m3 & a3);
      } else {
        v[j] = a0 & a1 & a2 & a3;
      }
    }
  }
  // children I.. of the level-U node over leaves L0.., folded into its thermometer (t0: >= 1
  // child fired, t1: >= 2)
  template <int KL, int U, int L0, int I, typename F>
  __device__ __forceinline__ void children(F& fetch, uint32_t (&s0)[KW], uint32_t (&s1)[KW]) {
    uint32_t c[KW];
    node<KL, U - 1, L0 + I * ipow(BB, U - 1)>(fetch, c);
#pragma unroll
    for (int j = 0; j < KW; ++j) {
      if constexpr (I == 0) {
        s0[j] = c[j];
        s1[j] = 0u;
      } else {
        s1[j] |= s0[j] & c[j];
        s0[j] |= c[j];
      }
    }
    if constexpr (I + 1 < BB) children<KL, U, L0, I + 1>(fetch, s0, s1);
  }
  // the fire bits of the level-U node whose first leaf is L0
  template <int KL, int U, int L0, typename F>
  __device__ __forceinline__ void node(F& fetch, uint32_t (&v)[KW]) {
    if constexpr (U == 0) {
      leaf<KL, L0>(fetch, v);
    } else {
      uint32_t s0[KW], s1[KW];
      children<KL, U, L0, 0>(fetch, s0, s1);
#pragma unroll
      for (int j = 0; j < KW; ++j) v[j] = KI == 2 ? s1[j] : s0[j];
    }
  }
  // a finished level-UIN node goes up the levels kept across groups
  __device__ __forceinline__ void push(const DirArgs& a, uint32_t (&v)[KW]) {
    if (UIN == a.nlev - 1) {
#pragma unroll
      for (int j = 0; j < KW; ++j) root[j] = v[j];
      return;
    }
#pragma unroll
    for (int u = 0; u < MAXU; ++u) {
      const int l = UIN + 1 + u;
      if (l >= a.nlev) break;
#pragma unroll
      for (int j = 0; j < KW; ++j) {
        t1[u][j] |= t0[u][j] & v[j];
        t0[u][j] |= v[j];
      }
      if (++cnt[u] < fan[u]) return;
#pragma unroll
      for (int j = 0; j < KW; ++j) {
        v[j] = KI == 2 ? t1[u][j] : t0[u][j];
        t0[u][j] = t1[u][j] = 0;
      }
      cnt[u] = 0;
      ++node_i[u];
      fan[u] = min(a.B, a.level_nodes[l - 1] - a.B * node_i[u]);
      if (l == a.nlev - 1) {
#pragma unroll
        for (int j = 0; j < KW; ++j) root[j] = v[j];
      }
    }
  }
  template <int KL, int K, typename F>
  __device__ __forceinline__ void tops(const DirArgs& a, F& fetch) {
    uint32_t v[KW];
    node<KL, UIN, K * SPAN>(fetch, v);
    push(a, v);
    if constexpr (K + 1 < NTOP) tops<KL, K + 1>(a, fetch);
  }
  template <typename F>
  __device__ __forceinline__ void group(const DirArgs& a, int, F& fetch) {
    switch (a.KL) {
      case 1: tops<1, 0>(a, fetch); break;
      case 2: tops<2, 0>(a, fetch); break;
      case 3: tops<3, 0>(a, fetch); break;
      default: tops<4, 0>(a, fetch); break;
    }
  }
  __device__ __forceinline__ void store(int32_t* row, int j) const { store_bits(row, root[j]); }
};

// One CTA: DM tile `tile` (32 DMs, lane = DM) x time tile bx (NW warps x KW words).
// bars: the CTA's two staging mbarriers (initialised once per CTA with one arrival per warp);
// k0: staging rounds this CTA ran before (round k uses buffer k & 1, phase parity (k >> 1) & 1).
// Returns false when a staging wait ran out (the CTA must stop).
template <int MODE, int KW, int NPL, int MAXU>
__device__ __forceinline__ bool direct_cta(const DirArgs& a, int bx, int tile, unsigned long long* bars, int k0) {
  extern __shared__ __align__(128) uint32_t sm[];
  const int lane = threadIdx.x, wd = threadIdx.y, NW = blockDim.y;
  const int tid = wd * 32 + lane, nthr = 32 * NW;
  const int cspan = a.cspan;
  const int SG = kDG * a.sgroups;                  // channels per staging round
  const int wbuf = SG * cspan;                     // window words per buffer
  uint32_t* win = sm;                              // [2][SG][cspan]
  uint16_t* met = reinterpret_cast<uint16_t*>(sm + 2 * wbuf);  // [2][SG][32]
  int32_t* sbase = reinterpret_cast<int32_t*>(sm + 2 * wbuf + SG * 32);  // [nchan]
  const long long aw0 = a.word0 + static_cast<long long>(bx) * a.tile_words;
  const int lead = static_cast<int>(aw0 & 3);
  const long long aw4 = aw0 - lead;
  const int ngroups = a.nchan / SG;

  // ring index of every channel's first staged word for this CTA (R is a multiple of 4 and
  // base4 < R, so one conditional subtract after a single 64-bit modulo per CTA)
  {
    const int r0 = static_cast<int>(aw4 % a.R);
    for (int c = tid; c < a.nchan; c += nthr) {
      int st0 = r0 + a.base4[static_cast<size_t>(tile) * a.nchan + c];
      if (st0 >= a.R) st0 -= a.R;
      sbase[c] = st0;
    }
  }
  __syncthreads();

  // Stage round g into buffer b. Every warp issues the bulk copies of its share of the SG
  // channel windows (and warp 0 the round's offset table) after announcing its bytes on the
  // buffer's mbarrier, so the transaction count never runs ahead of the copies and no warp
  // carries the whole round's issue cost.
  const int share = (SG + NW - 1) / NW;
  auto issue = [&](int g) {
    const int b = (k0 + g) & 1;
    const uint32_t bar = smem_u32(&bars[b]);
    const int i0 = wd * share, i1 = min(SG, i0 + share);
    // the buffer's previous contents were read by every warp before the last barrier
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (lane == 0)
      bar_expect(bar, static_cast<uint32_t>((i1 > i0 ? i1 - i0 : 0) * cspan * 4 + (wd == 0 ? SG * 64 : 0)));
    __syncwarp();
    for (int i = i0 + lane; i < i1; i += 32) {
      const int c = g * SG + i;
      bulk_g2s(smem_u32(win + b * wbuf + i * cspan), a.ring + static_cast<size_t>(c) * 2 * a.R + sbase[c],
               static_cast<uint32_t>(cspan * 4), bar);
    }
    if (wd == 0 && lane == 0)
      bulk_g2s(smem_u32(met + b * SG * 32), a.meta + (static_cast<size_t>(tile) * a.nchan + g * SG) * 32,
               static_cast<uint32_t>(SG * 64), bar);
  };

  DState<MODE, KW, NPL, MAXU> st;
  st.init(a);
  st.set_counting(a, aw0 + wd * KW, tile * 32 + lane < a.ndm);
  // a warp none of whose words is emitted here (the short last tile of a call) only keeps the
  // CTA's barriers
  const bool busy = wd * KW < min(a.tile_words, a.nwords - bx * a.tile_words);
  issue(0);
  int g = 0, abort = 0;
  for (; g < ngroups; ++g) {
    const int b = (k0 + g) & 1;
    if (g + 1 < ngroups) issue(g + 1);  // buffer b ^ 1 was released by the last barrier
    const bool ok = bar_wait(smem_u32(&bars[b]), ((k0 + g) >> 1) & 1, a.wait_cycles);
    if (ok && busy) {
#pragma unroll 1
      for (int h = 0; h < a.sgroups; ++h) {
        const uint16_t* M = met + b * SG * 32 + h * kDG * 32 + lane;
        const uint32_t* Wb = win + b * wbuf + h * kDG * cspan + lead + wd * KW;
        auto fetch = [&](int ci, uint32_t (&v)[KW]) {
          const uint32_t m = M[ci * 32];
          const uint32_t* p = Wb + ci * cspan + (m >> 5);
          uint32_t x[KW + 1];
#pragma unroll
          for (int j = 0; j <= KW; ++j) x[j] = p[j];
#pragma unroll
          for (int j = 0; j < KW; ++j) v[j] = __funnelshift_r(x[j], x[j + 1], m);
        };
        st.group(a, g * a.sgroups + h, fetch);
      }
    }
    abort = __syncthreads_or(!ok);
    if (abort) break;
  }
  if (abort) {
    // a staging wait ran out: report it, and give the copies still in flight (groups g and
    // g + 1) another bounded wait before the CTA's shared memory is released
    if (tid == 0) {
      atomicOr(a.status, kStatusTreeTimeout);
      for (int gi = g; gi < g + 2 && gi < ngroups; ++gi)
        bar_wait(smem_u32(&bars[(k0 + gi) & 1]), ((k0 + gi) >> 1) & 1, kDirWaitCycles);
    }
    return false;
  }
  st.flush(a, lane);
  const int drow = tile * 32 + lane;
  if (drow >= a.ndm || !a.store) return true;
  const int lw = a.Lp >> 5;
#pragma unroll
  for (int j = 0; j < KW; ++j) {
    const int w = wd * KW + j;
    const long long aw = aw0 + w;
    if (w >= a.tile_words || aw - a.word0 >= a.nwords) continue;
    const int col = static_cast<int>(aw % lw) * 32;
    st.store(a.plane + static_cast<size_t>(drow) * a.Lp + col, j);
  }
  return true;
}

__device__ __forceinline__ void init_bars(unsigned long long* bars) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    // one arrival per warp: every warp stages its share of a round
    bar_init(smem_u32(&bars[0]), blockDim.y);
    bar_init(smem_u32(&bars[1]), blockDim.y);
    bar_init_fence();
  }
}

template <int MODE, int KW, int NPL, int MAXU>
__global__ void __launch_bounds__(256, 2) k_snd(const __grid_constant__ DirArgs a) {
  __shared__ __align__(8) unsigned long long bars[2];
  init_bars(bars);
  direct_cta<MODE, KW, NPL, MAXU>(a, blockIdx.x, blockIdx.y, bars, 0);
}

// Many beams, persistent: each CTA takes (beam, DM tile, time tile) work items from a device
// counter (m.queue, zero at launch) until none is left; item i belongs to the last beam b with
// first[b] <= i, its time tile fastest.
template <int MODE, int KW, int NPL, int MAXU>
__global__ void __launch_bounds__(256, 2) k_snd_multi(const __grid_constant__ DirMulti m) {
  __shared__ __align__(8) unsigned long long bars[2];
  __shared__ int s_item;
  init_bars(bars);
  int k0 = 0;
  for (;;) {
    if (threadIdx.x == 0 && threadIdx.y == 0) s_item = static_cast<int>(atomicAdd(m.queue, 1u));
    __syncthreads();
    const int i = s_item;
    __syncthreads();
    if (i >= m.total) return;
    int lo = 0, hi = m.nbeams - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (m.first[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const DirArgs& a = m.beam[lo];
    const int local = i - m.first[lo];
    if (!direct_cta<MODE, KW, NPL, MAXU>(a, local % m.ntx[lo], local / m.ntx[lo], bars, k0)) return;
    k0 += a.nchan / (kDG * a.sgroups);
  }
}

template <int MODE, int KW, int NPL, int MAXU>
cudaError_t run_direct(const DirArgs& a, dim3 grid, dim3 block, int smem, cudaStream_t s) {
  auto kern = k_snd<MODE, KW, NPL, MAXU>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <int MODE, int KW, int NPL, int MAXU>
cudaError_t run_direct_multi(const DirMulti& m, int ctas, dim3 block, int smem, cudaStream_t s) {
  auto kern = k_snd_multi<MODE, KW, NPL, MAXU>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  // persistent: as many CTAs as fit on the GPU at once (fewer if there are fewer items)
  int dev = 0, nsm = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, static_cast<int>(block.x * block.y), smem);
  if (e == cudaSuccess) e = cudaMemsetAsync(m.queue, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  const int grid = per_sm > 0 && nsm * per_sm < ctas ? nsm * per_sm : ctas;
  kern<<<grid, block, smem, s>>>(m);
  return cudaGetLastError();
}

struct DGoSingle {
  const DirArgs* a;
  dim3 grid, block;
  int smem;
  cudaStream_t s;
  template <int MODE, int KW, int NPL, int MAXU>
  cudaError_t go() { return run_direct<MODE, KW, NPL, MAXU>(*a, grid, block, smem, s); }
};

struct DGoMulti {
  const DirMulti* m;
  int ctas;
  dim3 block;
  int smem;
  cudaStream_t s;
  template <int MODE, int KW, int NPL, int MAXU>
  cudaError_t go() { return run_direct_multi<MODE, KW, NPL, MAXU>(*m, ctas, block, smem, s); }
};

template <typename F>
cudaError_t dispatch_direct(int id, F&& f) {
  switch (id) {
    case kDirFloat11: return f.template go<kFloat, 4, 11, 0>();
    case kDirFloat13: return f.template go<kFloat, 4, 13, 0>();
    case kDirGraded9U1: return f.template go<kGraded, 4, 9, 1>();
    case kDirGraded9U2: return f.template go<kGraded, 2, 9, 2>();
    case kDirGraded11U0: return f.template go<kGraded, 4, 11, 0>();
    case kDirGraded13U0: return f.template go<kGraded, 4, 13, 0>();
    case kDirBinary4: return f.template go<kBinary, 4, 1, 4>();
    case kDirBinary8: return f.template go<kBinary, 4, 1, 8>();
    case kDirBinary12: return f.template go<kBinary, 2, 1, 12>();
    case kDirBinReg2K1: return f.template go<kBinReg + 21, 4, 1, 4>();
    case kDirBinReg2K2: return f.template go<kBinReg + 22, 4, 1, 4>();
    case kDirBinReg4K1: return f.template go<kBinReg + 41, 4, 1, 4>();
    case kDirBinReg4K2: return f.template go<kBinReg + 42, 4, 1, 4>();
    case kDirBinReg8K1: return f.template go<kBinReg + 81, 4, 1, 3>();
    case kDirBinReg8K2: return f.template go<kBinReg + 82, 4, 1, 3>();
    default: return cudaErrorInvalidValue;
  }
}

void direct_args(const Plan& p, int64_t e_prev, int64_t e_new, DirArgs& a, int* ntx) {
  const DevPtrs& dp = p.dp;
  const DirectGeom& g = p.dgeom;
  a = DirArgs{};
  a.ring = dp.ring;
  a.R = p.R;
  a.nchan = p.nchan;
  a.ndm = p.ndm;
  a.B = p.B;
  a.KL = p.KL;
  a.KI = p.KI;
  a.N = p.N;
  a.nlev = p.nlev;
  for (int l = 0; l < kMaxLevels; ++l) a.level_nodes[l] = l < p.nlev ? p.level_nodes[l] : 1;
  a.sub_groups = g.sub_groups;
  a.sub_lev = g.sub_lev;
  a.meta = dp.dmeta;
  a.base4 = dp.dbase;
  a.cspan = g.cspan;
  a.sgroups = g.sgroups;
  a.tile_words = g.tile_words;
  a.word0 = e_prev >> 5;
  a.nwords = static_cast<int>(((e_new - 1) >> 5) - (e_prev >> 5) + 1);
  a.plane = dp.plane;
  a.Lp = p.Lp;
  a.status = dp.counters + kCntStatus;
  a.wait_cycles = p.wait_limit > 0 ? p.wait_limit : kDirWaitCycles;
  a.e_prev = e_prev;
  a.e_new = e_new;
  a.store = 1;
  a.level_fires = (p.flags & SND_FLAG_LEVEL_RATES) && p.mode == SND_MODE_BINARY ? dp.level_fires : nullptr;
  *ntx = (a.nwords + g.tile_words - 1) / g.tile_words;
}

}  // namespace

cudaError_t launch_tree_direct(const Plan& p, int64_t e_prev, int64_t e_new, cudaStream_t s) {
  if (e_new <= e_prev) return cudaSuccess;
  DirArgs a;
  int ntx = 0;
  direct_args(p, e_prev, e_new, a, &ntx);
  const DirectGeom& g = p.dgeom;
  const DevPtrs& dp = p.dp;
  p.launches += 1;
  DGoSingle go{&a, dim3(ntx, g.ndm_tiles), dim3(32, g.warps), g.smem_bytes, s};
  cudaError_t e = dispatch_direct(g.inst, go);
  if (e != cudaSuccess || !(p.flags & SND_FLAG_LEVEL_RATES) || p.mode == SND_MODE_BINARY) return e;
  // float / graded: a node is nonzero iff some channel of its subtree fired, i.e. iff the
  // same node of the binary tree with K_L = K_I = 1 fires; that tree's fire counts are the
  // per-level rates (a counting pass that writes no plane)
  DirArgs r = a;
  r.KL = r.KI = 1;
  r.store = 0;
  r.level_fires = dp.level_fires;
  r.tile_words = g.warps * g.rates_kw;
  p.launches += 1;
  DGoSingle gr{&r, dim3((r.nwords + r.tile_words - 1) / r.tile_words, g.ndm_tiles), dim3(32, g.warps), g.smem_bytes,
               s};
  return dispatch_direct(g.rates_inst, gr);
}

cudaError_t launch_tree_direct_batch(const Plan* const* plans, const int64_t* e_prev, const int64_t* e_new, int n,
                                     cudaStream_t s) {
  std::vector<int> done(n, 0);
  for (int i = 0; i < n; ++i) {
    if (done[i]) continue;
    const int key = plans[i]->dgeom.inst;
    const int warps = plans[i]->dgeom.warps;
    DirMulti m{};
    int smem = 0, ctas = 0;
    bool counted = false;
    for (int j = i; j < n && m.nbeams < kMaxDirBeams; ++j) {
      if (done[j] || plans[j]->dgeom.inst != key || plans[j]->dgeom.warps != warps) continue;
      done[j] = 1;
      if (e_new[j] <= e_prev[j]) continue;
      int ntx = 0;
      direct_args(*plans[j], e_prev[j], e_new[j], m.beam[m.nbeams], &ntx);
      m.first[m.nbeams] = ctas;
      m.ntx[m.nbeams] = ntx;
      ctas += ntx * plans[j]->dgeom.ndm_tiles;
      smem = smem > plans[j]->dgeom.smem_bytes ? smem : plans[j]->dgeom.smem_bytes;
      if (!counted) plans[j]->launches += 1;
      counted = true;
      ++m.nbeams;
    }
    if (m.nbeams == 0) continue;
    m.total = ctas;
    m.queue = reinterpret_cast<unsigned int*>(plans[i]->dp.counters + kCntTreeQueue);
    DGoMulti go{&m, ctas, dim3(32, warps), smem, s};
    const cudaError_t e = dispatch_direct(key, go);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace snd
