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

#include "snd_internal.h"

namespace snd {
namespace {

struct TreeArgs {
  const uint32_t* ring;
  int R, nchan, ndm, nleaves;
  int C, B, KL, KI, N, nlev;
  int level_nodes[kMaxLevels];
  const int32_t* tp_off;
  const int32_t* tp_pid;
  const int32_t* tp_smin;
  const int32_t* tp_leaf;
  const uint8_t* dl_lp;
  const int32_t* dl_sh;
  const int32_t* pat_rel;
  int G, span, maxpat;
  long long word0;  // absolute index of the first output word
  int nwords;       // output words of this call
  int32_t* plane;
  int Lp;
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

// Per-thread tree state for MODE.
template <int MODE, int MAXL, int KW, int TH>
struct TreeState;

template <int MAXL, int KW, int TH>
struct TreeState<kBinary, MAXL, KW, TH> {
  static constexpr int kLeafPlanes = 1;
  // acc[l][j][i] = 1[count of level-l node (word j) >= i + 1]  (thermometer code)
  uint32_t acc[MAXL][KW][TH];
  uint32_t root[KW];
  // one-hot word masks selecting the K_I plane (a runtime-indexed select would push the
  // accumulators to local memory)
  uint32_t ksel[TH];
  int cnt[MAXL], node[MAXL], fan[MAXL];
  __device__ __forceinline__ void init(const TreeArgs& a) {
#pragma unroll
    for (int i = 0; i < TH; ++i) ksel[i] = (i == a.KI - 1) ? 0xFFFFFFFFu : 0u;
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
#pragma unroll
      for (int j = 0; j < KW; ++j)
#pragma unroll
        for (int i = 0; i < TH; ++i) acc[l][j][i] = 0;
      cnt[l] = 0;
      node[l] = 0;
      fan[l] = (l >= 1 && l < a.nlev) ? min(a.B, a.level_nodes[l - 1]) : 1;
    }
#pragma unroll
    for (int j = 0; j < KW; ++j) root[j] = 0;
  }
  // leaf value from its channel bits (binary: quorum K_L over the cluster)
  __device__ __forceinline__ static void leaf(const TreeArgs& a, const uint32_t* x, int cs, uint32_t* out) {
    uint32_t t[TH];
#pragma unroll
    for (int i = 0; i < TH; ++i) t[i] = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c < cs) {
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
  __device__ __forceinline__ void push(const TreeArgs& a, uint32_t (*v)[1]) {
    if (a.nlev == 1) {
#pragma unroll
      for (int j = 0; j < KW; ++j) root[j] = v[j][0];
      return;
    }
    uint32_t cur[KW];
#pragma unroll
    for (int j = 0; j < KW; ++j) cur[j] = v[j][0];
#pragma unroll
    for (int l = 1; l < MAXL; ++l) {
      if (l >= a.nlev) break;
#pragma unroll
      for (int j = 0; j < KW; ++j) {
#pragma unroll
        for (int i = TH - 1; i > 0; --i) acc[l][j][i] |= acc[l][j][i - 1] & cur[j];
        acc[l][j][0] |= cur[j];
      }
      if (++cnt[l] < fan[l]) break;
#pragma unroll
      for (int j = 0; j < KW; ++j) {
        uint32_t r = 0;
#pragma unroll
        for (int i = 0; i < TH; ++i) {
          r |= acc[l][j][i] & ksel[i];
          acc[l][j][i] = 0;
        }
        cur[j] = r;
      }
      cnt[l] = 0;
      ++node[l];
      fan[l] = min(a.B, a.level_nodes[l - 1] - a.B * node[l]);
      if (l == a.nlev - 1) {
#pragma unroll
        for (int j = 0; j < KW; ++j) root[j] = cur[j];
      }
    }
  }
  __device__ __forceinline__ void store(int32_t* dst, int j) const { store_bits(dst, root[j]); }
};

template <int MAXL, int KW, int TH>
struct TreeState<kGraded, MAXL, KW, TH> {
  static constexpr int kLeafPlanes = 3;
  uint32_t acc[MAXL][KW][8];
  uint32_t root[KW][8];
  int cnt[MAXL], node[MAXL], fan[MAXL];
  __device__ __forceinline__ void init(const TreeArgs& a) {
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
#pragma unroll
      for (int j = 0; j < KW; ++j)
#pragma unroll
        for (int p = 0; p < 8; ++p) acc[l][j][p] = 0;
      cnt[l] = 0;
      node[l] = 0;
      fan[l] = (l >= 1 && l < a.nlev) ? min(a.B, a.level_nodes[l - 1]) : 1;
    }
#pragma unroll
    for (int j = 0; j < KW; ++j)
#pragma unroll
      for (int p = 0; p < 8; ++p) root[j][p] = 0;
  }
  __device__ __forceinline__ static void leaf(const TreeArgs& a, const uint32_t* x, int cs, uint32_t* out) {
    uint32_t c[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i < cs) {
        const uint32_t k0 = c[0] & x[i];
        c[0] ^= x[i];
        const uint32_t k1 = c[1] & k0;
        c[1] ^= k0;
        c[2] |= k1;
      }
    }
    if (a.N < 7) clamp_planes<3>(c, 0u, a.N);
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
  }
  __device__ __forceinline__ void push(const TreeArgs& a, uint32_t (*v)[3]) {
    uint32_t cur[KW][8];
#pragma unroll
    for (int j = 0; j < KW; ++j) {
#pragma unroll
      for (int p = 0; p < 8; ++p) cur[j][p] = (p < 3) ? v[j][p < 3 ? p : 0] : 0u;
    }
    if (a.nlev == 1) {
#pragma unroll
      for (int j = 0; j < KW; ++j)
#pragma unroll
        for (int p = 0; p < 8; ++p) root[j][p] = cur[j][p];
      return;
    }
#pragma unroll
    for (int l = 1; l < MAXL; ++l) {
      if (l >= a.nlev) break;
#pragma unroll
      for (int j = 0; j < KW; ++j) {
        // min(min(a+b,N)+c,N) = min(a+b+c,N) for non-negative values: saturate per child
        const uint32_t over = add_planes<8, 8>(acc[l][j], cur[j]);
        if (a.N == 255) {
#pragma unroll
          for (int p = 0; p < 8; ++p) acc[l][j][p] |= over;
        } else {
          clamp_planes<8>(acc[l][j], over, a.N);
        }
      }
      if (++cnt[l] < fan[l]) break;
#pragma unroll
      for (int j = 0; j < KW; ++j)
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          cur[j][p] = acc[l][j][p];
          acc[l][j][p] = 0;
        }
      cnt[l] = 0;
      ++node[l];
      fan[l] = min(a.B, a.level_nodes[l - 1] - a.B * node[l]);
      if (l == a.nlev - 1) {
#pragma unroll
        for (int j = 0; j < KW; ++j)
#pragma unroll
          for (int p = 0; p < 8; ++p) root[j][p] = cur[j][p];
      }
    }
  }
  __device__ __forceinline__ void store(int32_t* dst, int j) const { store_word<8>(dst, root[j]); }
};

template <int MAXL, int KW, int TH>
struct TreeState<kFloat, MAXL, KW, TH> {
  // Mode C has no per-node rule, so the root count is the sum of all leaf counts: a small
  // 6-plane counter (flushed every 9 leaves, <= 63) feeding a 16-plane counter.
  static constexpr int kLeafPlanes = 3;
  uint32_t small[KW][6];
  uint32_t big[KW][16];
  int nsmall;
  __device__ __forceinline__ void init(const TreeArgs&) {
#pragma unroll
    for (int j = 0; j < KW; ++j) {
#pragma unroll
      for (int p = 0; p < 6; ++p) small[j][p] = 0;
#pragma unroll
      for (int p = 0; p < 16; ++p) big[j][p] = 0;
    }
    nsmall = 0;
  }
  __device__ __forceinline__ static void leaf(const TreeArgs&, const uint32_t* x, int cs, uint32_t* out) {
    uint32_t c[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i < cs) {
        const uint32_t k0 = c[0] & x[i];
        c[0] ^= x[i];
        const uint32_t k1 = c[1] & k0;
        c[1] ^= k0;
        c[2] |= k1;
      }
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
  }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int j = 0; j < KW; ++j) {
      add_planes<16, 6>(big[j], small[j]);
#pragma unroll
      for (int p = 0; p < 6; ++p) small[j][p] = 0;
    }
    nsmall = 0;
  }
  __device__ __forceinline__ void push(const TreeArgs&, uint32_t (*v)[3]) {
#pragma unroll
    for (int j = 0; j < KW; ++j) add_planes<6, 3>(small[j], v[j]);
    if (++nsmall == 9) flush();
  }
  __device__ __forceinline__ void finish() { flush(); }
  __device__ __forceinline__ void store(int32_t* dst, int j) const { store_word<16>(dst, big[j]); }
};

template <int MODE, int MAXL, int KW, int TH>
__global__ void __launch_bounds__(256) k_tree(TreeArgs a) {
  using State = TreeState<MODE, MAXL, KW, TH>;
  constexpr int PL = State::kLeafPlanes;
  extern __shared__ __align__(16) uint32_t sm[];
  const int DT = blockDim.y;
  const int lane = threadIdx.x, wd = threadIdx.y;
  const int tid = wd * 32 + lane, nthr = 32 * DT;
  constexpr int TW = 32 * KW;
  const int tile = blockIdx.y;
  const long long aw0 = a.word0 + static_cast<long long>(blockIdx.x) * TW;
  const int awp = static_cast<int>(aw0 % a.R);
  const int drow = tile * DT + wd;
  const int d = min(drow, a.ndm - 1);
  const int NL = a.nleaves, C = a.C, G = a.G, span = a.span;

  uint32_t* series = sm;                                                   // maxpat*PL*span
  uint32_t* meta = series + static_cast<size_t>(a.maxpat) * PL * span;     // DT*G
  int* eoff = reinterpret_cast<int*>(meta + DT * G);                        // maxpat*C
  int* esh = eoff + a.maxpat * C;                                           // maxpat*C
  int* eleaf = esh + a.maxpat * C;                                          // maxpat

  State st;
  st.init(a);

  for (int g0 = 0; g0 < NL; g0 += G) {
    const int g1 = min(NL, g0 + G);
    const int ng = g1 - g0;
    const int ebase = a.tp_off[tile * NL + g0];
    const int ne = a.tp_off[tile * NL + g1] - ebase;
    for (int i = tid; i < ne; i += nthr) {
      const int pid = a.tp_pid[ebase + i];
      const int smin = a.tp_smin[ebase + i];
      eleaf[i] = a.tp_leaf[ebase + i];
      for (int ci = 0; ci < C; ++ci) {
        const int rel = a.pat_rel[pid * C + ci];
        eoff[i * C + ci] = (smin >> 5) + (rel >> 5);
        esh[i * C + ci] = rel & 31;
      }
    }
    for (int i = tid; i < DT * ng; i += nthr) {
      const int dl = i / ng, kl = i - dl * ng;
      const int dd = min(tile * DT + dl, a.ndm - 1);
      const int k = g0 + kl;
      const size_t at = static_cast<size_t>(dd) * NL + k;
      const int s = a.dl_sh[at];
      const int e = a.tp_off[tile * NL + k] - ebase + a.dl_lp[at];
      const int j0 = (s >> 5) - (a.tp_smin[ebase + e] >> 5);
      meta[dl * G + kl] = (static_cast<uint32_t>(e * PL * span + j0) << 5) | static_cast<uint32_t>(s & 31);
    }
    __syncthreads();
    // phase 1: distinct (leaf, pattern) series of this group
    for (int it = tid; it < ne * span; it += nthr) {
      const int e = it / span, j = it - e * span;
      const int c0 = eleaf[e] * C;
      const int cs = min(C, a.nchan - c0);
      uint32_t x[8];
#pragma unroll
      for (int ci = 0; ci < 8; ++ci) {
        if (ci < cs) {
          const uint32_t* row = a.ring + static_cast<size_t>(c0 + ci) * 2 * a.R;
          const int ph = awp + eoff[e * C + ci] + j;
          x[ci] = funnel(__ldg(row + ph), __ldg(row + ph + 1), esh[e * C + ci]);
        } else {
          x[ci] = 0;
        }
      }
      uint32_t v[PL];
      State::leaf(a, x, cs, v);
#pragma unroll
      for (int p = 0; p < PL; ++p) series[(e * PL + p) * span + j] = v[p];
    }
    __syncthreads();
    // phase 2: every DM gathers its leaf values and pushes them up its tree
    for (int kl = 0; kl < ng; ++kl) {
      const uint32_t m = meta[wd * G + kl];
      const int off = static_cast<int>(m >> 5);
      const int sh = static_cast<int>(m & 31);
      uint32_t v[KW][PL];
#pragma unroll
      for (int jw = 0; jw < KW; ++jw) {
        const int w = lane + 32 * jw;
#pragma unroll
        for (int p = 0; p < PL; ++p) {
          const uint32_t* s = series + off + p * span + w;
          v[jw][p] = funnel(s[0], s[1], sh);
        }
      }
      st.push(a, v);
    }
    __syncthreads();
  }
  if constexpr (MODE == kFloat) st.finish();
  if (drow >= a.ndm) return;
  const int lw = a.Lp >> 5;
#pragma unroll
  for (int jw = 0; jw < KW; ++jw) {
    const long long aw = aw0 + lane + 32 * jw;
    if (aw - a.word0 >= a.nwords) continue;
    const int col = static_cast<int>(aw % lw) * 32;
    st.store(a.plane + static_cast<size_t>(d) * a.Lp + col, jw);
  }
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

template <int MODE, int MAXL, int KW, int TH>
cudaError_t run_tree(const TreeArgs& a, dim3 grid, dim3 block, int smem, cudaStream_t s) {
  auto kern = k_tree<MODE, MAXL, KW, TH>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <int MODE, int KW, int TH>
cudaError_t dispatch_levels(const Plan& p, const TreeArgs& a, dim3 grid, dim3 block, int smem,
                            cudaStream_t s) {
  if (p.nlev <= 4) return run_tree<MODE, 4, KW, TH>(a, grid, block, smem, s);
  if (p.nlev <= 8) return run_tree<MODE, 8, KW, TH>(a, grid, block, smem, s);
  return run_tree<MODE, 16, KW, TH>(a, grid, block, smem, s);
}

}  // namespace

int tree_kw(int mode, int nlev, int kmax) {
  const int maxl = nlev <= 4 ? 4 : (nlev <= 8 ? 8 : 16);
  const int per_level = (mode == SND_MODE_BINARY) ? (kmax <= 2 ? 2 : 8) : (mode == SND_MODE_GRADED ? 8 : 0);
  return (maxl * per_level * 2 <= 64) ? 2 : 1;
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
  TreeArgs a{};
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
  a.tp_pid = dp.tp_pid;
  a.tp_smin = dp.tp_smin;
  a.tp_leaf = dp.tp_leaf;
  a.dl_lp = dp.dl_lp;
  a.dl_sh = dp.dl_sh;
  a.pat_rel = dp.pat_rel;
  a.G = p.geom.group_leaves;
  a.span = p.geom.span;
  a.maxpat = p.geom.max_pat_group;
  a.word0 = e_prev >> 5;
  a.nwords = static_cast<int>(((e_new - 1) >> 5) - (e_prev >> 5) + 1);
  a.plane = dp.plane;
  a.Lp = p.Lp;
  const TreeGeom& g = p.geom;
  dim3 block(32, g.dms_per_cta);
  dim3 grid((a.nwords + g.tile_words - 1) / g.tile_words, g.ndm_tiles);
  const int smem = g.smem_bytes;
  p.launches += 1;
  if (p.mode == SND_MODE_BINARY) {
    const int kmax = p.KL > p.KI ? p.KL : p.KI;
    if (kmax <= 2) {
      if (g.kw == 1) return dispatch_levels<kBinary, 1, 2>(p, a, grid, block, smem, s);
      return dispatch_levels<kBinary, 2, 2>(p, a, grid, block, smem, s);
    }
    if (g.kw == 1) return dispatch_levels<kBinary, 1, 8>(p, a, grid, block, smem, s);
    return dispatch_levels<kBinary, 2, 8>(p, a, grid, block, smem, s);
  }
  if (p.mode == SND_MODE_GRADED) {
    if (g.kw == 1) return dispatch_levels<kGraded, 1, 1>(p, a, grid, block, smem, s);
    return dispatch_levels<kGraded, 2, 1>(p, a, grid, block, smem, s);
  }
  return run_tree<kFloat, 4, 2, 1>(a, grid, block, smem, s);
}

}  // namespace snd
