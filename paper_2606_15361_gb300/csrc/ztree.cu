// Labelled-payload Mode C tree with stored partial sums (Methods, "Tree activation modes",
// Mode C; payload x_c(t) = z_c(t) 1[P_c(t) >= u_c] from "Input encoding").
//
// Each node below the root is stored in ST (FP16 or FP32) before its parent reads it, and
// every node adds its children in index order in FP32 starting from 0 (a leaf's children
// are its C channel payloads, already in ST). The root stays FP32; the plane is
// root * fp32(1/sqrt(N_f)). The tree is evaluated per (DM, output time) in "absolute time"
// form: channel c of DM d is read at t + delta_c(d), so the node values equal those of the
// paper's per-node delay lines and the rounding points are exactly the node outputs.
//
// CTA = 16 trial DMs (one warp each) x 64*NP consecutive output samples; lane L holds the
// sample pairs t0 + 64 j + 2 L, + 1 (slot j). Leaves are processed in groups whose channel
// windows (from a 16-byte aligned ring position at or before the tile's smallest delay per
// channel: tile width + the tile's delay spread) are copied by the TMA engine into one of two
// shared-memory buffers while the previous group is summed from the other. The open nodes of
// every level are per-thread FP32 registers (MAXL levels x 2 NP samples).

#include <cuda_fp16.h>

#include "bulk.h"
#include "snd_internal.h"

namespace snd {
namespace {

struct ZArgs {
  const void* zring;
  int Rz, nchan, ndm, nleaves, C, B, nlev;
  int level_nodes[kMaxLevels];
  const int32_t* delays;  // [ndm][nchan]
  const int32_t* zwb;     // [ndm_tiles][nchan]
  const int32_t* carry;   // [nleaves] levels a finished leaf completes (its carry depth)
  int win, G;             // staged samples per channel, leaves per group
  long long t0;           // first output sample of this call
  int nout;
  float* out;             // plane ring (omode 0, column t mod Lp) or caller plane (omode 1, column t - t0)
  long long ostride;
  int omode, Lp;
  float scale;
  uint32_t* status;        // plan status word (a staging wait that gives up sets kStatusTreeTimeout)
  long long wait_cycles;   // bound of a staging wait (clock cycles)
};

// Two consecutive stored values x = (lo, hi) added to two FP32 sums: lo_sum += lo, hi_sum += hi,
// each rounded once to nearest. FP16: the mixed-precision add of the sm_100 family takes the
// FP16 operand as is (its conversion to FP32 is exact), so each result equals
// fp32(value) + sum rounded once, as an FP32 add of the converted value would give.
__device__ __forceinline__ void add_pair(float& lo_sum, float& hi_sum, uint32_t x, const __half*) {
  asm("{\n .reg .b16 l, h;\n mov.b32 {l, h}, %2;\n add.rn.f32.f16 %0, l, %0;\n add.rn.f32.f16 %1, h, %1;\n}"
      : "+f"(lo_sum), "+f"(hi_sum)
      : "r"(x));
}
__device__ __forceinline__ void add_pair(float& lo_sum, float& hi_sum, uint2 x, const float*) {
  lo_sum = __fadd_rn(lo_sum, __uint_as_float(x.x));
  hi_sum = __fadd_rn(hi_sum, __uint_as_float(x.y));
}
// parent += stored(v): the value rounded to the storage type, added in FP32
__device__ __forceinline__ float add_stored(float parent, float v, const __half*) {
  const __half h = __float2half_rn(v);
  float r;
  asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(r) : "h"(__half_as_ushort(h)), "f"(parent));
  return r;
}
__device__ __forceinline__ float add_stored(float parent, float v, const float*) { return __fadd_rn(parent, v); }

// the pair (window[i], window[i + 1]) of a staged channel window, i = 2 k + odd: one aligned
// load, or for an odd start two aligned words and a byte permute
__device__ __forceinline__ uint32_t load_pair(const __half* w, int k, bool odd) {
  const uint32_t* W = reinterpret_cast<const uint32_t*>(w);
  if (!odd) return W[k];
  return __byte_perm(W[k], W[k + 1], 0x5432);
}
__device__ __forceinline__ uint2 load_pair(const float* w, int k, bool odd) {
  if (!odd) return reinterpret_cast<const uint2*>(w)[k];
  return make_uint2(__float_as_uint(w[2 * k + 1]), __float_as_uint(w[2 * k + 2]));
}
template <typename ST> struct PairT;           // two stored values
template <> struct PairT<__half> { using T = uint32_t; };
template <> struct PairT<float> { using T = uint2; };

// CTA = DT trial DMs (one warp each) x 64 NP consecutive output samples: lane L holds samples
// t0 + 64 j + 2 L and + 1 (pair slot j < NP). Leaves are processed in groups of G; a group's
// channel windows (each from a 16-byte aligned ring position: the tile's smallest delay, the
// tile width and its delay spread) are copied by the TMA engine into one of two shared-memory
// buffers while the previous group is summed from the other, so staging overlaps the adds.
template <typename ST, int MAXL, int NP, int CT>
__global__ void __launch_bounds__(512, 2) k_tree_z(const __grid_constant__ ZArgs a) {
  using P2 = typename PairT<ST>::T;
  constexpr int EPC = 16 / sizeof(ST);  // stored values per 16 bytes
  extern __shared__ __align__(16) unsigned char zsm[];
  __shared__ __align__(8) unsigned long long bars[2];
  const int DT = blockDim.y;
  const int lane = threadIdx.x, wd = threadIdx.y, tid = wd * 32 + lane, nthr = 32 * DT;
  const int tile = blockIdx.y;
  const long long tb = a.t0 + static_cast<long long>(blockIdx.x) * (64 * NP);
  const int d = tile * DT + wd;
  const bool active = d < a.ndm;
  const int GC = a.G * a.C;
  const int WZ = a.win + 2 * EPC;  // staged values per channel: the window, its slack and one chunk
  const size_t bufb = static_cast<size_t>(GC) * WZ * sizeof(ST) + static_cast<size_t>(4) * DT * GC;
  const ST* ring = static_cast<const ST*>(a.zring);
  const int* wb = a.zwb + static_cast<size_t>(tile) * a.nchan;
  const int ngroups = (a.nleaves + a.G - 1) / a.G;
  if (tid == 0) {
    bar_init(smem_u32(&bars[0]), 1);
    bar_init(smem_u32(&bars[1]), 1);
    bar_init_fence();
  }
  __syncthreads();

  // stage group gi into buffer gi & 1: warp 0 issues one bulk copy per channel window (two
  // across the ring's end) after announcing the bytes; every thread fills the DM offsets
  auto issue = [&](int gi) {
    unsigned char* buf = zsm + (gi & 1) * bufb;
    ST* win = reinterpret_cast<ST*>(buf);
    int* drel = reinterpret_cast<int*>(buf + static_cast<size_t>(GC) * WZ * sizeof(ST));
    const int c0 = gi * a.G * a.C, nc = min(a.nchan, (gi + 1) * a.G * a.C) - c0;
    if (wd == 0) {
      const uint32_t bar = smem_u32(&bars[gi & 1]);
      // the buffer was last read by generic loads, before the barrier that ended that group
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (lane == 0) bar_expect(bar, static_cast<uint32_t>(nc) * WZ * sizeof(ST));
      __syncwarp();
      for (int cl = lane; cl < nc; cl += 32) {
        const int c = c0 + cl;
        const ST* row = ring + static_cast<size_t>(c) * a.Rz;
        const int r0 = static_cast<int>(((tb + wb[c]) & ~static_cast<long long>(EPC - 1)) % a.Rz);
        const int n1 = min(WZ, a.Rz - r0);
        ST* dst = win + static_cast<size_t>(cl) * WZ;
        bulk_g2s(smem_u32(dst), row + r0, static_cast<uint32_t>(n1 * sizeof(ST)), bar);
        if (n1 < WZ) bulk_g2s(smem_u32(dst + n1), row, static_cast<uint32_t>((WZ - n1) * sizeof(ST)), bar);
      }
    }
    for (int i = tid; i < DT * nc; i += nthr) {
      const int w = i / nc, cl = i - w * nc;
      const int dd = min(tile * DT + w, a.ndm - 1);
      const int c = c0 + cl;
      const int slack = static_cast<int>((tb + wb[c]) & (EPC - 1));
      drel[w * GC + cl] = a.delays[static_cast<size_t>(dd) * a.nchan + c] - wb[c] + slack;
    }
  };

  float acc[MAXL][2 * NP];
  float root[2 * NP];
#pragma unroll
  for (int l = 0; l < MAXL; ++l)
#pragma unroll
    for (int j = 0; j < 2 * NP; ++j) acc[l][j] = 0.0f;
#pragma unroll
  for (int j = 0; j < 2 * NP; ++j) root[j] = 0.0f;

  issue(0);
  __syncthreads();  // group 0's DM offsets
  for (int gi = 0; gi < ngroups; ++gi) {
    if (gi + 1 < ngroups) issue(gi + 1);  // its buffer was released by the last barrier
    const bool ok = bar_wait(smem_u32(&bars[gi & 1]), (gi >> 1) & 1, a.wait_cycles);
    if (__syncthreads_or(!ok)) {
      // a staging wait ran out: report it, and let the copies in flight land (normal bound)
      // before the CTA's shared memory is released
      if (tid == 0) {
        atomicOr(a.status, kStatusTreeTimeout);
        for (int g2 = gi; g2 < gi + 2 && g2 < ngroups; ++g2)
          bar_wait(smem_u32(&bars[g2 & 1]), (g2 >> 1) & 1, kStageWaitCycles);
      }
      return;
    }
    const unsigned char* buf = zsm + (gi & 1) * bufb;
    const ST* win = reinterpret_cast<const ST*>(buf);
    const int* drel = reinterpret_cast<const int*>(buf + static_cast<size_t>(GC) * WZ * sizeof(ST));
    const int k0 = gi * a.G, k1 = min(a.nleaves, k0 + a.G);
    if (active) {
      for (int k = k0; k < k1; ++k) {
        const int cl0 = (k - k0) * a.C;
        const int cn = min(a.C, a.nchan - k * a.C);
        float v[2 * NP];
#pragma unroll
        for (int j = 0; j < 2 * NP; ++j) v[j] = 0.0f;
        auto add_channel = [&](int cl) {
          const int rel = drel[wd * GC + cl];
          const ST* w = win + static_cast<size_t>(cl) * WZ;
          const int kb = (rel >> 1) + lane;
          const bool odd = rel & 1;
          P2 x[NP];
#pragma unroll
          for (int j = 0; j < NP; ++j) x[j] = load_pair(w, kb + 32 * j, odd);
#pragma unroll
          for (int j = 0; j < NP; ++j) add_pair(v[2 * j], v[2 * j + 1], x[j], ring);
        };
        if (CT) {
#pragma unroll
          for (int ci = 0; ci < (CT > 0 ? CT : 1); ++ci) add_channel(cl0 + ci);
        } else {
          for (int ci = 0; ci < cn; ++ci) add_channel(cl0 + ci);
        }
        if (a.nlev == 1) {  // a single leaf is the root: its FP32 sum is not stored
#pragma unroll
          for (int j = 0; j < 2 * NP; ++j) root[j] = v[j];
          continue;
        }
        // the stored leaf goes into its parent's sum (acc[l] holds the open node of level
        // l + 1); when it is the parent's last child the parent is finished, and so on up
        // `depth` levels. depth depends on the leaf only, so the branch is warp-uniform and
        // taken by one leaf in B.
#pragma unroll
        for (int j = 0; j < 2 * NP; ++j) acc[0][j] = add_stored(acc[0][j], v[j], ring);
        const int depth = __ldg(a.carry + k);
        if (depth > 0) {
#pragma unroll
          for (int l = 0; l + 1 < MAXL; ++l) {
            if (l < depth) {
              const bool to_root = (l + 1 == a.nlev - 1);
#pragma unroll
              for (int j = 0; j < 2 * NP; ++j) {
                const float x = acc[l][j];
                acc[l][j] = 0.0f;
                if (to_root) {
                  root[j] = x;
                } else {
                  acc[l + 1][j] = add_stored(acc[l + 1][j], x, ring);
                }
              }
            }
          }
        }
      }
    }
    __syncthreads();  // every reader of this buffer is done: the group after next may refill it
  }
  if (!active) return;
  float* orow = a.out + static_cast<size_t>(d) * a.ostride;
#pragma unroll
  for (int j = 0; j < 2 * NP; ++j) {
    const long long t = tb + 64 * (j >> 1) + 2 * lane + (j & 1);
    if (t - a.t0 >= a.nout) continue;
    const long long col = a.omode ? (t - a.t0) : (t % a.Lp);
    orow[col] = __fmul_rn(root[j], a.scale);
  }
}

template <typename ST, int MAXL, int NP>
cudaError_t run_z(const ZArgs& a, dim3 grid, dim3 block, int smem, cudaStream_t s) {
  // the compile-time 4-channel leaf applies when every leaf has 4 channels
  auto kern = (a.C == 4 && a.nchan % 4 == 0) ? k_tree_z<ST, MAXL, NP, 4> : k_tree_z<ST, MAXL, NP, 0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tree_z(const Plan& p, int64_t e_prev, int64_t e_new, void* d_plane_out, cudaStream_t s) {
  if (e_new <= e_prev) return cudaSuccess;
  const ZGeom& z = p.zgeom;
  ZArgs a{};
  a.zring = p.dp.zring;
  a.Rz = z.Rz;
  a.nchan = p.nchan;
  a.ndm = p.ndm;
  a.nleaves = p.nleaves;
  a.C = p.C;
  a.B = p.B;
  a.nlev = p.nlev;
  for (int l = 0; l < kMaxLevels; ++l) a.level_nodes[l] = l < p.nlev ? p.level_nodes[l] : 1;
  a.delays = p.dp.delays;
  a.zwb = p.dp.zwb;
  a.carry = p.dp.zcarry;
  a.win = z.win;
  a.G = z.group_leaves;
  a.t0 = e_prev;
  a.nout = static_cast<int>(e_new - e_prev);
  if (d_plane_out) {
    a.out = static_cast<float*>(d_plane_out);
    a.ostride = a.nout;
    a.omode = 1;
  } else {
    a.out = reinterpret_cast<float*>(p.dp.plane);
    a.ostride = p.Lp;
    a.omode = 0;
  }
  a.Lp = p.Lp;
  a.scale = static_cast<float>(1.0 / std::sqrt(static_cast<double>(p.nchan)));
  a.status = p.dp.counters + kCntStatus;
  a.wait_cycles = p.wait_limit > 0 ? p.wait_limit : kStageWaitCycles;
  dim3 block(32, z.dms_per_cta);
  dim3 grid(static_cast<unsigned>((a.nout + z.tile_samples - 1) / z.tile_samples), z.ndm_tiles);
  p.launches += 1;
  if (z.fp16) {
    if (z.maxl == 4) return run_z<__half, 4, 4>(a, grid, block, z.smem_bytes, s);
    if (z.maxl == 8) return run_z<__half, 8, 2>(a, grid, block, z.smem_bytes, s);
    return run_z<__half, 16, 1>(a, grid, block, z.smem_bytes, s);
  }
  if (z.maxl == 4) return run_z<float, 4, 4>(a, grid, block, z.smem_bytes, s);
  if (z.maxl == 8) return run_z<float, 8, 2>(a, grid, block, z.smem_bytes, s);
  return run_z<float, 16, 1>(a, grid, block, z.smem_bytes, s);
}

}  // namespace snd
