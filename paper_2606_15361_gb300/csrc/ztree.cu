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
// windows (the tile's smallest delay per channel onwards, tile width + the tile's delay
// spread) are staged from the payload ring in shared memory, twice (as stored and shifted by
// one value) so that every pair is one aligned load. The open nodes of every level are
// per-thread FP32 registers (MAXL levels x 2 NP samples).

#include <cuda_fp16.h>

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

template <typename ST> struct PairT;           // two stored values
template <> struct PairT<__half> { using T = uint32_t; };
template <> struct PairT<float> { using T = uint2; };

// one 16-byte chunk of stored values shifted by one value: (a1 .. a_last, b0)
__device__ __forceinline__ uint4 shift_one(uint4 a, uint4 b, const __half*) {
  return make_uint4(__byte_perm(a.x, a.y, 0x5432), __byte_perm(a.y, a.z, 0x5432), __byte_perm(a.z, a.w, 0x5432),
                    __byte_perm(a.w, b.x, 0x5432));
}
__device__ __forceinline__ uint4 shift_one(uint4 a, uint4 b, const float*) { return make_uint4(a.y, a.z, a.w, b.x); }

// CTA = DT trial DMs (one warp each) x 64 NP consecutive output samples: lane L holds samples
// t0 + 64 j + 2 L and + 1 (pair slot j < NP). Per staged channel, shared memory holds its window
// twice: as stored (copy 0) and shifted by one value (copy 1), both from a 16-byte aligned ring
// position; a DM whose offset into the window is even reads its pairs from copy 0, odd from
// copy 1, so every pair is one aligned 4- (FP16) or 8-byte (FP32) load.
template <typename ST, int MAXL, int NP, int CT>
__global__ void __launch_bounds__(512, 2) k_tree_z(ZArgs a) {
  using P2 = typename PairT<ST>::T;
  constexpr int EPC = 16 / sizeof(ST);  // stored values per 16-byte chunk
  extern __shared__ __align__(16) unsigned char zsm[];
  const int DT = blockDim.y;
  const int lane = threadIdx.x, wd = threadIdx.y, tid = wd * 32 + lane, nthr = 32 * DT;
  const int tile = blockIdx.y;
  const long long tb = a.t0 + static_cast<long long>(blockIdx.x) * (64 * NP);
  const int d = tile * DT + wd;
  const bool active = d < a.ndm;
  const int GC = a.G * a.C;
  const int WZ = a.win + 2 * EPC;  // staged values per copy: the window, its alignment slack and one chunk
  const int nck = WZ / EPC;        // chunks per copy
  ST* win = reinterpret_cast<ST*>(zsm);  // [GC][2][WZ]
  int* drel = reinterpret_cast<int*>(zsm + static_cast<size_t>(GC) * 2 * WZ * sizeof(ST));
  const ST* ring = static_cast<const ST*>(a.zring);
  const int* wb = a.zwb + static_cast<size_t>(tile) * a.nchan;

  float acc[MAXL][2 * NP];
  float root[2 * NP];
#pragma unroll
  for (int l = 0; l < MAXL; ++l)
#pragma unroll
    for (int j = 0; j < 2 * NP; ++j) acc[l][j] = 0.0f;
#pragma unroll
  for (int j = 0; j < 2 * NP; ++j) root[j] = 0.0f;

  for (int k0 = 0; k0 < a.nleaves; k0 += a.G) {
    const int k1 = min(a.nleaves, k0 + a.G);
    const int c0 = k0 * a.C, nc = min(a.nchan, k1 * a.C) - c0;
    __syncthreads();  // the previous group's readers are done
    // stage: a warp per channel, chunk q of it from ring samples (start & ~(EPC-1)) + EPC q
    // (Rz is a multiple of EPC, so a chunk never straddles the ring's end)
    for (int cl = wd; cl < nc; cl += DT) {
      const int c = c0 + cl;
      const ST* row = ring + static_cast<size_t>(c) * a.Rz;
      const int r0 = static_cast<int>(((tb + wb[c]) & ~static_cast<long long>(EPC - 1)) % a.Rz);
      ST* dst = win + static_cast<size_t>(cl) * 2 * WZ;
      for (int q = lane; q < nck; q += 32) {
        int r = r0 + q * EPC;
        if (r >= a.Rz) r -= a.Rz;
        const uint4 x = *reinterpret_cast<const uint4*>(row + r);
        r += EPC;
        if (r >= a.Rz) r -= a.Rz;
        const uint4 y = *reinterpret_cast<const uint4*>(row + r);
        *reinterpret_cast<uint4*>(dst + q * EPC) = x;
        *reinterpret_cast<uint4*>(dst + WZ + q * EPC) = shift_one(x, y, ring);
      }
    }
    for (int i = tid; i < DT * nc; i += nthr) {
      const int w = i / nc, cl = i - w * nc;
      const int dd = min(tile * DT + w, a.ndm - 1);
      const int c = c0 + cl;
      const int slack = static_cast<int>((tb + wb[c]) & (EPC - 1));
      drel[w * GC + cl] = a.delays[static_cast<size_t>(dd) * a.nchan + c] - wb[c] + slack;
    }
    __syncthreads();
    if (!active) continue;
    // pairs of channel cl: copy (rel & 1), pair index rel / 2 + 32 j + lane
    auto pairs = [&](int cl) -> const P2* {
      const int rel = drel[wd * GC + cl];
      return reinterpret_cast<const P2*>(win + static_cast<size_t>(cl) * 2 * WZ + (rel & 1) * WZ + (rel & ~1)) + lane;
    };
    for (int k = k0; k < k1; ++k) {
      const int cl0 = (k - k0) * a.C;
      const int cn = min(a.C, a.nchan - k * a.C);
      float v[2 * NP];
#pragma unroll
      for (int j = 0; j < 2 * NP; ++j) v[j] = 0.0f;
      if (CT) {
        // C channels known at compile time: all C x NP loads of the leaf are independent
        P2 x[CT > 0 ? CT : 1][NP];
#pragma unroll
        for (int ci = 0; ci < CT; ++ci) {
          const P2* src = pairs(cl0 + ci);
#pragma unroll
          for (int j = 0; j < NP; ++j) x[ci][j] = src[32 * j];
        }
#pragma unroll
        for (int ci = 0; ci < CT; ++ci)
#pragma unroll
          for (int j = 0; j < NP; ++j) add_pair(v[2 * j], v[2 * j + 1], x[ci][j], ring);
      } else {
        for (int ci = 0; ci < cn; ++ci) {
          const P2* src = pairs(cl0 + ci);
#pragma unroll
          for (int j = 0; j < NP; ++j) add_pair(v[2 * j], v[2 * j + 1], src[32 * j], ring);
        }
      }
      if (a.nlev == 1) {  // a single leaf is the root: its FP32 sum is not stored
#pragma unroll
        for (int j = 0; j < 2 * NP; ++j) root[j] = v[j];
        continue;
      }
      // the stored leaf goes into its parent's sum (acc[l] holds the open node of level l + 1);
      // when it is the parent's last child the parent is finished, and so on up `depth`
      // levels. depth depends on the leaf only, so the branch is warp-uniform and taken by one
      // leaf in B.
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
