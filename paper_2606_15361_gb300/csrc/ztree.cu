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
// CTA = 16 trial DMs (one warp each) x 32*SPT consecutive output samples; sample
// t0 + j*32 + lane belongs to lane `lane`, slot j. Leaves are processed in groups whose
// channel windows (the tile's smallest delay per channel onwards, tile width + the tile's
// delay spread) are staged from the payload ring in shared memory. The open nodes of every
// level are per-thread FP32 registers (MAXL levels x SPT samples).

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

__device__ __forceinline__ float zload(const float* p) { return *p; }
__device__ __forceinline__ float zload(const __half* p) { return __half2float(*p); }
__device__ __forceinline__ float zstore_round(float v, const float*) { return v; }
__device__ __forceinline__ float zstore_round(float v, const __half*) { return __half2float(__float2half_rn(v)); }

template <typename ST, int MAXL, int SPT, int CT>
__global__ void __launch_bounds__(512, 2) k_tree_z(ZArgs a) {
  extern __shared__ __align__(16) unsigned char zsm[];
  const int DT = blockDim.y;
  const int lane = threadIdx.x, wd = threadIdx.y, tid = wd * 32 + lane, nthr = 32 * DT;
  const int tile = blockIdx.y;
  const long long tb = a.t0 + static_cast<long long>(blockIdx.x) * (32 * SPT);
  const int d = tile * DT + wd;
  const bool active = d < a.ndm;
  const int GC = a.G * a.C;
  ST* win = reinterpret_cast<ST*>(zsm);
  int* drel = reinterpret_cast<int*>(zsm + ((static_cast<size_t>(GC) * a.win * sizeof(ST) + 15) & ~size_t(15)));
  const ST* ring = static_cast<const ST*>(a.zring);
  const int* wb = a.zwb + static_cast<size_t>(tile) * a.nchan;

  float acc[MAXL][SPT];
  float root[SPT];
#pragma unroll
  for (int l = 0; l < MAXL; ++l)
#pragma unroll
    for (int j = 0; j < SPT; ++j) acc[l][j] = 0.0f;
#pragma unroll
  for (int j = 0; j < SPT; ++j) root[j] = 0.0f;

  for (int k0 = 0; k0 < a.nleaves; k0 += a.G) {
    const int k1 = min(a.nleaves, k0 + a.G);
    const int c0 = k0 * a.C, nc = min(a.nchan, k1 * a.C) - c0;
    __syncthreads();  // the previous group's readers are done
    for (int cl = wd; cl < nc; cl += DT) {
      const int c = c0 + cl;
      const int ph = static_cast<int>((tb + wb[c]) % a.Rz);
      const ST* row = ring + static_cast<size_t>(c) * a.Rz;
      ST* dst = win + static_cast<size_t>(cl) * a.win;
      // the window may wrap around the ring end: copy the two runs
      const int n1 = min(a.win, a.Rz - ph);
      for (int i = lane; i < n1; i += 32) dst[i] = row[ph + i];
      for (int i = n1 + lane; i < a.win; i += 32) dst[i] = row[i - n1];
    }
    for (int i = tid; i < DT * nc; i += nthr) {
      const int w = i / nc, cl = i - w * nc;
      const int dd = min(tile * DT + w, a.ndm - 1);
      drel[w * GC + cl] = a.delays[static_cast<size_t>(dd) * a.nchan + c0 + cl] - wb[c0 + cl];
    }
    __syncthreads();
    if (!active) continue;
    for (int k = k0; k < k1; ++k) {
      const int cl0 = (k - k0) * a.C;
      const int cn = min(a.C, a.nchan - k * a.C);
      float v[SPT];
#pragma unroll
      for (int j = 0; j < SPT; ++j) v[j] = 0.0f;
      if (CT) {
        // C channels known at compile time: all C x SPT loads of the leaf are independent
        const ST* src[CT > 0 ? CT : 1];
#pragma unroll
        for (int ci = 0; ci < CT; ++ci)
          src[ci] = win + static_cast<size_t>(cl0 + ci) * a.win + drel[wd * GC + cl0 + ci] + lane;
        float x[CT > 0 ? CT : 1][SPT];
#pragma unroll
        for (int ci = 0; ci < CT; ++ci)
#pragma unroll
          for (int j = 0; j < SPT; ++j) x[ci][j] = zload(src[ci] + 32 * j);
#pragma unroll
        for (int ci = 0; ci < CT; ++ci)
#pragma unroll
          for (int j = 0; j < SPT; ++j) v[j] = __fadd_rn(v[j], x[ci][j]);
      } else {
        for (int ci = 0; ci < cn; ++ci) {
          const ST* src = win + static_cast<size_t>(cl0 + ci) * a.win + drel[wd * GC + cl0 + ci] + lane;
#pragma unroll
          for (int j = 0; j < SPT; ++j) v[j] = __fadd_rn(v[j], zload(src + 32 * j));
        }
      }
      if (a.nlev == 1) {  // a single leaf is the root: its FP32 sum is not stored
#pragma unroll
        for (int j = 0; j < SPT; ++j) root[j] = v[j];
        continue;
      }
      // the stored leaf goes into its parent's sum (acc[l] holds the open node of level l + 1);
      // when it is the parent's last child the parent is finished, and so on up `depth`
      // levels. depth depends on the leaf only, so the branch is warp-uniform and taken by one
      // leaf in B.
#pragma unroll
      for (int j = 0; j < SPT; ++j) acc[0][j] = __fadd_rn(acc[0][j], zstore_round(v[j], ring));
      const int depth = __ldg(a.carry + k);
      if (depth > 0) {
#pragma unroll
        for (int l = 0; l + 1 < MAXL; ++l) {
          if (l < depth) {
            const bool to_root = (l + 1 == a.nlev - 1);
#pragma unroll
            for (int j = 0; j < SPT; ++j) {
              const float x = acc[l][j];
              acc[l][j] = 0.0f;
              if (to_root) {
                root[j] = x;
              } else {
                acc[l + 1][j] = __fadd_rn(acc[l + 1][j], zstore_round(x, ring));
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
  for (int j = 0; j < SPT; ++j) {
    const long long t = tb + 32 * j + lane;
    if (t - a.t0 >= a.nout) continue;
    const long long col = a.omode ? (t - a.t0) : (t % a.Lp);
    orow[col] = __fmul_rn(root[j], a.scale);
  }
}

template <typename ST, int MAXL, int SPT>
cudaError_t run_z(const ZArgs& a, dim3 grid, dim3 block, int smem, cudaStream_t s) {
  // the compile-time 4-channel leaf applies when every leaf has 4 channels
  auto kern = (a.C == 4 && a.nchan % 4 == 0) ? k_tree_z<ST, MAXL, SPT, 4> : k_tree_z<ST, MAXL, SPT, 0>;
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
    if (z.maxl == 4) return run_z<__half, 4, 8>(a, grid, block, z.smem_bytes, s);
    if (z.maxl == 8) return run_z<__half, 8, 4>(a, grid, block, z.smem_bytes, s);
    return run_z<__half, 16, 2>(a, grid, block, z.smem_bytes, s);
  }
  if (z.maxl == 4) return run_z<float, 4, 8>(a, grid, block, z.smem_bytes, s);
  if (z.maxl == 8) return run_z<float, 8, 4>(a, grid, block, z.smem_bytes, s);
  return run_z<float, 16, 2>(a, grid, block, z.smem_bytes, s);
}

}  // namespace snd
