// Learned candidate sifter (the paper's "Discussion" leaves a learned classifier to future
// work): DM-time snippets around candidates, classified by a small CNN that is trained and
// run on the GPU with BF16 tensor-core GEMMs.
//
// Network (input 1 x 64 x 256): three 3x3 convolutions (16, 32, 64 channels, zero padding
// 1, bias, ReLU), each followed by 2x2 max pooling; fc1 16384 -> 128 (ReLU); fc2 128 -> 1.
// Loss: mean binary cross-entropy on the logit. Parameters are one flat FP32 vector:
// W1[16][1][3][3], b1, W2[32][16][3][3], b2, W3[64][32][3][3], b3, Wf1[128][16384], bf1,
// Wf2[128], bf2. Adam keeps FP32 moments; the GEMMs read BF16 copies of the weights.
//
// conv2 and conv3 run with their pooling as k_conv_halo (TMA-loaded input rows, each tap a
// descriptor view into them; in training the epilogue also keeps the argmax of every pooled
// cell); their input gradients run on the same kernel (the convolution of dY with the flipped
// kernel, BF16 channels-last output);
// fc1 and every backward GEMM are C = A B^T with both operands K-major BF16 (k_gemm): TMA
// (128-byte swizzle) fills a 4-stage shared-memory ring, one thread issues tcgen05.mma
// (M = 128, N = BN, K = 16 per instruction) into a TMEM accumulator, and four warps read it
// back with tcgen05.ld for the epilogue (bias, ReLU, BF16 or FP32, row-major or transposed
// store, or FP32 atomic add for split-K). conv1 (one input channel) runs as k_conv1_tc.
// The pooled maps that feed conv2 and conv3 and the output gradients dY that feed the input
// gradients are channels-last ([b][h][w][c]); gradients routed through the pooling are also
// kept channel-major (dY^T[c][m], m = (b, h, w)) for the weight gradients, which read the
// patches of conv2's and conv3's inputs as 9 TMA boxes a K step from three horizontally
// shifted channel-major copies of the input (k_shift3); conv1's is a direct reduction.
//   forward conv:   pool(relu(x (x) W + b))                               (k_conv_halo)
//   weight grad:    dW[cout][k] += dY^T[cout][m] . patch[m][k]           (k_gemm, 9 tap boxes, split-K)
//   input grad:     dX^T[cin][m] = dY (x) flipped W                        (k_conv_halo, DX)
// Every mbarrier wait is bounded (about 2 s of clock); a wait that gives up sets a device
// error word that the host turns into SND_ERR_TIMEOUT, and the kernel still frees its TMEM.

#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/snd.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int kBM = 128, kBK = 64, kStages = 4;
constexpr int kH = 64, kW = 256, kFeat = 64 * 8 * 32, kHid = 128;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

struct ConvL {
  int cin, cout, h, w, kc, kp;
};
constexpr ConvL kConv[3] = {{1, 16, 64, 256, 9, 64}, {16, 32, 32, 128, 144, 192}, {32, 64, 16, 64, 288, 320}};

// flat parameter offsets
constexpr long long kOffW[3] = {0, 16 * 9 + 16, 16 * 9 + 16 + 32 * 144 + 32};
constexpr long long kOffB[3] = {16 * 9, 16 * 9 + 16 + 32 * 144, 16 * 9 + 16 + 32 * 144 + 32 + 64 * 288};
constexpr long long kOffWf1 = 16 * 9 + 16 + 32 * 144 + 32 + 64 * 288 + 64;
constexpr long long kOffBf1 = kOffWf1 + static_cast<long long>(kHid) * kFeat;
constexpr long long kOffWf2 = kOffBf1 + kHid;
constexpr long long kOffBf2 = kOffWf2 + kHid;
constexpr long long kNumParams = kOffBf2 + 1;

enum : uint32_t { kErrWait = 1u };

// ---------------------------------------------------------------- tcgen05 GEMM

struct Epi {
  const float* bias;  // [N] or null
  int relu;
  void* out;
  int out_bf16;       // BF16 store (else FP32)
  int transposed;     // out[n * ldo + m] (else out[m * ldo + n])
  int atomic;         // FP32 atomic add (split-K)
  long long ldo;
};

// Weight-gradient mode of k_gemm: K runs over the pixels m = (b, y, x) of an h x w map. The B
// tile of N-tile j is one TMA box of S[kx][ci][b][y'][x] = map[b][y'][x + kx - 1][ci] (zero
// outside): 64 pixels x rows y - 1 .. y + 1 x channels 16 j .. 16 j + 15 x kx = 0..2, i.e. 144
// rows r = kx * 48 + ci * 3 + ky, weight column (16 j + ci) * 9 + 3 ky + kx. The A box holds
// the arows output-channel rows of dY^T only (the MMA's other rows read stale shared memory
// and their accumulators are never stored).
struct Wg {
  int h, w, arows;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait on an mbarrier phase
__device__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d_rows(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                                 int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1, int c2,
                                            int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1) << 16;            // leading byte offset (unused for swizzled K-major)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;    // stride byte offset: next 8-row group
  d |= static_cast<uint64_t>(1) << 46;            // descriptor version
  d |= static_cast<uint64_t>(2) << 61;            // 128-byte swizzle
  return d;
}

// instruction descriptor of kind::f16: FP32 accumulate, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t mma_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(kBM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive TMEM columns of this warp's 32 lanes (one wait)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// BF16 of relu(v + bias), two values packed
__device__ __forceinline__ uint32_t act_pack2(float v0, float b0, float v1, float b1) {
  const __nv_bfloat162 pr = __floats2bfloat162_rn(fmaxf(v0 + b0, 0.0f), fmaxf(v1 + b1, 0.0f));
  return *reinterpret_cast<const uint32_t*>(&pr);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Persistent, warp-specialised GEMM. 192 threads: warps 0-3 drain the accumulator (warp w
// owns TMEM lanes 32w..32w+31, i.e. tile rows), warp 4 issues the TMA loads, warp 5 owns
// the TMEM allocation and one of its threads issues the MMAs. A CTA walks the output tiles
// t = blockIdx.x, + gridDim.x, ... (blockIdx.z = K split); the accumulator is double
// buffered in TMEM (2 x BN columns), so the epilogue of tile j overlaps the MMAs of tile
// j + 1, and the shared-memory stage ring runs across tiles.
template <int BN, bool WG = false>
__global__ void __launch_bounds__(192, 1)
    k_gemm(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap mb, int M, int N, int ktiles,
           int kt_per_split, Epi epi, uint32_t* err, Wg wg) {
  constexpr uint32_t kABytes = kBM * kBK * 2, kBBytes = BN * kBK * 2;
  // TMEM: two accumulator buffers of BN columns, allocated as a power of two (at least 32)
  constexpr uint32_t kCols = 2 * BN <= 32 ? 32 : (2 * BN <= 64 ? 64 : (2 * BN <= 128 ? 128 : (2 * BN <= 256 ? 256 : 512)));
  static_assert(!WG || BN == 144, "weight-gradient tile: 9 taps x 16 channels");
  extern __shared__ uint8_t gsm_raw[];
  __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages], bar_tfull[2], bar_tempty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  uint8_t* gsm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sA = smem_u32(gsm), sB = sA + kStages * kABytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = (M + kBM - 1) / kBM, nt = (N + BN - 1) / BN;
  const int ntiles = mt * nt;
  const int kt0 = blockIdx.z * kt_per_split;
  const int nkt = min(ktiles, kt0 + kt_per_split) - kt0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bar_tfull[b]), 1);
      mbar_init(smem_u32(&bar_tempty[b]), 4);  // one arrival per epilogue warp
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* abort_v = &abort_flag;

  if (nkt > 0) {
    if (warp == 4) {
      if (lane == 0) {
        // producer: the K steps of every tile of this CTA through the stage ring
        int it = 0;
        for (int t = blockIdx.x; t < ntiles && !*abort_v; t += gridDim.x) {
          const int m0 = (t % mt) * kBM, n0 = (t / mt) * BN;
          for (int i = 0; i < nkt; ++i, ++it) {
            const int s = it % kStages;
            if (it >= kStages && !mbar_wait(smem_u32(&bar_empty[s]), ((it / kStages) & 1) ^ 1)) {
              atomicOr(err, kErrWait);
              *abort_v = 1;
              break;
            }
            const uint32_t fb = smem_u32(&bar_full[s]);
            if constexpr (WG) {
              // K step = 64 pixels of one image row (64 divides w)
              mbar_expect_tx(fb, static_cast<uint32_t>(wg.arows) * kBK * 2 + kBBytes);
              tma_load_2d(sA + s * kABytes, &ma, fb, (kt0 + i) * kBK, m0);
              const int px = (kt0 + i) * kBK;
              const int x0 = px % wg.w, r = px / wg.w;
              const int y = r % wg.h, b = r / wg.h;
              tma_load_5d(sB + s * kBBytes, &mb, fb, x0, y - 1, b, (n0 / BN) * 16, 0);
            } else {
              mbar_expect_tx(fb, kABytes + kBBytes);
              tma_load_2d(sA + s * kABytes, &ma, fb, (kt0 + i) * kBK, m0);
              tma_load_2d(sB + s * kBBytes, &mb, fb, (kt0 + i) * kBK, n0);
            }
          }
        }
      }
    } else if (warp == 5) {
      if (lane == 0) {
        // MMA issuer: tile j accumulates into TMEM buffer j & 1 once the epilogue freed it
        constexpr uint32_t idesc = mma_idesc(BN);
        int it = 0, j = 0;
        for (int t = blockIdx.x; t < ntiles && !*abort_v; t += gridDim.x, ++j) {
          const int b = j & 1;
          if (j >= 2 && !mbar_wait(smem_u32(&bar_tempty[b]), ((j >> 1) & 1) ^ 1)) {
            atomicOr(err, kErrWait);
            *abort_v = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t acc = tmem + static_cast<uint32_t>(b * BN);
          for (int i = 0; i < nkt; ++i, ++it) {
            const int s = it % kStages;
            if (!mbar_wait(smem_u32(&bar_full[s]), (it / kStages) & 1)) {
              atomicOr(err, kErrWait);
              *abort_v = 1;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
              const uint64_t da = sw128_desc(sA + s * kABytes + kk * 32);
              const uint64_t db = sw128_desc(sB + s * kBBytes + kk * 32);
              umma_bf16(acc, da, db, idesc, (i | kk) != 0 ? 1u : 0u);
            }
            umma_commit(smem_u32(&bar_empty[s]));
          }
          umma_commit(smem_u32(&bar_tfull[b]));
        }
      }
    } else {
      // epilogue warps 0-3
      int j = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
        const int b = j & 1;
        bool ok = !*abort_v && mbar_wait(smem_u32(&bar_tfull[b]), (j >> 1) & 1);
        ok = __all_sync(0xFFFFFFFFu, ok);
        if (!ok) {
          if (lane == 0) atomicOr(err, kErrWait);
          *abort_v = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int m0 = (t % mt) * kBM, n0 = (t / mt) * BN;
        const int row = m0 + warp * 32 + lane;
        const uint32_t tbase = tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(b * BN);
#pragma unroll 1
        for (int c = 0; c < BN; c += 8) {
          float v[8];
          tmem_ld8(tbase + static_cast<uint32_t>(c), v);
          if (row >= M) continue;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int n = n0 + c + q;
            if (n >= N) continue;
            float x = v[q];
            if (epi.bias) x += epi.bias[n];
            if (epi.relu) x = fmaxf(x, 0.0f);
            long long idx = epi.transposed ? static_cast<long long>(n) * epi.ldo + row
                                           : static_cast<long long>(row) * epi.ldo + n;
            if constexpr (WG) {
              const int r = c + q, kx = r / 48, ci = (n0 / BN) * 16 + (r % 48) / 3, ky = r % 3;
              idx = static_cast<long long>(row) * epi.ldo + ci * 9 + 3 * ky + kx;
            }
            if (epi.atomic) {
              atomicAdd(static_cast<float*>(epi.out) + idx, x);
            } else if (epi.out_bf16) {
              static_cast<bf16*>(epi.out)[idx] = __float2bfloat16_rn(x);
            } else {
              static_cast<float*>(epi.out)[idx] = x;
            }
          }
        }
        // the buffer may take the tile after next
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_tempty[b]));
      }
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 5) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
  }
}

// Arguments of k_conv_halo (the input map itself comes as a TMA tensor map)
struct ConvArgs {
  int n, h;          // snippets, image rows (the kernel's W is a template argument)
  const float* bias;  // [cout]; unused in DX mode
  // the 2x2 max pooling of the activations. pool_cl: pooled map channels-last
  // p[(b, y2, x2)][cout]; else p[b][(c, y2, x2)] (fc1's input rows)
  bf16* p;
  int pool_cl;
  // training: the argmax 0..3 of every pooled cell (first maximum of the four BF16 activations
  // in row-major order), 2 bits a channel: am[(c / 16) * npix + pooled pixel] bits 2 (c % 16);
  // null in inference
  uint32_t* am;
  // DX: the convolution itself, channels-last BF16 [(b, y, x)][cout] (no bias, ReLU or pooling)
  bf16* dx;
};

// The 2x2 max pooling of 16 channels with its argmax, for training (the backward pass routes
// the gradient to the argmax). Lane pairs (x even, x odd) hold one pooled cell; v0 / v1 are the
// FP32 sums of the lane's pixel in the upper / lower row. Each activation is bias, ReLU and
// BF16 rounding of its sum; the cell takes the first maximum in row-major order (upper left,
// upper right, lower left, lower right), as the oracle's pooling does. Even lanes get the packed pooled
// values in pk and write the 16 argmaxes, 2 bits each (channel c0 + q at bits 2q, 2q + 1), as one
// word am[(c0 / 16) * npix + pix].
__device__ __forceinline__ void pool_argmax16(const float* v0, const float* v1, const float* bias, int lane,
                                              uint32_t* pk, uint32_t* am, int c0, long long npix, long long pix) {
  uint32_t code = 0;
#pragma unroll
  for (int q = 0; q < 16; q += 2) {
    float best[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float u = __bfloat162float(__float2bfloat16_rn(fmaxf(v0[q + e] + bias[q + e], 0.0f)));
      const float l = __bfloat162float(__float2bfloat16_rn(fmaxf(v1[q + e] + bias[q + e], 0.0f)));
      const float ur = __shfl_xor_sync(0xFFFFFFFFu, u, 1), lr = __shfl_xor_sync(0xFFFFFFFFu, l, 1);
      int a = 0;
      float bv = u;
      if (ur > bv) { bv = ur; a = 1; }
      if (l > bv) { bv = l; a = 2; }
      if (lr > bv) { bv = lr; a = 3; }
      best[e] = bv;
      code |= static_cast<uint32_t>(a) << (2 * (q + e));
    }
    const __nv_bfloat162 pr = __floats2bfloat162_rn(best[0], best[1]);
    pk[q >> 1] = *reinterpret_cast<const uint32_t*>(&pr);
  }
  if (!(lane & 1)) am[static_cast<long long>(c0 >> 4) * npix + pix] = code;
}

// ---------------------------------------------------------------- halo convolution

// shared-memory matrix descriptor, K-major without swizzle: core matrices of 8 rows x 16 bytes
// (rows 16 bytes apart), lbo bytes between core matrices along K, sbo along M / N
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;  // descriptor version; layout type 0: no swizzle
  return d;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1, int c2,
                                            int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// Shared-memory stages of k_conv_halo: three when they and the weights fit in half an SM's
// shared memory (two CTAs a SM), else two.
__host__ __device__ constexpr int halo_stages(int cin, int cout, int w) {
  return 3 * (cin / 8) * 4 * (w + 2) * 16 + 9 * (cin / 8) * cout * 16 + 128 <= 113 * 1024 ? 3 : 2;
}

// Forward 3x3 convolution with its 2x2 max pooling (inference), without any gather. A work
// item is one pair of image rows (y0, y0 + 1) of one snippet; the TMA engine loads the four
// input rows y0 - 1 .. y0 + 2 of the channels-last map once, W + 2 pixels wide (-1 .. W, zero
// outside the map), as 8-channel planes (16 bytes a pixel). An M tile is one image row (two
// tiles per item, accumulated side by side in TMEM), and the A operand of tap (ky, kx) is a
// plain K-major view 128 pixels long starting ky rows down and kx pixels in: 8 channels per
// core matrix, the next 8 one plane further. For W = 64 the tile's last 64 rows run into the
// next row (and for the last tap past the stage) and are not used. The weights sit in shared
// memory as [tap][plane][cout][8]. 320 threads: two epilogue warpgroups (warps 0-3 and 4-7),
// each draining one of the two TMEM accumulator buffers (items alternate between them), warp 8
// issues the TMA loads and warp 9 owns TMEM and issues the MMAs; two or three shared-memory
// stages. DX: the input gradient of a convolution, i.e. the same convolution of the output
// gradient dY (channels-last) with the flipped, channel-transposed kernel; the epilogue writes
// the sums rounded to BF16, channels-last [(b, y, x)][c].
template <int CIN, int COUT, int W, bool TRAIN, bool DX = false>
__global__ void __launch_bounds__(320, 2)
    k_conv_halo(const __grid_constant__ CUtensorMap mx, ConvArgs a, const bf16* __restrict__ wb, int kp,
                uint32_t* err) {
  constexpr int NPL = CIN / 8;                 // 8-channel planes
  constexpr int T = 2;                         // M tiles (image rows) per item
  constexpr int PITCH = W + 2;                 // pixels per loaded row
  constexpr int PB = 4 * PITCH * 16;           // bytes of one plane (4 rows)
  constexpr int SB = NPL * PB;                 // bytes of one stage
  constexpr int KS = NPL / 2;                  // K steps of 16 per tap
  constexpr int S = halo_stages(CIN, COUT, W);  // stages
  constexpr uint32_t kCols = 2 * T * COUT < 32 ? 32 : 2 * T * COUT;
  static_assert(W == 128 || W == 64, "tile geometry");
  extern __shared__ uint8_t hsm_raw[];
  __shared__ __align__(8) uint64_t bar_full[S], bar_empty[S], bar_tfull[2], bar_tempty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ float bsm[COUT];
  uint8_t* hsm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(hsm_raw) + 127) & ~uintptr_t(127));
  const uint32_t sX = smem_u32(hsm), sW = sX + S * SB;
  bf16* wsm = reinterpret_cast<bf16*>(hsm + S * SB);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = a.n * (a.h >> 1);

  // weights: wb[co][tap * CIN + ci] (tap-major K) -> wsm[((tap * NPL + ci / 8) * COUT + co) * 8 + ci % 8]
  for (int i = threadIdx.x; i < COUT * 9 * CIN; i += blockDim.x) {
    const int co = i / (9 * CIN), k = i - co * (9 * CIN);
    const int tap = k / CIN, ci = k - tap * CIN;
    wsm[((tap * NPL + ci / 8) * COUT + co) * 8 + (ci & 7)] = wb[static_cast<long long>(co) * kp + k];
  }
  if (threadIdx.x < COUT) bsm[threadIdx.x] = DX ? 0.0f : a.bias[threadIdx.x];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the tensor core reads them
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bar_tfull[b]), 1);
      mbar_init(smem_u32(&bar_tempty[b]), 4);  // one arrival per warp of the buffer's warpgroup
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 9) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* abort_v = &abort_flag;

  if (warp == 8) {
    if (lane == 0) {
      int j = 0;
      for (int it = blockIdx.x; it < items && !*abort_v; it += gridDim.x, ++j) {
        const int s = j % S;
        if (j >= S && !mbar_wait(smem_u32(&bar_empty[s]), ((j / S) & 1) ^ 1)) {
          atomicOr(err, kErrWait);
          *abort_v = 1;
          break;
        }
        const int b = it / (a.h >> 1), y0 = 2 * (it - b * (a.h >> 1));
        const uint32_t fb = smem_u32(&bar_full[s]);
        mbar_expect_tx(fb, SB);
#pragma unroll
        for (int pc = 0; pc < NPL; ++pc) tma_load_4d(sX + s * SB + pc * PB, &mx, fb, 8 * pc, -1, y0 - 1, b);
      }
    }
  } else if (warp == 9) {
    if (lane == 0) {
      constexpr uint32_t idesc = mma_idesc(COUT);
      int j = 0;
      for (int it = blockIdx.x; it < items && !*abort_v; it += gridDim.x, ++j) {
        const int s = j % S, bb = j & 1;
        if (j >= 2 && !mbar_wait(smem_u32(&bar_tempty[bb]), ((j >> 1) & 1) ^ 1)) {
          atomicOr(err, kErrWait);
          *abort_v = 1;
          break;
        }
        if (!mbar_wait(smem_u32(&bar_full[s]), (j / S) & 1)) {
          atomicOr(err, kErrWait);
          *abort_v = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int tau = 0; tau < T; ++tau) {
          const uint32_t acc = tmem + static_cast<uint32_t>((bb * T + tau) * COUT);
#pragma unroll
          for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3;
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
              const uint32_t aaddr = sX + s * SB + (2 * ks) * PB + ((tau + ky) * PITCH + kx) * 16;
              const uint32_t baddr = sW + ((tap * NPL + 2 * ks) * COUT) * 16;
              umma_bf16(acc, kmajor_desc(aaddr, PB, 128), kmajor_desc(baddr, COUT * 16, 128), idesc,
                        (tap | ks) != 0 ? 1u : 0u);
            }
          }
        }
        umma_commit(smem_u32(&bar_empty[s]));
        umma_commit(smem_u32(&bar_tfull[bb]));
      }
    }
  } else {
    // epilogue warpgroup grp (warps 4 grp ..): the items j with j & 1 == grp, from TMEM buffer
    // grp; warp wq of the group reads TMEM lanes 32 wq ..
    const int grp = warp >> 2, wq = warp & 3;
    int j = grp;
    const int h2 = a.h >> 1, w2 = W >> 1;
    for (int it = blockIdx.x + grp * gridDim.x; it < items; it += 2 * gridDim.x, j += 2) {
      const int bb = grp;
      bool ok = !*abort_v && mbar_wait(smem_u32(&bar_tfull[bb]), (j >> 1) & 1);
      ok = __all_sync(0xFFFFFFFFu, ok);
      if (!ok) {
        if (lane == 0) atomicOr(err, kErrWait);
        *abort_v = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t lanes = static_cast<uint32_t>(wq * 32) << 16;
      if (DX && 32 * wq < W) {
        // the two rows' sums rounded to BF16, channels-last (a lane's 16 channels are 32
        // contiguous bytes, the lanes consecutive pixels)
        const int b = it / h2, y0 = 2 * (it - b * h2);
        const long long m0 = (static_cast<long long>(b) * a.h + y0) * W + 32 * wq + lane;
#pragma unroll 1
        for (int c = 0; c < COUT; c += 16) {
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            float v[16];
            tmem_ld16(tmem + lanes + static_cast<uint32_t>((bb * T + r) * COUT + c), v);
            uint32_t pk[8];
#pragma unroll
            for (int q = 0; q < 16; q += 2) {
              const __nv_bfloat162 pr = __floats2bfloat162_rn(v[q], v[q + 1]);
              pk[q >> 1] = *reinterpret_cast<const uint32_t*>(&pr);
            }
            uint4* dst = reinterpret_cast<uint4*>(a.dx + (m0 + r * W) * COUT + c);
            dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
          }
        }
      } else if (!DX && 32 * wq < W) {
        // pixel x = 32 wq + lane of rows y0 (tile 0) and y0 + 1 (tile 1). Bias, ReLU and the
        // BF16 rounding are monotone non-decreasing, so the maximum of the four rounded
        // activations is the rounded activation of the largest of the four sums: the pooling
        // runs on the FP32 accumulators and one value per pooled cell is rounded.
        const int b = it / h2, yp = it - b * h2;
        const int x2 = (32 * wq + lane) >> 1;
#pragma unroll 1
        for (int c = 0; c < COUT; c += 16) {
          float v0[16], v1[16];
          tmem_ld16(tmem + lanes + static_cast<uint32_t>((bb * T) * COUT + c), v0);
          tmem_ld16(tmem + lanes + static_cast<uint32_t>((bb * T + 1) * COUT + c), v1);
          uint32_t pk[8];
          if constexpr (TRAIN) {
            // training: the four rounded activations and their argmax (first maximum)
            pool_argmax16(v0, v1, bsm + c, lane, pk, a.am, c, static_cast<long long>(a.n) * h2 * w2,
                          (static_cast<long long>(b) * h2 + yp) * w2 + x2);
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const float m = fmaxf(v0[q], v1[q]);
              v0[q] = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, 1));
            }
          }
          if (!(lane & 1)) {
            if constexpr (!TRAIN) {
#pragma unroll
              for (int q = 0; q < 16; q += 2) pk[q >> 1] = act_pack2(v0[q], bsm[c + q], v0[q + 1], bsm[c + q + 1]);
            }
            if (a.pool_cl) {  // channels-last [(b, y2, x2)][COUT]
              uint4* dst = reinterpret_cast<uint4*>(a.p + ((static_cast<long long>(b) * h2 + yp) * w2 + x2) * COUT + c);
              dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
              dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            } else {  // fc1's rows [b][(c, y2, x2)]
              bf16* dst = a.p + static_cast<long long>(b) * COUT * h2 * w2 + static_cast<long long>(yp) * w2 + x2;
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                const bf16 v = __ushort_as_bfloat16(
                    static_cast<unsigned short>((q & 1) ? (pk[q >> 1] >> 16) : (pk[q >> 1] & 0xFFFFu)));
                dst[static_cast<long long>(c + q) * h2 * w2] = v;

              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_tempty[bb]));
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 9) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
  }
}

// conv1 (one input channel) on the tensor cores. A work item is one pair of image rows
// (y0, y0 + 1) of one half (128 pixels) of one snippet row; its two M tiles are the two rows.
// The TMA engine loads the four input rows y0 - 1 .. y0 + 2 (FP32, 136 values from x0 - 4,
// zero outside the snippet) into a deep ring of small raw stages; four builder warps turn
// them into U: for every pixel its three horizontal taps (x - 1, x, x + 1) as BF16 and five
// zeros, 16 bytes. The A operand of a row tile is then a K-major view into U whose K core
// matrices are the U rows of the vertical taps, one U row apart (a fourth, of zero weight,
// reads the next row or a zero row): two MMAs of K = 16 per tile, weights [ky][cout][8] with
// zeros past kx = 2 and ky = 2.
// The epilogue writes the 2x2 max pooling of the activations, channels-last [(b, y2, x2)][16];
// TRAIN: also the argmax of every pooled cell (am). 320 threads: warps 0-3 epilogue,
// warps 4-7 build U, warp 8 owns TMEM and issues the MMAs, warp 9 issues the TMA loads.
// Rounding: BF16 snippet values and weights, FP32 sums (the tensor core adds the nine
// products in its own order), bias, ReLU, BF16 store.
template <bool TRAIN>
__global__ void __launch_bounds__(320, 1)
    k_conv1_tc(const __grid_constant__ CUtensorMap mx, int n, const float* __restrict__ w, const float* __restrict__ bias,
               bf16* __restrict__ out, uint32_t* __restrict__ am, uint32_t* err) {
  constexpr int RS = 12, US = 4;               // raw and U stages
  constexpr int RAWW = 136;                    // FP32 values per loaded row (x0 - 4 .. x0 + 131)
  constexpr int RB = 4 * RAWW * 4;             // raw bytes per stage
  constexpr int UB = 5 * 128 * 16;             // U bytes per stage (row 4 stays zero)
  constexpr uint32_t kCols = 64;               // 2 buffers x 2 tiles x 16 channels
  extern __shared__ uint8_t csm_raw[];
  __shared__ __align__(8) uint64_t bar_raw[RS], bar_rawfree[RS], bar_u[US], bar_uempty[US], bar_tfull[2],
      bar_tempty[2];
  __shared__ __align__(16) bf16 wsm[4 * 16 * 8];
  __shared__ float bsm[16];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  uint8_t* csm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(csm_raw) + 127) & ~uintptr_t(127));
  const uint32_t sU = smem_u32(csm), sR = sU + US * UB;
  const float* raw = reinterpret_cast<const float*>(csm + US * UB);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = n * 32 * 2;

  // weights [ky][c][j]: bf16(w[c][3 ky + j]) for j, ky < 3, else 0; U's zero row 4 of every stage
  for (int i = threadIdx.x; i < 4 * 16 * 8; i += blockDim.x) {
    const int ky = i / 128, c = (i / 8) % 16, jx = i % 8;
    wsm[i] = __float2bfloat16_rn((ky < 3 && jx < 3) ? w[c * 9 + ky * 3 + jx] : 0.0f);
  }
  if (threadIdx.x < 16) bsm[threadIdx.x] = bias[threadIdx.x];
  for (int i = threadIdx.x; i < US * 128; i += blockDim.x)
    *reinterpret_cast<uint4*>(csm + (i / 128) * UB + (4 * 128 + i % 128) * 16) = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    for (int s = 0; s < RS; ++s) {
      mbar_init(smem_u32(&bar_raw[s]), 1);
      mbar_init(smem_u32(&bar_rawfree[s]), 4);  // one arrival per builder warp
    }
    for (int s = 0; s < US; ++s) {
      mbar_init(smem_u32(&bar_u[s]), 4);
      mbar_init(smem_u32(&bar_uempty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bar_tfull[b]), 1);
      mbar_init(smem_u32(&bar_tempty[b]), 4);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* abort_v = &abort_flag;

  if (warp == 9) {
    if (lane == 0) {
      int j = 0;
      for (int it = blockIdx.x; it < items && !*abort_v; it += gridDim.x, ++j) {
        const int r = j % RS;
        if (j >= RS && !mbar_wait(smem_u32(&bar_rawfree[r]), ((j / RS) & 1) ^ 1)) {
          atomicOr(err, kErrWait);
          *abort_v = 1;
          break;
        }
        const int b = it >> 6, yp = (it >> 1) & 31, hx = it & 1;
        const uint32_t rb = smem_u32(&bar_raw[r]);
        mbar_expect_tx(rb, RB);
        tma_load_2d_rows(sR + r * RB, &mx, rb, hx * 128 - 4, 2 * yp - 1, b);
      }
    }
  } else if (warp >= 4 && warp < 8) {
    const int pr = threadIdx.x - 128;  // pixel of the half row
    int j = 0;
    for (int it = blockIdx.x; it < items && !*abort_v; it += gridDim.x, ++j) {
      const int r = j % RS, u = j % US;
      bool ok = mbar_wait(smem_u32(&bar_raw[r]), (j / RS) & 1);
      if (ok && j >= US) ok = mbar_wait(smem_u32(&bar_uempty[u]), ((j / US) & 1) ^ 1);
      if (!ok) {
        atomicOr(err, kErrWait);
        *abort_v = 1;
        break;
      }
      const float* rs = raw + r * (RB / 4);
      uint8_t* us = csm + u * UB;
#pragma unroll
      for (int row = 0; row < 4; ++row) {
        // raw value of pixel pr + d is rs[row * RAWW + 4 + pr + d]
        const float* rr = rs + row * RAWW + 4 + pr;
        const __nv_bfloat162 p01 = __floats2bfloat162_rn(rr[-1], rr[0]);
        const __nv_bfloat162 p2 = __floats2bfloat162_rn(rr[1], 0.0f);
        *reinterpret_cast<uint4*>(us + (row * 128 + pr) * 16) =
            make_uint4(*reinterpret_cast<const uint32_t*>(&p01), *reinterpret_cast<const uint32_t*>(&p2), 0u, 0u);
      }
      // the raw stage is read (and may be refilled by the TMA engine) and U is written (for
      // the tensor core): proxy fence, then one arrival per warp on each
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(&bar_rawfree[r]));
        mbar_arrive(smem_u32(&bar_u[u]));
      }
    }
  } else if (warp == 8) {
    if (lane == 0) {
      constexpr uint32_t idesc = mma_idesc(16);
      int j = 0;
      for (int it = blockIdx.x; it < items && !*abort_v; it += gridDim.x, ++j) {
        const int u = j % US, bb = j & 1;
        if (j >= 2 && !mbar_wait(smem_u32(&bar_tempty[bb]), ((j >> 1) & 1) ^ 1)) {
          atomicOr(err, kErrWait);
          *abort_v = 1;
          break;
        }
        if (!mbar_wait(smem_u32(&bar_u[u]), (j / US) & 1)) {
          atomicOr(err, kErrWait);
          *abort_v = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int tau = 0; tau < 2; ++tau) {
          const uint32_t acc = tmem + static_cast<uint32_t>((bb * 2 + tau) * 16);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            // K core matrices: U rows tau + 2h, tau + 2h + 1 (vertical taps 2h, 2h + 1)
            const uint32_t aaddr = sU + u * UB + ((tau + 2 * h) * 128) * 16;
            const uint32_t baddr = smem_u32(wsm) + (2 * h) * 16 * 16;
            umma_bf16(acc, kmajor_desc(aaddr, 128 * 16, 128), kmajor_desc(baddr, 16 * 16, 128), idesc, h ? 1u : 0u);
          }
        }
        umma_commit(smem_u32(&bar_uempty[u]));
        umma_commit(smem_u32(&bar_tfull[bb]));
      }
    }
  } else {
    // epilogue warps 0-3 (TMEM lanes 32 warp ..: pixel 32 warp + lane of the half row)
    int j = 0;
    for (int it = blockIdx.x; it < items; it += gridDim.x, ++j) {
      const int bb = j & 1;
      bool ok = !*abort_v && mbar_wait(smem_u32(&bar_tfull[bb]), (j >> 1) & 1);
      ok = __all_sync(0xFFFFFFFFu, ok);
      if (!ok) {
        if (lane == 0) atomicOr(err, kErrWait);
        *abort_v = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t lanes = static_cast<uint32_t>(warp * 32) << 16;
      const int b = it >> 6, yp = (it >> 1) & 31, hx = it & 1;
      const int xg = hx * 128 + warp * 32 + lane;
      float v0[16], v1[16];
      tmem_ld16(tmem + lanes + static_cast<uint32_t>((bb * 2) * 16), v0);
      tmem_ld16(tmem + lanes + static_cast<uint32_t>((bb * 2 + 1) * 16), v1);
      {
        uint32_t pk[8];
        if constexpr (TRAIN) {
          // training: the four rounded activations and their argmax (first maximum)
          pool_argmax16(v0, v1, bsm, lane, pk, am, 0, static_cast<long long>(n) * 32 * 128,
                        (static_cast<long long>(b) * 32 + yp) * 128 + (xg >> 1));
        } else {
          // the maximum of the four rounded activations is the rounded activation of the
          // largest of the four sums (bias, ReLU and BF16 rounding are monotone non-decreasing)
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float m = fmaxf(v0[q], v1[q]);
            v0[q] = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, 1));
          }
        }
        if (!(lane & 1)) {
          if constexpr (!TRAIN) {
#pragma unroll
            for (int q = 0; q < 16; q += 2) pk[q >> 1] = act_pack2(v0[q], bsm[q], v0[q + 1], bsm[q + 1]);
          }
          uint4* dst = reinterpret_cast<uint4*>(out + ((static_cast<long long>(b) * 32 + yp) * 128 + (xg >> 1)) * 16);
          dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_tempty[bb]));
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 8) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
  }
}

// ---------------------------------------------------------------- layer kernels

// conv1's weight gradient dW[co][tap] += sum over pixels m of dY^T[co][m] * x[m + tap offset]
// (the snippet values rounded to BF16, as the forward convolution reads them; zero outside the
// snippet). 16 x 9 outputs, so the CUDA cores reduce it directly: a CTA takes one snippet and 4
// output channels (blockIdx.y) and stages the snippet in shared memory; a warp takes one image
// row at a time (rows warp, warp + 8, ...), a lane 8 consecutive pixels, whose gradients come
// as one 16-byte load per channel. A thread keeps its 36 partial sums in registers; the CTA's
// sums are added atomically.
__global__ void __launch_bounds__(256) k_dw1(const float* __restrict__ x, int n, const bf16* __restrict__ dyT,
                                             float* __restrict__ dw) {
  constexpr int XP = kW + 16;  // staged row (BF16): pixel xx at xx + 8, zero at 7 and kW + 8
  __shared__ __align__(16) bf16 xs[kH + 2][XP];
  __shared__ float red[8][36];
  const int b = blockIdx.x, c0 = blockIdx.y * 4;
  const float* xb = x + static_cast<long long>(b) * kH * kW;
  const int tx = threadIdx.x;
  for (int r = 0; r < kH + 2; ++r) {
    const int yy = r - 1;
    xs[r][tx + 8] = __float2bfloat16_rn((yy >= 0 && yy < kH) ? xb[yy * kW + tx] : 0.0f);
  }
  if (tx < kH + 2) {
    xs[tx][7] = __float2bfloat16_rn(0.0f);
    xs[tx][kW + 8] = __float2bfloat16_rn(0.0f);
  }
  __syncthreads();
  const long long mtot = static_cast<long long>(n) * kH * kW;
  const int warp = tx >> 5, lane = tx & 31;
  float acc[4][9];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[j][k] = 0.0f;
  const bf16* dyb = dyT + static_cast<long long>(c0) * mtot + static_cast<long long>(b) * kH * kW + 8 * lane;
  // the gradients of the warp's next row are loaded while the current row is summed
  uint4 gn[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) gn[j] = *reinterpret_cast<const uint4*>(dyb + j * mtot + warp * kW);
#pragma unroll 1
  for (int y = warp; y < kH; y += 8) {
    uint4 gq[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) gq[j] = gn[j];
    if (y + 8 < kH) {
#pragma unroll
      for (int j = 0; j < 4; ++j) gn[j] = *reinterpret_cast<const uint4*>(dyb + j * mtot + (y + 8) * kW);
    }
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      // pixels 8 lane - 1 .. 8 lane + 8 of input row y + ky - 1 (staged row y + ky)
      const bf16* row = &xs[y + ky][8 * lane + 8];
      const uint4 mid = *reinterpret_cast<const uint4*>(row);
      const bf16* mv = reinterpret_cast<const bf16*>(&mid);
      float win[10];
      win[0] = __bfloat162float(row[-1]);
#pragma unroll
      for (int k = 0; k < 8; ++k) win[k + 1] = __bfloat162float(mv[k]);
      win[9] = __bfloat162float(row[8]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bf16* g = reinterpret_cast<const bf16*>(&gq[j]);
#pragma unroll
        for (int px = 0; px < 8; ++px) {
          const float gv = __bfloat162float(g[px]);
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) acc[j][ky * 3 + kx] = fmaf(gv, win[px + kx], acc[j][ky * 3 + kx]);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float v = acc[j][k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
      if (lane == 0) red[warp][j * 9 + k] = v;
    }
  __syncthreads();
  if (tx < 36) {
    float v = 0.0f;
#pragma unroll
    for (int w8 = 0; w8 < 8; ++w8) v += red[w8][tx];
    atomicAdd(dw + c0 * 9 + tx, v);
  }
}

// The three horizontally shifted channel-major copies of a channels-last BF16 map
// x[n][h][w][CIN] that the weight-gradient GEMM reads: S[kx][ci][(b, y, xx)] =
// x[b][y][xx + kx - 1][ci], zero where xx + kx - 1 is outside the row. A thread takes 8
// consecutive pixels of one row and one 32-bit word (2 channels) of them, the lanes of a
// warp the words of consecutive pixel groups (coalesced loads): it loads that word of the 10
// pixels it needs and writes 2 x 3 rows of 8 values (16 bytes each).
template <int CIN>
__global__ void __launch_bounds__(256) k_shift3(const bf16* __restrict__ x, int n, int h, int w, bf16* __restrict__ S) {
  constexpr int NW = CIN / 2;  // 32-bit words per pixel
  const long long m = static_cast<long long>(n) * h * w;
  const long long total = m / 8 * NW;  // w is a multiple of 8
  const uint32_t* xw = reinterpret_cast<const uint32_t*>(x);
  for (long long id = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; id < total;
       id += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long gi = id / NW;
    const int q = static_cast<int>(id - gi * NW);
    const long long p0 = gi * 8;  // first pixel (b, y, x0)
    const int x0 = static_cast<int>(p0 % w);
    uint32_t wv[10];  // word q of pixels x0 - 1 .. x0 + 8
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      const int xx = x0 - 1 + k;
      wv[k] = (xx >= 0 && xx < w) ? xw[(p0 - 1 + k) * NW + q] : 0u;
    }
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const uint32_t sel = hf ? 0x7632u : 0x5410u;  // channel 2 q + hf: the high or low halves
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        uint32_t o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) o[e] = __byte_perm(wv[kx + 2 * e], wv[kx + 2 * e + 1], sel);
        *reinterpret_cast<uint4*>(S + (static_cast<long long>(kx) * CIN + 2 * q + hf) * m + p0) =
            make_uint4(o[0], o[1], o[2], o[3]);
      }
    }
  }
}

// out[c * ldo + r] = in[r * cols + c] for r < rows (BF16): 32 x 32 tiles through shared memory,
// both sides coalesced. fc1's input rows transposed for its weight gradient.
__global__ void __launch_bounds__(256) k_transpose(const bf16* __restrict__ in, int rows, int cols,
                                                   bf16* __restrict__ out, long long ldo) {
  __shared__ bf16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = in[static_cast<long long>(r) * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[static_cast<long long>(c) * ldo + r] = tile[threadIdx.x][i];
  }
}

// Gradient through the pooling and the ReLU: the argmax position of each pooled cell gets
// dP if its activation is positive, the other three positions zero. A thread owns one pooled
// pixel and 16 channels c0 .. c0 + 15 (blockIdx.y), the lanes of a warp consecutive pixels of
// one image row (w / 2 is a multiple of 32). CL: dP and the pooled map are channels-last BF16
// [pix][CN] (conv1's and conv2's pooled maps, whose gradient the next layer's input-gradient
// convolution writes), read as 16-byte vectors; else (conv3) dP is FP32 and the pooled map
// BF16, both in fc1's row layout [b][(c, y2, x2)]. Writes dyT[c][m] as two 4-byte pairs per
// channel (upper and lower row), coalesced along the row, and, when dy is set, the
// channels-last dy[m][CN] of its four pixels as 16-byte stores. The bias gradient
// db[c] = sum over m of dY[c][m] (the BF16 values) is reduced over the CTA and added
// atomically.
template <int CN, bool CL>
__global__ void __launch_bounds__(256) k_unpool(const void* __restrict__ dpv, const uint32_t* __restrict__ am,
                                                const bf16* __restrict__ pooled, int n, int h, int w,
                                                bf16* __restrict__ dyT, bf16* __restrict__ dy, float* __restrict__ db) {
  __shared__ float red[8][16];
  // pooled pixel counts and map sizes stay below 2^31 (the workspace is sized for them)
  const int h2 = h / 2, w2 = w / 2;
  const int npix = n * h2 * w2;
  const long long mtot = static_cast<long long>(n) * h * w;
  const int pix = blockIdx.x * 256 + threadIdx.x, c0 = blockIdx.y * 16;
  const bool valid = pix < npix;
  const int x2 = pix % w2, r = pix / w2;
  const int y2 = r % h2, b = r / h2;
  const long long m00 = (static_cast<long long>(b) * h + 2 * y2) * w + 2 * x2;
  // the 16 gradients (as BF16) and the 16 pooled activations of the pixel
  uint32_t gw[8], pw[8];
  uint32_t code = 0;
  if (valid) {
    code = am[static_cast<long long>(blockIdx.y) * npix + pix];
    if constexpr (CL) {
      const uint4* gs = reinterpret_cast<const uint4*>(static_cast<const bf16*>(dpv) + static_cast<long long>(pix) * CN + c0);
      const uint4* ps = reinterpret_cast<const uint4*>(pooled + static_cast<long long>(pix) * CN + c0);
      const uint4 g0 = gs[0], g1 = gs[1], p0 = ps[0], p1 = ps[1];
      gw[0] = g0.x; gw[1] = g0.y; gw[2] = g0.z; gw[3] = g0.w; gw[4] = g1.x; gw[5] = g1.y; gw[6] = g1.z; gw[7] = g1.w;
      pw[0] = p0.x; pw[1] = p0.y; pw[2] = p0.z; pw[3] = p0.w; pw[4] = p1.x; pw[5] = p1.y; pw[6] = p1.z; pw[7] = p1.w;
    } else {
      const float* dpf = static_cast<const float*>(dpv);
      const long long f0 = static_cast<long long>(b) * CN * h2 * w2 + (static_cast<long long>(c0) * h2 + y2) * w2 + x2;
#pragma unroll
      for (int q = 0; q < 16; q += 2) {
        const long long fa = f0 + static_cast<long long>(q) * h2 * w2, fb = fa + static_cast<long long>(h2) * w2;
        const __nv_bfloat162 gp = __floats2bfloat162_rn(dpf[fa], dpf[fb]);
        gw[q >> 1] = *reinterpret_cast<const uint32_t*>(&gp);
        pw[q >> 1] = static_cast<uint32_t>(__bfloat16_as_ushort(pooled[fa])) |
                     (static_cast<uint32_t>(__bfloat16_as_ushort(pooled[fb])) << 16);
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) gw[q] = pw[q] = 0u;
  }
  float bsum[16];
  uint32_t d0[8], d1[8], d2[8], d3[8];  // dy of the four pixels (channel pairs)
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int a = (code >> (2 * j)) & 3;
    const uint32_t graw = (gw[j >> 1] >> ((j & 1) * 16)) & 0xFFFFu;
    const uint32_t praw = (pw[j >> 1] >> ((j & 1) * 16)) & 0xFFFFu;
    const bool live = __bfloat162float(__ushort_as_bfloat16(static_cast<unsigned short>(praw))) > 0.0f;
    const uint32_t u = live ? graw : 0u;
    bsum[j] = __bfloat162float(__ushort_as_bfloat16(static_cast<unsigned short>(u)));
    const uint32_t top = a == 0 ? u : (a == 1 ? (u << 16) : 0u);
    const uint32_t bot = a == 2 ? u : (a == 3 ? (u << 16) : 0u);
    if (valid) {
      const int c = c0 + j;
      *reinterpret_cast<uint32_t*>(dyT + static_cast<long long>(c) * mtot + m00) = top;
      *reinterpret_cast<uint32_t*>(dyT + static_cast<long long>(c) * mtot + m00 + w) = bot;
    }
    const int sh = (j & 1) * 16;
    const uint32_t e0 = (a == 0 ? u : 0u) << sh, e1 = (a == 1 ? u : 0u) << sh;
    const uint32_t e2 = (a == 2 ? u : 0u) << sh, e3 = (a == 3 ? u : 0u) << sh;
    if (j & 1) {
      d0[j >> 1] |= e0; d1[j >> 1] |= e1; d2[j >> 1] |= e2; d3[j >> 1] |= e3;
    } else {
      d0[j >> 1] = e0; d1[j >> 1] = e1; d2[j >> 1] = e2; d3[j >> 1] = e3;
    }
  }
  if (dy && valid) {
    uint4* q0 = reinterpret_cast<uint4*>(dy + m00 * CN + c0);
    uint4* q1 = reinterpret_cast<uint4*>(dy + (m00 + 1) * CN + c0);
    uint4* q2 = reinterpret_cast<uint4*>(dy + (m00 + w) * CN + c0);
    uint4* q3 = reinterpret_cast<uint4*>(dy + (m00 + w + 1) * CN + c0);
    q0[0] = make_uint4(d0[0], d0[1], d0[2], d0[3]); q0[1] = make_uint4(d0[4], d0[5], d0[6], d0[7]);
    q1[0] = make_uint4(d1[0], d1[1], d1[2], d1[3]); q1[1] = make_uint4(d1[4], d1[5], d1[6], d1[7]);
    q2[0] = make_uint4(d2[0], d2[1], d2[2], d2[3]); q2[1] = make_uint4(d2[4], d2[5], d2[6], d2[7]);
    q3[0] = make_uint4(d3[0], d3[1], d3[2], d3[3]); q3[1] = make_uint4(d3[4], d3[5], d3[6], d3[7]);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    float v = bsum[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    float v = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) v += red[k][threadIdx.x];
    atomicAdd(db + c0 + threadIdx.x, v);
  }
}

// fc1's bias and ReLU, fc2, the loss and its gradient, one warp per sample. Forward only
// when y is null.
__global__ void k_head(const float* __restrict__ hf, const float* __restrict__ params, int n,
                       const float* __restrict__ y, float* __restrict__ logits, float* __restrict__ grads,
                       float* __restrict__ loss, bf16* __restrict__ dh, bf16* __restrict__ dhT, int ldt) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const float* wf2 = params + kOffWf2;
  const float* bf1 = params + kOffBf1;
  const float* hrow = hf + static_cast<long long>(warp) * kHid;  // fc1 pre-activation without bias
  float s = 0.0f;
  for (int j = lane; j < kHid; j += 32) s += fmaxf(hrow[j] + bf1[j], 0.0f) * wf2[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  const float z = s + params[kOffBf2];
  if (lane == 0 && logits) logits[warp] = z;
  if (!y) return;
  const float t = y[warp];
  const float sig = 1.0f / (1.0f + __expf(-z));
  const float dz = (sig - t) / static_cast<float>(n);
  if (lane == 0) {
    // log(1 + e^z) - t z, evaluated stably
    const float sp = fmaxf(z, 0.0f) + log1pf(__expf(-fabsf(z)));
    atomicAdd(loss, (sp - t * z) / static_cast<float>(n));
    atomicAdd(grads + kOffBf2, dz);
  }
  for (int j = lane; j < kHid; j += 32) {
    const float hv = fmaxf(hrow[j] + bf1[j], 0.0f);
    atomicAdd(grads + kOffWf2 + j, dz * hv);
    const float g = (hv > 0.0f) ? dz * wf2[j] : 0.0f;
    atomicAdd(grads + kOffBf1 + j, g);
    const bf16 bg = __float2bfloat16_rn(g);
    dh[static_cast<long long>(warp) * kHid + j] = bg;
    dhT[static_cast<long long>(j) * ldt + warp] = bg;
  }
}

// dst[r][ldd] (or dst[c][ldd] transposed) = bf16(src[r][cols]), zero-padded to ldd
__global__ void k_cast_w(const float* __restrict__ src, int rows, int cols, bf16* __restrict__ dst, int ldd,
                         int transposed, int dst_rows) {
  const long long total = static_cast<long long>(dst_rows) * ldd;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int a = static_cast<int>(i / ldd), b = static_cast<int>(i - static_cast<long long>(a) * ldd);
    float v = 0.0f;
    if (!transposed) {
      if (a < rows && b < cols) v = src[static_cast<long long>(a) * cols + b];
    } else {
      if (b < rows && a < cols) v = src[static_cast<long long>(b) * cols + a];
    }
    dst[i] = __float2bfloat16_rn(v);
  }
}

// dst[ci][tap*cout + co] = bf16(src[co][ci*9 + (8 - tap)]), zero to kp: the kernel of the input
// gradient as a forward convolution of dY (rotated by 180 degrees, in and out channels swapped)
__global__ void k_cast_w_flip(const float* __restrict__ src, int cout, int cin, bf16* __restrict__ dst, int kp) {
  const long long total = static_cast<long long>(cin) * kp;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int ci = static_cast<int>(i / kp), k = static_cast<int>(i - static_cast<long long>(ci) * kp);
    float v = 0.0f;
    if (k < 9 * cout) {
      const int tap = k / cout, co = k - tap * cout;
      v = src[static_cast<long long>(co) * 9 * cin + ci * 9 + (8 - tap)];
    }
    dst[i] = __float2bfloat16_rn(v);
  }
}

// dst[co][tap*cin + ci] = bf16(src[co][ci*9 + tap]) (the tap-major K of k_conv_halo), zero to kp
__global__ void k_cast_w_tap(const float* __restrict__ src, int cout, int cin, bf16* __restrict__ dst, int kp) {
  const long long total = static_cast<long long>(cout) * kp;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int co = static_cast<int>(i / kp), k = static_cast<int>(i - static_cast<long long>(co) * kp);
    float v = 0.0f;
    if (k < 9 * cin) {
      const int tap = k / cin, ci = k - tap * cin;
      v = src[static_cast<long long>(co) * 9 * cin + ci * 9 + tap];
    }
    dst[i] = __float2bfloat16_rn(v);
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, long long np, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < np;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gi;
    const float v = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    p[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
  }
}

// One block per snippet: 64 x 256 plane cells around (row, col), standardised with the FP64
// mean and population std of the present cells (std 0 -> 1); missing cells are 0.
__global__ void __launch_bounds__(256) k_snippets(const float* __restrict__ plane, long long ld, int ndm,
                                                  long long ncols, const int32_t* __restrict__ rows,
                                                  const int64_t* __restrict__ cols, int n, float* __restrict__ out) {
  const int s = blockIdx.x;
  if (s >= n) return;
  const int r0 = rows[s] - 32;
  const long long c0 = cols[s] - 128;
  double s1 = 0.0, s2 = 0.0;
  long long cnt = 0;
  for (int i = threadIdx.x; i < kH * kW; i += blockDim.x) {
    const int r = r0 + i / kW;
    const long long c = c0 + (i % kW);
    if (r >= 0 && r < ndm && c >= 0 && c < ncols) {
      const double v = plane[static_cast<long long>(r) * ld + c];
      s1 += v;
      s2 += v * v;
      ++cnt;
    }
  }
  __shared__ double r1[8], r2[8];
  __shared__ long long rc[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, o);
    s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, o);
    cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = s1;
    r2[threadIdx.x >> 5] = s2;
    rc[threadIdx.x >> 5] = cnt;
  }
  __syncthreads();
  s1 = s2 = 0.0;
  cnt = 0;
  for (int k = 0; k < 8; ++k) {
    s1 += r1[k];
    s2 += r2[k];
    cnt += rc[k];
  }
  const double mu = cnt ? s1 / cnt : 0.0;
  const double var = cnt ? s2 / cnt - mu * mu : 0.0;
  const double sd = var > 0.0 ? sqrt(var) : 1.0;
  float* o = out + static_cast<long long>(s) * kH * kW;
  for (int i = threadIdx.x; i < kH * kW; i += blockDim.x) {
    const int r = r0 + i / kW;
    const long long c = c0 + (i % kW);
    float v = 0.0f;
    if (r >= 0 && r < ndm && c >= 0 && c < ncols)
      v = static_cast<float>((plane[static_cast<long long>(r) * ld + c] - mu) / sd);
    o[i] = v;
  }
}

// ---------------------------------------------------------------- host side

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 2-D K-major BF16 operand: `rows` rows of `kext` valid elements, `pitch` elements apart;
// boxes of 64 x box_rows, 128-byte swizzle, zero fill outside.
bool make_map(CUtensorMap* m, const void* base, long long kext, long long rows, long long pitch, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(base) & 15u) || (pitch * 2) % 16 != 0 || kext < 1 || rows < 1)
    return false;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(kext), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(pitch * 2)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(kBK), static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, bool WG = false>
cudaError_t launch_gemm_bn(const CUtensorMap& ma, const CUtensorMap& mb, int M, int N, int ktiles, int splits,
                           const Epi& epi, uint32_t* err, cudaStream_t s, Wg wg = Wg{0, 0, 0}) {
  const int smem = kStages * (kBM + BN) * kBK * 2 + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_gemm<BN, WG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  // CTAs: every output tile gets its own, and K is split (at most `splits` ways, at least 8 K
  // steps a split) so that tiles x splits fill the GPU once (shared memory bounds the CTAs per
  // SM); with more tiles than that, each CTA walks several tiles
  const long long tiles = 1LL * ((M + kBM - 1) / kBM) * ((N + BN - 1) / BN);
  const int per_sm = std::max(1, (227 * 1024) / smem);
  const long long slots = 152LL * per_sm;
  long long want_splits = std::max<long long>(1, slots / std::max<long long>(1, tiles));
  want_splits = std::min<long long>(want_splits, std::max(1, ktiles / 8));
  const int nsplit = static_cast<int>(std::max<long long>(1, std::min<long long>(splits, want_splits)));
  const int per = (ktiles + nsplit - 1) / nsplit;
  const int nz = (ktiles + per - 1) / per;
  dim3 grid(static_cast<unsigned>(std::min(tiles, std::max<long long>(1, slots / nz))), 1, nz);
  k_gemm<BN, WG><<<grid, 192, smem, s>>>(ma, mb, M, N, ktiles, per, epi, err, wg);
  return cudaGetLastError();
}

// C[M][N] = A[M][K] . B[N][K]^T, A and B BF16 K-major with pitches lda / ldb (elements).
// splits > 1 splits K over CTAs (epi.atomic must be set, output pre-zeroed).
int gemm(const bf16* A, long long lda, const bf16* B, long long ldb, int M, int N, long long K, const Epi& epi,
         int splits, uint32_t* err, cudaStream_t s, int64_t* launches) {
  const int BN = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, K, M, lda, kBM) || !make_map(&mb, B, K, N, ldb, BN)) return SND_ERR_UNSUPPORTED;
  const int ktiles = static_cast<int>((K + kBK - 1) / kBK);
  splits = std::max(1, std::min(splits, ktiles));
  cudaError_t e;
  if (BN == 32) {
    e = launch_gemm_bn<32>(ma, mb, M, N, ktiles, splits, epi, err, s);
  } else if (BN == 64) {
    e = launch_gemm_bn<64>(ma, mb, M, N, ktiles, splits, epi, err, s);
  } else {
    e = launch_gemm_bn<128>(ma, mb, M, N, ktiles, splits, epi, err, s);
  }
  if (launches) *launches += 1;
  return e == cudaSuccess ? SND_OK : SND_ERR_CUDA;
}

// Weight gradient of a 3x3 convolution, dW[cout][ci * 9 + tap] += sum over pixels m of
// dY^T[cout][m] * x[m + tap offset][ci], with k_gemm in weight-gradient mode: A = dY^T (K-major
// over the n * h * w pixels), B from the three horizontally shifted channel-major copies of
// the input map S[3][cin][n][h][w] (k_shift3). cin a multiple of 16, w a multiple of 64.
int gemm_wg(const bf16* dyT, int cout, const bf16* S, int n, int h, int w, int cin, float* dw, uint32_t* err,
            cudaStream_t s, int64_t* launches) {
  EncodeTiledFn fn = encode_fn();
  const long long m = 1LL * n * h * w;
  if (!fn || cin % 16 != 0 || w % kBK != 0 || (reinterpret_cast<uintptr_t>(S) & 15u)) return SND_ERR_UNSUPPORTED;
  CUtensorMap ma, mb;
  if (cout > kBM || cout % 8 != 0 || !make_map(&ma, dyT, m, cout, m, cout)) return SND_ERR_UNSUPPORTED;
  const cuuint64_t dims[5] = {static_cast<cuuint64_t>(w), static_cast<cuuint64_t>(h), static_cast<cuuint64_t>(n),
                              static_cast<cuuint64_t>(cin), 3};
  const cuuint64_t strides[4] = {static_cast<cuuint64_t>(w) * 2, static_cast<cuuint64_t>(h) * w * 2,
                                 static_cast<cuuint64_t>(m) * 2, static_cast<cuuint64_t>(cin) * m * 2};
  const cuuint32_t box[5] = {static_cast<cuuint32_t>(kBK), 3, 1, 16, 3};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  if (fn(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(S), dims, strides, box, estr,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return SND_ERR_UNSUPPORTED;
  Epi e{nullptr, 0, dw, 0, 0, 1, 9LL * cin};
  const int ktiles = static_cast<int>(m / kBK);
  const cudaError_t ce = launch_gemm_bn<144, true>(ma, mb, cout, 9 * cin, ktiles, ktiles, e, err, s, Wg{h, w, cout});
  if (launches) *launches += 1;
  return ce == cudaSuccess ? SND_OK : SND_ERR_CUDA;
}

// Persistent grid of a kernel with `smem` bytes of dynamic shared memory, `threads` per CTA
// and `tmem_cols` TMEM columns: as many CTAs as fit on an SM at once by shared memory (the
// carveout set to its maximum), threads, registers and TMEM (512 columns, so that no CTA's
// allocation ever waits for another's), times the SMs, at most `items`.
template <typename K>
cudaError_t persistent_grid(K kern, int smem, int threads, int tmem_cols, int items, int* grid) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  cudaFuncAttributes fa{};
  int dev = 0, nsm = 0;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int regs = ((std::max(fa.numRegs, 1) + 7) / 8) * 8;
  int per_sm = (227 * 1024) / (smem + static_cast<int>(fa.sharedSizeBytes) + 1024);
  per_sm = std::min(per_sm, 2048 / threads);
  per_sm = std::min(per_sm, 65536 / (regs * ((threads + 31) / 32) * 32));
  per_sm = std::min(per_sm, 512 / tmem_cols);
  *grid = std::max(1, std::min(items, nsm * std::max(per_sm, 1)));
  return cudaSuccess;
}

// Forward 3x3 convolution and 2x2 max pooling of a channels-last [n][h][w][cin] BF16 map
// with k_conv_halo: pooled output channels-last [(b, y2, x2)][cout] (pool_cl) or
// [b][(c, y2, x2)], with am set (training) also the argmax of every pooled cell. With dx set
// instead: the plain convolution (no bias, ReLU or pooling) into dx[(b, y, x)][cout] BF16,
// which with dY as x and the flipped kernel is a layer's input gradient. Weights wb[cout][kp]
// BF16, tap-major K.
int conv_halo(const bf16* x, int n, int h, int w, int cin, const bf16* wb, int kp, int cout, const float* bias,
              bf16* pool, int pool_cl, uint32_t* err, cudaStream_t s, int64_t* launches, uint32_t* am = nullptr,
              bf16* dx = nullptr) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(x) & 15u)) return SND_ERR_UNSUPPORTED;
  const cuuint64_t dims[4] = {static_cast<cuuint64_t>(cin), static_cast<cuuint64_t>(w), static_cast<cuuint64_t>(h),
                              static_cast<cuuint64_t>(n)};
  const cuuint64_t strides[3] = {static_cast<cuuint64_t>(cin) * 2, static_cast<cuuint64_t>(w) * cin * 2,
                                 static_cast<cuuint64_t>(h) * w * cin * 2};
  // four rows with a pixel of zero padding each side
  const cuuint32_t box[4] = {8, static_cast<cuuint32_t>(w + 2), 4, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUtensorMap mx;
  if (fn(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(x), dims, strides, box, estr,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return SND_ERR_UNSUPPORTED;
  ConvArgs a{n, h, bias, pool, pool_cl, am, dx};
  const int items = n * (h / 2);
  auto go = [&](auto kern, int npl, int cw) {
    // stages x planes x 4 rows x (w + 2) pixels x 16 bytes, then the weights
    const int stage = npl * 4 * (w + 2) * 16;
    const int smem = 128 + halo_stages(8 * npl, cw, w) * stage + 9 * npl * cw * 16;
    int grid = 0;
    const cudaError_t e = persistent_grid(kern, smem, 320, 4 * cw, items, &grid);
    if (e != cudaSuccess) return e;
    kern<<<grid, 320, smem, s>>>(mx, a, wb, kp, err);
    return cudaGetLastError();
  };
  cudaError_t e;
  if (h % 2 != 0) return SND_ERR_UNSUPPORTED;
  if (dx) {
    if (cin == 32 && cout == 16 && w == 128) {
      e = go(k_conv_halo<32, 16, 128, false, true>, 4, 16);
    } else if (cin == 64 && cout == 32 && w == 64) {
      e = go(k_conv_halo<64, 32, 64, false, true>, 8, 32);
    } else {
      return SND_ERR_UNSUPPORTED;
    }
  } else if (cin == 16 && cout == 32 && w == 128) {
    e = am ? go(k_conv_halo<16, 32, 128, true>, 2, 32) : go(k_conv_halo<16, 32, 128, false>, 2, 32);
  } else if (cin == 32 && cout == 64 && w == 64) {
    e = am ? go(k_conv_halo<32, 64, 64, true>, 4, 64) : go(k_conv_halo<32, 64, 64, false>, 4, 64);
  } else {
    return SND_ERR_UNSUPPORTED;
  }
  if (launches) *launches += 1;
  return e == cudaSuccess ? SND_OK : SND_ERR_CUDA;
}

// conv1 of FP32 snippets x[n][64][256] on the tensor cores (k_conv1_tc) with its pooling,
// channels-last [(b, y2, x2)][16]; with am set (training) also the argmax of every pooled cell.
int conv1_tc(const float* x, int n, const float* w, const float* bias, bf16* out, uint32_t* am, uint32_t* err,
             cudaStream_t s, int64_t* launches) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(x) & 15u)) return SND_ERR_UNSUPPORTED;
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(kW), static_cast<cuuint64_t>(kH), static_cast<cuuint64_t>(n)};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(kW) * 4, static_cast<cuuint64_t>(kH) * kW * 4};
  const cuuint32_t box[3] = {136, 4, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUtensorMap mx;
  if (fn(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(x), dims, strides, box, estr,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return SND_ERR_UNSUPPORTED;
  const int smem = 128 + 4 * (5 * 128 * 16) + 12 * (4 * 136 * 4);
  const int items = n * 64;
  auto go = [&](auto kern) {
    int grid = 0;
    const cudaError_t e = persistent_grid(kern, smem, 320, 64, items, &grid);
    if (e != cudaSuccess) return e;
    kern<<<grid, 320, smem, s>>>(mx, n, w, bias, out, am, err);
    return cudaGetLastError();
  };
  const cudaError_t e = am ? go(k_conv1_tc<true>) : go(k_conv1_tc<false>);
  if (launches) *launches += 1;
  return e == cudaSuccess ? SND_OK : SND_ERR_CUDA;
}

int grid_for(long long total) { return static_cast<int>(std::min<long long>((total + 255) / 256, 152LL * 32)); }

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Sifter {
  int bm = 0;        // batch capacity (multiple of 64)
  int training = 0;
  uint64_t seed = 0;
  std::vector<float> init;
  size_t ws_bytes = 0;
  char* ws = nullptr;
  bool bound = false;
  int sticky = 0;
  int64_t step = 0;
  int64_t launches = 0;
  cudaStream_t last = nullptr;
  struct {
    size_t params, grads, m1, m2, err, loss, wb[3], wT[3], wf1b, wf1T, p[3], am[3], p3, p3T, hf,
        logits, dh, dhT, dp3, dy[3], dyT[3], s3[3], dp[3];
  } o{};
};

template <typename T>
T* at(const Sifter& f, size_t off) {
  return reinterpret_cast<T*>(f.ws + off);
}

void layout(Sifter& f) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t a = o;
    o = align256(o + bytes);
    return a;
  };
  const long long B = f.bm;
  const size_t P = static_cast<size_t>(kNumParams);
  f.o.params = take(4 * P);
  f.o.grads = take(4 * P);
  f.o.m1 = take(f.training ? 4 * P : 0);
  f.o.m2 = take(f.training ? 4 * P : 0);
  f.o.err = take(16);
  f.o.loss = take(16);
  for (int l = 0; l < 3; ++l) {
    const ConvL& c = kConv[l];
    const long long m = B * c.h * c.w;
    f.o.wb[l] = take(2ull * c.cout * c.kp);
    f.o.wT[l] = take(2ull * c.cin * ((9 * c.cout + kBK - 1) / kBK * kBK));
    f.o.p[l] = take(2ull * c.cout * m / 4);
    f.o.am[l] = take(4ull * (c.cout / 16) * (m / 4));
    if (f.training) {
      f.o.dy[l] = take(l > 0 ? 2ull * m * c.cout : 0);
      f.o.dyT[l] = take(2ull * c.cout * m);
      f.o.s3[l] = take(l > 0 ? 2ull * 3 * c.cin * m : 0);  // the shifted copies of the layer's input
      f.o.dp[l] = take(l < 2 ? 2ull * c.cout * m / 4 : 0);
    }
  }
  f.o.wf1b = take(2ull * kHid * kFeat);
  f.o.wf1T = take(f.training ? 2ull * kFeat * kHid : 0);
  f.o.p3 = take(2ull * B * kFeat);
  f.o.p3T = take(2ull * B * kFeat);
  f.o.hf = take(4ull * B * kHid);
  f.o.logits = take(4ull * B);
  if (f.training) {
    f.o.dh = take(2ull * B * kHid);
    f.o.dhT = take(2ull * B * kHid);
    f.o.dp3 = take(4ull * B * kFeat);
  }
  f.ws_bytes = o;
}

// counter-based uniform in [-1, 1): splitmix64 of (seed, index)
float uniform_pm1(uint64_t seed, uint64_t i) {
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return static_cast<float>(static_cast<double>(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
}

int fail(Sifter& f, int code) {
  if (!f.sticky) f.sticky = code;
  return code;
}

// BF16 copies of the weights (and the transposes the input-gradient GEMMs read)
cudaError_t prep_weights(Sifter& f, cudaStream_t s) {
  const float* P = at<float>(f, f.o.params);
  for (int l = 0; l < 3; ++l) {
    const ConvL& c = kConv[l];
    if (l == 0) {
      k_cast_w<<<grid_for(1LL * c.cout * c.kp), 256, 0, s>>>(P + kOffW[l], c.cout, c.kc, at<bf16>(f, f.o.wb[l]), c.kp,
                                                           0, c.cout);
    } else {  // tap-major K for k_conv_halo
      k_cast_w_tap<<<grid_for(1LL * c.cout * c.kp), 256, 0, s>>>(P + kOffW[l], c.cout, c.cin, at<bf16>(f, f.o.wb[l]),
                                                               c.kp);
    }
    f.launches++;
    if (f.training && l > 0) {  // the input gradient's flipped kernel, [cin][kpd]
      const int kpd = (9 * c.cout + kBK - 1) / kBK * kBK;
      k_cast_w_flip<<<grid_for(1LL * c.cin * kpd), 256, 0, s>>>(P + kOffW[l], c.cout, c.cin, at<bf16>(f, f.o.wT[l]),
                                                               kpd);
      f.launches++;
    }
  }
  k_cast_w<<<grid_for(1LL * kHid * kFeat), 256, 0, s>>>(P + kOffWf1, kHid, kFeat, at<bf16>(f, f.o.wf1b), kFeat, 0,
                                                        kHid);
  f.launches++;
  if (f.training) {
    k_cast_w<<<grid_for(1LL * kHid * kFeat), 256, 0, s>>>(P + kOffWf1, kHid, kFeat, at<bf16>(f, f.o.wf1T), kHid, 1,
                                                          kFeat);
    f.launches++;
  }
  return cudaGetLastError();
}

// forward pass of n snippets x[n][64][256] (FP32) into the hidden layer and the logits
int forward(Sifter& f, const float* x, int n, cudaStream_t s) {
  uint32_t* err = at<uint32_t>(f, f.o.err);
  const float* P = at<float>(f, f.o.params);
  // every convolution runs with its 2x2 max pooling in the epilogue; a sifter with training
  // state also keeps the argmax of every pooled cell (and fc1's input rows transposed), which
  // is all the backward pass needs of the forward activations
  uint32_t* am[3] = {nullptr, nullptr, nullptr};
  if (f.training)
    for (int l = 0; l < 3; ++l) am[l] = at<uint32_t>(f, f.o.am[l]);
  {
    const int rc = conv1_tc(x, n, P + kOffW[0], P + kOffB[0], at<bf16>(f, f.o.p[0]), am[0], err, s, &f.launches);
    if (rc) return rc;
  }
  for (int l = 1; l < 3; ++l) {
    const ConvL& c = kConv[l];
    // channels-last for conv3, fc1's feature rows after conv3
    const int rc = conv_halo(at<bf16>(f, f.o.p[l - 1]), n, c.h, c.w, c.cin, at<bf16>(f, f.o.wb[l]), c.kp, c.cout,
                             P + kOffB[l], l == 1 ? at<bf16>(f, f.o.p[l]) : at<bf16>(f, f.o.p3), l == 1 ? 1 : 0, err, s,
                             &f.launches, am[l]);
    if (rc) return rc;
  }
  if (f.training) {  // fc1's input rows transposed, for its weight gradient
    k_transpose<<<dim3((kFeat + 31) / 32, (n + 31) / 32), dim3(32, 8), 0, s>>>(at<bf16>(f, f.o.p3), n, kFeat,
                                                                             at<bf16>(f, f.o.p3T), f.bm);
    f.launches++;
  }
  // fc1 pre-activation (bias and ReLU are applied where it is read, in k_head), computed as
  // its transpose hf^T[hid][b] = Wf1 . F^T and stored transposed into hf[b][hid] (the lanes
  // of an epilogue warp hold consecutive hid: coalesced); K split over CTAs: only
  // ceil(n / 128) output tiles exist
  if (cudaMemsetAsync(at<float>(f, f.o.hf), 0, 4ull * n * kHid, s) != cudaSuccess) return SND_ERR_CUDA;
  Epi e{nullptr, 0, at<float>(f, f.o.hf), 0, 1, 1, kHid};
  const int ntiles = (n + kBM - 1) / kBM;
  const int splits = std::max(1, std::min(kFeat / kBK, 2 * 152 / ntiles));
  return gemm(at<bf16>(f, f.o.wf1b), kFeat, at<bf16>(f, f.o.p3), kFeat, kHid, n, kFeat, e, splits, err, s,
              &f.launches);
}

// gradients of the mean loss over n snippets into the grads vector (zeroed here)
int backward(Sifter& f, const float* x, const float* y, int n, cudaStream_t s) {
  uint32_t* err = at<uint32_t>(f, f.o.err);
  float* G = at<float>(f, f.o.grads);
  const float* P = at<float>(f, f.o.params);
  if (cudaMemsetAsync(G, 0, 4ull * kNumParams, s) != cudaSuccess ||
      cudaMemsetAsync(at<float>(f, f.o.loss), 0, 4, s) != cudaSuccess)
    return SND_ERR_CUDA;
  k_head<<<(n * 32 + 255) / 256, 256, 0, s>>>(at<float>(f, f.o.hf), P, n, y, at<float>(f, f.o.logits), G,
                                               at<float>(f, f.o.loss), at<bf16>(f, f.o.dh), at<bf16>(f, f.o.dhT), f.bm);
  f.launches++;
  // fc1: dWf1 = dH^T . F ; dF = dH . Wf1, each computed as its transpose (M = the 16384
  // features) and stored transposed, so the lanes of an epilogue warp write consecutive
  // features (coalesced)
  {
    Epi e{nullptr, 0, G + kOffWf1, 0, 1, 0, kFeat};
    // K = n valid columns of rows pitched by the batch capacity (the rest reads as zero)
    int rc = gemm(at<bf16>(f, f.o.p3T), f.bm, at<bf16>(f, f.o.dhT), f.bm, kFeat, kHid, n, e, 1, err, s, &f.launches);
    if (rc) return rc;
    Epi e2{nullptr, 0, at<float>(f, f.o.dp3), 0, 1, 0, kFeat};
    rc = gemm(at<bf16>(f, f.o.wf1T), kHid, at<bf16>(f, f.o.dh), kHid, kFeat, n, kHid, e2, 1, err, s, &f.launches);
    if (rc) return rc;
  }
  for (int l = 2; l >= 0; --l) {
    const ConvL& c = kConv[l];
    const long long m = 1LL * n * c.h * c.w;
    bf16* dyT = at<bf16>(f, f.o.dyT[l]);
    bf16* dy = l > 0 ? at<bf16>(f, f.o.dy[l]) : nullptr;
    {
      // the routed gradient and, fused, the bias gradient
      const dim3 ub(static_cast<unsigned>((m / 4 + 255) / 256), static_cast<unsigned>(c.cout / 16));
      const uint32_t* am = at<uint32_t>(f, f.o.am[l]);
      const bf16* yl = l == 2 ? at<bf16>(f, f.o.p3) : at<bf16>(f, f.o.p[l]);  // the pooled map
      float* db = G + kOffB[l];
      if (l == 0) {
        k_unpool<16, true><<<ub, 256, 0, s>>>(at<bf16>(f, f.o.dp[l]), am, yl, n, c.h, c.w, dyT, dy, db);
      } else if (l == 1) {
        k_unpool<32, true><<<ub, 256, 0, s>>>(at<bf16>(f, f.o.dp[l]), am, yl, n, c.h, c.w, dyT, dy, db);
      } else {
        k_unpool<64, false><<<ub, 256, 0, s>>>(at<float>(f, f.o.dp3), am, yl, n, c.h, c.w, dyT, dy, db);
      }
    }
    f.launches++;
    // weight gradient
    if (l == 0) {
      static_assert(kW == 256 && kH + 2 <= 256, "k_dw1 geometry");
      k_dw1<<<dim3(static_cast<unsigned>(n), 4), 256, 0, s>>>(x, n, dyT, G + kOffW[0]);
      f.launches++;
      break;
    }
    bf16* S = at<bf16>(f, f.o.s3[l]);
    {
      const unsigned sg = static_cast<unsigned>(std::min<long long>((m / 8 * (c.cin / 2) + 255) / 256, 152LL * 8));
      if (c.cin == 16) {
        k_shift3<16><<<sg, 256, 0, s>>>(at<bf16>(f, f.o.p[l - 1]), n, c.h, c.w, S);
      } else {
        k_shift3<32><<<sg, 256, 0, s>>>(at<bf16>(f, f.o.p[l - 1]), n, c.h, c.w, S);
      }
      f.launches++;
    }
    int rc = gemm_wg(dyT, c.cout, S, n, c.h, c.w, c.cin, G + kOffW[l], err, s, &f.launches);
    if (rc) return rc;
    // input gradient, straight into the previous pooled map's gradient dP[cin][m]: the
    // convolution of dY with the flipped kernel, on the halo kernel
    rc = conv_halo(dy, n, c.h, c.w, c.cout, at<bf16>(f, f.o.wT[l]), (9 * c.cout + kBK - 1) / kBK * kBK, c.cin, nullptr,
                   nullptr, 0, err, s, &f.launches, nullptr, at<bf16>(f, f.o.dp[l - 1]));
    if (rc) return rc;
  }
  return cudaGetLastError() == cudaSuccess ? SND_OK : SND_ERR_CUDA;
}

int check_run(Sifter& f, const void* x, int n) {
  if (f.sticky) return f.sticky;
  if (!f.bound) return SND_ERR_STATE;
  if (!x || n < 1 || n > f.bm) return SND_ERR_ARG;
  return SND_OK;
}

int read_err(Sifter& f, cudaStream_t s) {
  uint32_t e = 0;
  if (cudaMemcpyAsync(&e, at<uint32_t>(f, f.o.err), 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(f, SND_ERR_CUDA);
  return e ? fail(f, SND_ERR_TIMEOUT) : SND_OK;
}

}  // namespace

extern "C" int snd_sifter_create(int32_t max_batch, int32_t training, uint64_t seed, snd_sifter_t* out) {
  if (out) *out = nullptr;
  if (!out || max_batch < 1 || max_batch > (1 << 16)) return SND_ERR_ARG;
  Sifter* f = new (std::nothrow) Sifter();
  if (!f) return SND_ERR_NOMEM;
  f->bm = (max_batch + 63) / 64 * 64;
  f->training = training ? 1 : 0;
  f->seed = seed;
  try {
    f->init.assign(static_cast<size_t>(kNumParams), 0.0f);
    auto fill = [&](long long off, long long count, int fan_in) {
      const float bound = std::sqrt(6.0f / static_cast<float>(fan_in));
      for (long long i = 0; i < count; ++i) f->init[off + i] = bound * uniform_pm1(seed, static_cast<uint64_t>(off + i));
    };
    for (int l = 0; l < 3; ++l) fill(kOffW[l], 1LL * kConv[l].cout * kConv[l].kc, kConv[l].kc);
    fill(kOffWf1, 1LL * kHid * kFeat, kFeat);
    fill(kOffWf2, kHid, kHid);
  } catch (...) {
    delete f;
    return SND_ERR_NOMEM;
  }
  layout(*f);
  *out = reinterpret_cast<snd_sifter_t>(f);
  return SND_OK;
}

extern "C" int64_t snd_sifter_num_params(void) { return kNumParams; }

extern "C" size_t snd_sifter_workspace_size(snd_sifter_t h) {
  return h ? reinterpret_cast<Sifter*>(h)->ws_bytes : 0;
}

extern "C" int snd_sifter_bind_workspace(snd_sifter_t h, void* d_ws, size_t bytes, void* stream) {
  if (!h) return SND_ERR_ARG;
  Sifter& f = *reinterpret_cast<Sifter*>(h);
  if (!d_ws || bytes < f.ws_bytes || (reinterpret_cast<uintptr_t>(d_ws) & 255u)) return SND_ERR_WORKSPACE;
  if (!encode_fn()) return SND_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  f.ws = static_cast<char*>(d_ws);
  if (cudaMemsetAsync(d_ws, 0, f.ws_bytes, s) != cudaSuccess ||
      cudaMemcpyAsync(f.ws + f.o.params, f.init.data(), 4ull * kNumParams, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      prep_weights(f, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return SND_ERR_CUDA;
  f.bound = true;
  f.sticky = 0;
  f.step = 0;
  f.last = s;
  return SND_OK;
}

extern "C" int snd_sifter_set_params(snd_sifter_t h, const float* host_params, int64_t n, void* stream) {
  if (!h || !host_params || n != kNumParams) return SND_ERR_ARG;
  Sifter& f = *reinterpret_cast<Sifter*>(h);
  if (!f.bound) return SND_ERR_STATE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(f.ws + f.o.params, host_params, 4ull * kNumParams, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      prep_weights(f, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return fail(f, SND_ERR_CUDA);
  if (f.training && (cudaMemsetAsync(f.ws + f.o.m1, 0, 4ull * kNumParams, s) != cudaSuccess ||
                     cudaMemsetAsync(f.ws + f.o.m2, 0, 4ull * kNumParams, s) != cudaSuccess))
    return fail(f, SND_ERR_CUDA);
  f.step = 0;
  return SND_OK;
}

extern "C" int snd_sifter_get_params(snd_sifter_t h, float* host_params, int64_t n) {
  if (!h || !host_params || n != kNumParams) return SND_ERR_ARG;
  Sifter& f = *reinterpret_cast<Sifter*>(h);
  if (!f.bound) return SND_ERR_STATE;
  if (cudaStreamSynchronize(f.last) != cudaSuccess ||
      cudaMemcpy(host_params, f.ws + f.o.params, 4ull * kNumParams, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(f, SND_ERR_CUDA);
  return SND_OK;
}

extern "C" int snd_sifter_forward(snd_sifter_t h, const float* d_x, int32_t n, float* d_logits, void* stream) {
  if (!h || !d_logits) return SND_ERR_ARG;
  Sifter& f = *reinterpret_cast<Sifter*>(h);
  int rc = check_run(f, d_x, n);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = forward(f, d_x, n, s);
  if (rc) return fail(f, rc);
  k_head<<<(n * 32 + 255) / 256, 256, 0, s>>>(at<float>(f, f.o.hf), at<float>(f, f.o.params), n, nullptr, d_logits,
                                               nullptr, nullptr, nullptr, nullptr, f.bm);
  f.launches++;
  f.last = s;
  return cudaGetLastError() == cudaSuccess ? SND_OK : fail(f, SND_ERR_CUDA);
}

extern "C" int snd_sifter_gradients(snd_sifter_t h, const float* d_x, const float* d_y, int32_t n, float* d_grads,
                                    float* d_loss, void* stream) {
  if (!h || !d_y) return SND_ERR_ARG;
  Sifter& f = *reinterpret_cast<Sifter*>(h);
  if (!f.training) return SND_ERR_STATE;
  int rc = check_run(f, d_x, n);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = forward(f, d_x, n, s);
  if (!rc) rc = backward(f, d_x, d_y, n, s);
  if (rc) return fail(f, rc);
  if (d_grads && cudaMemcpyAsync(d_grads, f.ws + f.o.grads, 4ull * kNumParams, cudaMemcpyDeviceToDevice, s) !=
                     cudaSuccess)
    return fail(f, SND_ERR_CUDA);
  if (d_loss && cudaMemcpyAsync(d_loss, f.ws + f.o.loss, 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return fail(f, SND_ERR_CUDA);
  f.last = s;
  return read_err(f, s);
}

extern "C" int snd_sifter_train_step(snd_sifter_t h, const float* d_x, const float* d_y, int32_t n, float lr,
                                     float* d_loss, void* stream) {
  if (!h || !d_y || !(lr > 0.0f)) return SND_ERR_ARG;
  Sifter& f = *reinterpret_cast<Sifter*>(h);
  if (!f.training) return SND_ERR_STATE;
  int rc = check_run(f, d_x, n);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = forward(f, d_x, n, s);
  if (!rc) rc = backward(f, d_x, d_y, n, s);
  if (rc) return fail(f, rc);
  ++f.step;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, static_cast<float>(f.step));
  const float c2 = 1.0f - std::pow(b2, static_cast<float>(f.step));
  k_adam<<<grid_for(kNumParams), 256, 0, s>>>(at<float>(f, f.o.params), at<float>(f, f.o.grads), at<float>(f, f.o.m1),
                                              at<float>(f, f.o.m2), kNumParams, lr, b1, b2, 1e-8f, c1, c2);
  f.launches++;
  if (prep_weights(f, s) != cudaSuccess) return fail(f, SND_ERR_CUDA);
  if (d_loss && cudaMemcpyAsync(d_loss, f.ws + f.o.loss, 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return fail(f, SND_ERR_CUDA);
  f.last = s;
  return cudaGetLastError() == cudaSuccess ? SND_OK : fail(f, SND_ERR_CUDA);
}

extern "C" int snd_sifter_status(snd_sifter_t h) {
  if (!h) return SND_ERR_ARG;
  Sifter& f = *reinterpret_cast<Sifter*>(h);
  if (!f.bound) return SND_ERR_STATE;
  if (f.sticky) return f.sticky;
  return read_err(f, f.last);
}

extern "C" int64_t snd_sifter_launches(snd_sifter_t h) { return h ? reinterpret_cast<Sifter*>(h)->launches : 0; }

extern "C" void snd_sifter_destroy(snd_sifter_t h) { delete reinterpret_cast<Sifter*>(h); }

extern "C" int snd_snippets(const float* d_plane, int64_t ld, int32_t ndm, int64_t ncols, const int32_t* d_rows,
                            const int64_t* d_cols, int32_t n, float* d_out, void* stream) {
  if (!d_plane || !d_rows || !d_cols || !d_out || n < 0 || ndm < 1 || ncols < 1 || ld < ncols) return SND_ERR_ARG;
  if (n == 0) return SND_OK;
  k_snippets<<<n, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_plane, ld, ndm, ncols, d_rows, d_cols, n, d_out);
  return cudaGetLastError() == cudaSuccess ? SND_OK : SND_ERR_CUDA;
}

extern "C" int snd_gemm_bf16(const void* d_a, int64_t lda, const void* d_b, int64_t ldb, int32_t m, int32_t n,
                             int64_t k, float* d_c, int64_t ldc, int32_t splits, uint32_t* d_err, void* stream) {
  if (!d_a || !d_b || !d_c || !d_err || m < 1 || n < 1 || k < 1 || lda < k || ldb < k || ldc < n || splits < 1)
    return SND_ERR_ARG;
  Epi e{nullptr, 0, d_c, 0, 0, splits > 1 ? 1 : 0, ldc};
  return gemm(static_cast<const bf16*>(d_a), lda, static_cast<const bf16*>(d_b), ldb, m, n, k, e, splits, d_err,
              static_cast<cudaStream_t>(stream), nullptr);
}
