// Delta encoder (Methods, "Input encoding"): per-channel two-pass sigma-clip statistics
// and x_c(t) = 1[z_c(t) > theta], written bit-packed into the mirrored spike ring.
//
// Statistics come from a 256-bin histogram per channel of the chunk, evaluated in a fixed
// FP64 order with explicit round-to-nearest intrinsics (no contraction), so the integer
// level u_c (fire iff P >= u_c) is one well-defined decision:
//   mu0 = S1/n, sigma0 = sqrt(max(0, S2/n - mu0^2)), clip to [mu0 -+ 5 sigma0],
//   S1c = (S1in + n_lo lo) + n_hi hi, S2c = (S2in + n_lo lo^2) + n_hi hi^2,
//   mu = S1c/n, sigma = sqrt(max(0, S2c/n - mu^2)), u = min{v in 0..255 : v > mu + theta sigma}.
//
// Ring layout: ring[c][2R] uint32; absolute sample a lives in word a>>5, bit a&31, stored at
// physical word (a>>5) mod R and again at R + that (the mirror lets any window of < R words
// be read contiguously).

#include <cuda_fp16.h>

#include "snd_internal.h"

namespace snd {
namespace {

constexpr int kHistRowsPerBlock = 2048;
constexpr int kHistWarps = 32;  // warps of a histogram CTA, each over every kHistWarps-th row

// CTA (bx, by) of the histogram: 32 channels x kHistRowsPerBlock samples, kHistWarps warps
__device__ __forceinline__ void hist_cta(const uint8_t* __restrict__ chunk, int nsamp, int nchan,
                                         uint32_t* __restrict__ hist, int bx, int by) {
  constexpr int NT = 32 * kHistWarps;
  __shared__ uint32_t h[256][32];
  const int lane = threadIdx.x, wy = threadIdx.y;
  const int tid = wy * 32 + lane;
  for (int i = tid; i < 256 * 32; i += NT) (&h[0][0])[i] = 0;
  __syncthreads();
  const int c = bx * 32 + lane;
  const int r0 = by * kHistRowsPerBlock;
  const int r1 = min(nsamp, r0 + kHistRowsPerBlock);
  if (c < nchan) {
    // eight rows' loads in flight per lane before their counts are added
    int r = r0 + wy;
    for (; r + 7 * kHistWarps < r1; r += 8 * kHistWarps) {
      uint32_t v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = __ldg(chunk + static_cast<size_t>(r + kHistWarps * k) * nchan + c);
#pragma unroll
      for (int k = 0; k < 8; ++k) atomicAdd(&h[v[k]][lane], 1u);
    }
    for (; r < r1; r += kHistWarps) atomicAdd(&h[__ldg(chunk + static_cast<size_t>(r) * nchan + c)][lane], 1u);
  }
  __syncthreads();
  for (int i = tid; i < 256 * 32; i += NT) {
    const int v = i >> 5, l = i & 31;
    const int cc = bx * 32 + l;
    const uint32_t n = h[v][l];
    if (cc < nchan && n) atomicAdd(&hist[static_cast<size_t>(cc) * 256 + v], n);
  }
}

__global__ void __launch_bounds__(32 * kHistWarps) k_hist(const uint8_t* __restrict__ chunk, int nsamp, int nchan,
                                              uint32_t* __restrict__ hist) {
  hist_cta(chunk, nsamp, nchan, hist, blockIdx.x, blockIdx.y);
}

// One warp per channel; lane l holds bins l, l+32, ..., l+224. Integer sums are exact; the
// FP64 steps run on lane 0 in the fixed order above. For integer v, v < lo <=> v < ceil(lo)
// and v > hi <=> v > floor(hi), and the smallest integer above thr is floor(thr) + 1, so the
// clip bounds and the level are exact integer decisions.
// With ztab set (labelled payload), every lane also writes the payload of its 8 values,
// z = (v - mu)/sigma in FP64 for v >= u (0 below), rounded once to FP16 (zmode bit 0) or FP32;
// with zmode bit 1 (the paper's own 0/1 spike payload) z = 1 for v >= u instead.
__device__ __forceinline__ void levels_warp(uint32_t* __restrict__ hist, int nchan, int nsamp, double theta,
                                            int32_t* __restrict__ levels, void* __restrict__ ztab, int zmode,
                                            const int c, const int lane) {
  if (c >= nchan) return;
  uint32_t* h = hist + static_cast<size_t>(c) * 256;
  long long n[8];
  long long s1 = 0, s2 = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int v = lane + 32 * k;
    n[k] = h[v];
    h[v] = 0;  // ready for the next chunk
    s1 += n[k] * v;
    s2 += n[k] * v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, o);
    s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, o);
  }
  const double nf = static_cast<double>(nsamp);
  const double mu0 = __ddiv_rn(static_cast<double>(s1), nf);
  const double var0 = __dsub_rn(__ddiv_rn(static_cast<double>(s2), nf), __dmul_rn(mu0, mu0));
  const double sig0 = var0 > 0.0 ? __dsqrt_rn(var0) : 0.0;
  const double lo = __dsub_rn(mu0, __dmul_rn(5.0, sig0));
  const double hi = __dadd_rn(mu0, __dmul_rn(5.0, sig0));
  const int ilo = static_cast<int>(fmin(fmax(ceil(lo), -1.0), 257.0));    // in range: v >= ilo
  const int ihi = static_cast<int>(fmin(fmax(floor(hi), -1.0), 257.0));   //           v <= ihi
  long long s1in = 0, s2in = 0, nlo = 0, nhi = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int v = lane + 32 * k;
    if (v < ilo) {
      nlo += n[k];
    } else if (v > ihi) {
      nhi += n[k];
    } else {
      s1in += n[k] * v;
      s2in += n[k] * v * v;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1in += __shfl_xor_sync(0xFFFFFFFFu, s1in, o);
    s2in += __shfl_xor_sync(0xFFFFFFFFu, s2in, o);
    nlo += __shfl_xor_sync(0xFFFFFFFFu, nlo, o);
    nhi += __shfl_xor_sync(0xFFFFFFFFu, nhi, o);
  }
  // every lane holds the same reduced sums, so every lane evaluates the same FP64 recipe
  const double s1c = __dadd_rn(__dadd_rn(static_cast<double>(s1in), __dmul_rn(static_cast<double>(nlo), lo)),
                               __dmul_rn(static_cast<double>(nhi), hi));
  const double s2c =
      __dadd_rn(__dadd_rn(static_cast<double>(s2in), __dmul_rn(static_cast<double>(nlo), __dmul_rn(lo, lo))),
                __dmul_rn(static_cast<double>(nhi), __dmul_rn(hi, hi)));
  const double mu = __ddiv_rn(s1c, nf);
  const double var = __dsub_rn(__ddiv_rn(s2c, nf), __dmul_rn(mu, mu));
  const double sig = var > 0.0 ? __dsqrt_rn(var) : 0.0;
  int u = 256;
  if (sig > 0.0) {
    const double thr = __dadd_rn(mu, __dmul_rn(theta, sig));
    if (thr < 0.0) {
      u = 0;
    } else if (thr < 255.0) {
      u = static_cast<int>(floor(thr)) + 1;
    }
  }
  if (lane == 0) levels[c] = u;
  if (ztab) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int v = lane + 32 * k;
      const double z = (v >= u) ? ((zmode & 2) ? 1.0 : __ddiv_rn(__dsub_rn(static_cast<double>(v), mu), sig)) : 0.0;
      if (zmode & 1) {
        static_cast<__half*>(ztab)[static_cast<size_t>(c) * 256 + v] = __double2half(z);
      } else {
        static_cast<float*>(ztab)[static_cast<size_t>(c) * 256 + v] = __double2float_rn(z);
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_levels(uint32_t* __restrict__ hist, int nchan, int nsamp, double theta,
                                                int32_t* __restrict__ levels, void* __restrict__ ztab, int zmode) {
  levels_warp(hist, nchan, nsamp, theta, levels, ztab, zmode, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
              threadIdx.x & 31);
}

// Labelled payload into the ring: zring[c][(t0 + r) mod Rz] = ztab[c][P_c(r)]. A CTA
// transposes 32 channels x 256 samples through shared memory, so both the chunk reads and
// the ring writes are contiguous runs; the 32 payload tables it uses stay in L1.
template <typename ST>
__global__ void __launch_bounds__(256) k_pack_z(const uint8_t* __restrict__ chunk, int nsamp, int nchan,
                                                const ST* __restrict__ ztab, long long t0, ST* __restrict__ zring,
                                                int Rz) {
  __shared__ ST tile[32][257];
  const int lane = threadIdx.x, wy = threadIdx.y;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 256;
  const int c = c0 + lane;
  for (int rl = wy; rl < 256; rl += 8) {
    const int r = r0 + rl;
    if (r < nsamp && c < nchan)
      tile[lane][rl] = __ldg(ztab + static_cast<size_t>(c) * 256 + chunk[static_cast<size_t>(r) * nchan + c]);
  }
  __syncthreads();
  for (int cl = wy; cl < 32; cl += 8) {
    if (c0 + cl >= nchan) break;
    ST* row = zring + static_cast<size_t>(c0 + cl) * Rz;
    for (int rl = lane; rl < 256; rl += 32) {
      const int r = r0 + rl;
      if (r < nsamp) row[static_cast<int>((t0 + r) % Rz)] = tile[cl][rl];
    }
  }
}

// One thread per (channel, ring word). Lanes run over channels, so each row read is a
// contiguous run of bytes. Bits of samples before the chunk keep the ring's old value.
__global__ void __launch_bounds__(256) k_pack(const uint8_t* __restrict__ chunk, int nsamp, int nchan,
                                              const int32_t* __restrict__ levels, long long t0,
                                              long long word0, int nwords, uint32_t* __restrict__ ring,
                                              int R) {
  const int c = blockIdx.x * 32 + threadIdx.x;
  const int q = blockIdx.y * 8 + threadIdx.y;
  if (c >= nchan || q >= nwords) return;
  const long long aw = word0 + q;
  const long long s0 = aw * 32;  // absolute sample of bit 0
  const int u = levels[c];
  uint32_t bits = 0;
#pragma unroll 4
  for (int i = 0; i < 32; ++i) {
    const long long a = s0 + i;
    const long long r = a - t0;
    if (r >= 0 && r < nsamp) {
      const int v = chunk[static_cast<size_t>(r) * nchan + c];
      bits |= static_cast<uint32_t>(v >= u) << i;
    }
  }
  const int phys = static_cast<int>(aw % R);
  uint32_t* row = ring + static_cast<size_t>(c) * 2 * R;
  // keep the bits of samples before the chunk (written by the previous chunk)
  const uint32_t keep = (s0 < t0) ? ((1u << static_cast<int>(t0 - s0)) - 1u) : 0u;
  const uint32_t w = (row[phys] & keep) | bits;
  row[phys] = w;
  row[phys + R] = w;
}

// Warp per (ring word, 32 channels): lane l holds sample 32*aw + l and loads its 32 channel
// bytes with two 16-byte loads; one ballot per channel turns the 32 comparisons into that
// channel's spike word. Requires nchan % 32 == 0 and a 16-byte aligned chunk.
__device__ __forceinline__ void pack32_warp(const uint8_t* __restrict__ chunk, int nsamp, int nchan,
                                            const int32_t* __restrict__ levels, long long t0, long long word0,
                                            int nwords, uint32_t* __restrict__ ring, int R, const int task,
                                            const int lane) {
  const int ncb = nchan >> 5;
  if (task >= nwords * ncb) return;
  const int q = task / ncb, cb = task - q * ncb;
  const int c0 = cb * 32;
  const long long aw = word0 + q;
  const long long r = aw * 32 + lane - t0;
  const bool valid = r >= 0 && r < nsamp;
  uint4 b0 = make_uint4(0, 0, 0, 0), b1 = b0;
  if (valid) {
    const uint4* src = reinterpret_cast<const uint4*>(chunk + static_cast<size_t>(r) * nchan + c0);
    b0 = __ldg(src);
    b1 = __ldg(src + 1);
  }
  const uint32_t wv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
  const int my_u = levels[c0 + lane];
  uint32_t mine = 0;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int u = __shfl_sync(0xFFFFFFFFu, my_u, j);
    const int v = static_cast<int>((wv[j >> 2] >> (8 * (j & 3))) & 0xFFu);
    const uint32_t word = __ballot_sync(0xFFFFFFFFu, valid && v >= u);
    if (lane == j) mine = word;
  }
  const long long s0 = aw * 32;
  const int phys = static_cast<int>(aw % R);
  uint32_t* row = ring + static_cast<size_t>(c0 + lane) * 2 * R;
  uint32_t w = mine;
  // only the chunk's first word keeps bits of samples before the chunk (previous chunk)
  if (s0 < t0) w |= row[phys] & ((1u << static_cast<int>(t0 - s0)) - 1u);
  row[phys] = w;
  row[phys + R] = w;
}

__global__ void __launch_bounds__(256) k_pack32(const uint8_t* __restrict__ chunk, int nsamp, int nchan,
                                                const int32_t* __restrict__ levels, long long t0, long long word0,
                                                int nwords, uint32_t* __restrict__ ring, int R) {
  pack32_warp(chunk, nsamp, nchan, levels, t0, word0, nwords, ring, R, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
              threadIdx.x & 31);
}

// Many plans' encoders, three launches in all: every kernel's CTAs are spread over the beams
// by a prefix of their CTA counts (a CTA finds its beam by binary search).
constexpr int kMaxEncBeams = 64;

struct EncBeam {
  const uint8_t* chunk;
  int nsamp, nchan;
  uint32_t* hist;
  int32_t* levels;
  double theta;
  long long t0, w0;
  int nwords;
  uint32_t* ring;
  int R;
  uint32_t* counters;  // the beam's matched-filter / candidate block counters, cleared here
  int hx;              // histogram CTAs along channels
};

struct EncMulti {
  int nbeams;
  int first_h[kMaxEncBeams], first_l[kMaxEncBeams], first_p[kMaxEncBeams];
  EncBeam beam[kMaxEncBeams];
};

__device__ __forceinline__ int beam_of(const int* first, int n, int i) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(32 * kHistWarps) k_hist_multi(const __grid_constant__ EncMulti m) {
  const int i = static_cast<int>(blockIdx.x);
  const int b = beam_of(m.first_h, m.nbeams, i);
  const EncBeam& e = m.beam[b];
  const int local = i - m.first_h[b];
  hist_cta(e.chunk, e.nsamp, e.nchan, e.hist, local % e.hx, local / e.hx);
}

__global__ void __launch_bounds__(256) k_levels_multi(const __grid_constant__ EncMulti m) {
  const int i = static_cast<int>(blockIdx.x);
  const int b = beam_of(m.first_l, m.nbeams, i);
  const EncBeam& e = m.beam[b];
  const int local = i - m.first_l[b];
  if (local == 0 && threadIdx.x == 0) {
    e.counters[kCntCells] = 0;
    e.counters[kCntRuns] = 0;
    e.counters[kCntBlockCands] = 0;
  }
  levels_warp(e.hist, e.nchan, e.nsamp, e.theta, e.levels, nullptr, 0, local * 8 + (threadIdx.x >> 5),
              threadIdx.x & 31);
}

__global__ void __launch_bounds__(256) k_pack32_multi(const __grid_constant__ EncMulti m) {
  const int i = static_cast<int>(blockIdx.x);
  const int b = beam_of(m.first_p, m.nbeams, i);
  const EncBeam& e = m.beam[b];
  const int local = i - m.first_p[b];
  pack32_warp(e.chunk, e.nsamp, e.nchan, e.levels, e.t0, e.w0, e.nwords, e.ring, e.R,
              local * 8 + (threadIdx.x >> 5), threadIdx.x & 31);
}

}  // namespace

cudaError_t launch_encode(const Plan& p, const uint8_t* d_chunk, int nsamp, cudaStream_t s) {
  const DevPtrs& dp = p.dp;
  dim3 hb(32, kHistWarps), hg((p.nchan + 31) / 32, (nsamp + kHistRowsPerBlock - 1) / kHistRowsPerBlock);
  k_hist<<<hg, hb, 0, s>>>(d_chunk, nsamp, p.nchan, dp.hist);
  const bool z = p.mode == SND_MODE_ZFLOAT;
  k_levels<<<(p.nchan * 32 + 255) / 256, 256, 0, s>>>(dp.hist, p.nchan, nsamp, p.enc_theta, dp.levels,
                                                      z ? dp.ztab : nullptr, p.zgeom.fp16 | (p.zgeom.unit << 1));
  const long long t0 = p.T;
  if (z) {
    dim3 zb(32, 8), zg((p.nchan + 31) / 32, (nsamp + 255) / 256);
    if (p.zgeom.fp16) {
      k_pack_z<__half><<<zg, zb, 0, s>>>(d_chunk, nsamp, p.nchan, static_cast<const __half*>(dp.ztab), t0,
                                         static_cast<__half*>(dp.zring), p.zgeom.Rz);
    } else {
      k_pack_z<float><<<zg, zb, 0, s>>>(d_chunk, nsamp, p.nchan, static_cast<const float*>(dp.ztab), t0,
                                        static_cast<float*>(dp.zring), p.zgeom.Rz);
    }
    p.launches += 3;
    return cudaGetLastError();
  }
  const long long w0 = t0 >> 5;
  const long long w1 = (t0 + nsamp - 1) >> 5;
  const int nwords = static_cast<int>(w1 - w0 + 1);
  if (p.nchan % 32 == 0 && (reinterpret_cast<uintptr_t>(d_chunk) & 15u) == 0) {
    const long long tasks = static_cast<long long>(nwords) * (p.nchan / 32);
    k_pack32<<<static_cast<unsigned>((tasks * 32 + 255) / 256), 256, 0, s>>>(d_chunk, nsamp, p.nchan, dp.levels, t0,
                                                                           w0, nwords, dp.ring, p.R);
  } else {
    dim3 pb(32, 8), pg((p.nchan + 31) / 32, (nwords + 7) / 8);
    k_pack<<<pg, pb, 0, s>>>(d_chunk, nsamp, p.nchan, dp.levels, t0, w0, nwords, dp.ring, p.R);
  }
  p.launches += 3;
  return cudaGetLastError();
}

// Encoders of several plans (bit-ring modes, 32-channel multiples, 16-byte aligned chunks) in
// three launches; each beam's matched-filter and candidate block counters are cleared by its
// first levels CTA. Plans outside those conditions take their own launch_encode (and the
// counters are cleared by a memset).
cudaError_t launch_encode_batch(const Plan* const* plans, const uint8_t* const* chunks, const int32_t* nsamp, int n,
                                cudaStream_t s) {
  EncMulti m{};
  int nh = 0, nl = 0, np = 0;
  const Plan* owner = nullptr;
  auto flush = [&]() -> cudaError_t {
    if (m.nbeams == 0) return cudaSuccess;
    k_hist_multi<<<nh, dim3(32, kHistWarps), 0, s>>>(m);
    k_levels_multi<<<nl, 256, 0, s>>>(m);
    k_pack32_multi<<<np, 256, 0, s>>>(m);
    owner->launches += 3;
    m.nbeams = 0;
    nh = nl = np = 0;
    owner = nullptr;
    return cudaGetLastError();
  };
  for (int i = 0; i < n; ++i) {
    const Plan& p = *plans[i];
    const bool fits = p.mode != SND_MODE_ZFLOAT && p.nchan % 32 == 0 &&
                      (reinterpret_cast<uintptr_t>(chunks[i]) & 15u) == 0;
    if (!fits) {
      cudaError_t e = launch_encode(p, chunks[i], nsamp[i], s);
      if (e == cudaSuccess) e = cudaMemsetAsync(p.dp.counters, 0, sizeof(uint32_t) * (kCntBlockCands + 1), s);
      if (e != cudaSuccess) return e;
      continue;
    }
    EncBeam& e = m.beam[m.nbeams];
    e.chunk = chunks[i];
    e.nsamp = nsamp[i];
    e.nchan = p.nchan;
    e.hist = p.dp.hist;
    e.levels = p.dp.levels;
    e.theta = p.enc_theta;
    e.t0 = p.T;
    e.w0 = p.T >> 5;
    e.nwords = static_cast<int>(((p.T + nsamp[i] - 1) >> 5) - e.w0 + 1);
    e.ring = p.dp.ring;
    e.R = p.R;
    e.counters = p.dp.counters;
    e.hx = (p.nchan + 31) / 32;
    m.first_h[m.nbeams] = nh;
    m.first_l[m.nbeams] = nl;
    m.first_p[m.nbeams] = np;
    nh += e.hx * ((nsamp[i] + kHistRowsPerBlock - 1) / kHistRowsPerBlock);
    nl += (p.nchan * 32 + 255) / 256;
    np += static_cast<int>((static_cast<long long>(e.nwords) * (p.nchan / 32) * 32 + 255) / 256);
    if (!owner) owner = &p;
    if (++m.nbeams == kMaxEncBeams) {
      const cudaError_t err = flush();
      if (err != cudaSuccess) return err;
    }
  }
  return flush();
}

}  // namespace snd
