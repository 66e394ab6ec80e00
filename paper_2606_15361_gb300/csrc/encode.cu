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

#include "snd_internal.h"

namespace snd {
namespace {

constexpr int kHistRowsPerBlock = 2048;

__global__ void __launch_bounds__(256) k_hist(const uint8_t* __restrict__ chunk, int nsamp, int nchan,
                                              uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256][32];
  const int lane = threadIdx.x, wy = threadIdx.y;
  const int tid = wy * 32 + lane;
  for (int i = tid; i < 256 * 32; i += 256) (&h[0][0])[i] = 0;
  __syncthreads();
  const int c = blockIdx.x * 32 + lane;
  const int r0 = blockIdx.y * kHistRowsPerBlock;
  const int r1 = min(nsamp, r0 + kHistRowsPerBlock);
  if (c < nchan) {
    for (int r = r0 + wy; r < r1; r += 8) {
      const uint32_t v = chunk[static_cast<size_t>(r) * nchan + c];
      atomicAdd(&h[v][lane], 1u);
    }
  }
  __syncthreads();
  for (int i = tid; i < 256 * 32; i += 256) {
    const int v = i >> 5, l = i & 31;
    const int cc = blockIdx.x * 32 + l;
    const uint32_t n = h[v][l];
    if (cc < nchan && n) atomicAdd(&hist[static_cast<size_t>(v) * nchan + cc], n);
  }
}

__global__ void k_levels(uint32_t* __restrict__ hist, int nchan, int nsamp, double theta,
                         int32_t* __restrict__ levels) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchan) return;
  // hist is [256][nchan]: consecutive threads read consecutive words
  uint32_t* h = hist + c;
  long long s1 = 0, s2 = 0;
  for (int v = 0; v < 256; ++v) {
    const long long n = h[static_cast<size_t>(v) * nchan];
    s1 += n * v;
    s2 += n * v * v;
  }
  const double nf = static_cast<double>(nsamp);
  const double mu0 = __ddiv_rn(static_cast<double>(s1), nf);
  const double var0 = __dsub_rn(__ddiv_rn(static_cast<double>(s2), nf), __dmul_rn(mu0, mu0));
  const double sig0 = var0 > 0.0 ? __dsqrt_rn(var0) : 0.0;
  const double lo = __dsub_rn(mu0, __dmul_rn(5.0, sig0));
  const double hi = __dadd_rn(mu0, __dmul_rn(5.0, sig0));
  long long s1in = 0, s2in = 0, nlo = 0, nhi = 0;
  for (int v = 0; v < 256; ++v) {
    const long long n = h[static_cast<size_t>(v) * nchan];
    h[static_cast<size_t>(v) * nchan] = 0;  // ready for the next chunk
    if (n == 0) continue;
    const double fv = static_cast<double>(v);
    if (fv < lo) {
      nlo += n;
    } else if (fv > hi) {
      nhi += n;
    } else {
      s1in += n * v;
      s2in += n * v * v;
    }
  }
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
    for (int v = 0; v < 256; ++v) {
      if (static_cast<double>(v) > thr) {
        u = v;
        break;
      }
    }
  }
  levels[c] = u;
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

}  // namespace

cudaError_t launch_encode(const Plan& p, const uint8_t* d_chunk, int nsamp, cudaStream_t s) {
  const DevPtrs& dp = p.dp;
  dim3 hb(32, 8), hg((p.nchan + 31) / 32, (nsamp + kHistRowsPerBlock - 1) / kHistRowsPerBlock);
  k_hist<<<hg, hb, 0, s>>>(d_chunk, nsamp, p.nchan, dp.hist);
  k_levels<<<(p.nchan + 127) / 128, 128, 0, s>>>(dp.hist, p.nchan, nsamp, p.enc_theta, dp.levels);
  const long long t0 = p.T;
  const long long w0 = t0 >> 5;
  const long long w1 = (t0 + nsamp - 1) >> 5;
  const int nwords = static_cast<int>(w1 - w0 + 1);
  dim3 pb(32, 8), pg((p.nchan + 31) / 32, (nwords + 7) / 8);
  k_pack<<<pg, pb, 0, s>>>(d_chunk, nsamp, p.nchan, dp.levels, t0, w0, nwords, dp.ring, p.R);
  p.launches += 3;
  return cudaGetLastError();
}

}  // namespace snd
