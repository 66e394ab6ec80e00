// DM-scaled boxcar matched filter (Methods, "Matched filtering").
//
// One CTA per DM row. The row segment [F_prev, E_new) of the plane ring (block start times
// [F_prev, F_new) plus the Wmax-1 samples their windows reach) is staged in shared memory,
// its exact integer sums give mu and sigma over the block's start times, and an in-place
// exclusive scan turns it into prefix sums so every boxcar is P[t+W] - P[t].
//
// Decision: a cell is in the mask iff max over the row's widths of
//   SNR(W) = (S_W - mu*W) / (sigma*sqrt(W))          (FP64, this operation order)
// reaches Theta. SNR(S) is monotone in the integer S, so thread 0 finds per width the
// smallest integer tau_W with SNR(tau_W) >= Theta by a bounded search around
// mu*W + Theta*sigma*sqrt(W); the per-cell test is then the exact integer compare
// S_W >= tau_W. Cells in the mask get their FP64 S/N maximum (ties -> smaller width)
// rounded to float and are appended to the block's cell list for peak selection.
// Mode A floors sigma at sigma_min; Mode C scores the integer root counts (S/N does not
// change under the 1/sqrt(N_f) scale).

#include <cmath>

#include "snd_internal.h"

namespace snd {
namespace {

struct MfArgs {
  const int32_t* plane;
  int Lp, ndm;
  long long f_prev, e_prev, e_new;
  int nb;  // start times in this block
  const uint16_t* width_mask;
  int binary;
  double theta, sigma_min;
  float out_scale;  // 1/sqrt(N_f) for the caller's float plane, else 0
  uint32_t* mask;
  int mw;
  MfCell* cells;
  int cell_cap;
  uint32_t* counters;
  void* plane_out;
  int nemit;
  int out_u8;       // caller's plane in uint8 (binary / graded roots are 0..255)
};

constexpr int kMfThreads = 256;

__device__ __forceinline__ double snr_of(long long s, double mu_w, double den) {
  return __ddiv_rn(__dsub_rn(static_cast<double>(s), mu_w), den);
}

__global__ void __launch_bounds__(kMfThreads, 3) k_mf(MfArgs a) {
  // smem: the row segment, placed so that every aligned group of four ring columns lands
  // on a 16-byte boundary (one 128-bit store per group), with pads on both sides
  extern __shared__ __align__(16) int32_t smem[];
  __shared__ long long red1[kMfThreads / 32], red2[kMfThreads / 32];
  __shared__ int tau[kNumWidthSlots];
  __shared__ double smu, ssig;
  __shared__ int s_ok;
  __shared__ uint32_t wsum[kMfThreads / 32];
  const int d = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int NWARP = kMfThreads / 32;
  const int len = static_cast<int>(a.e_new - a.f_prev);
  const int c0 = static_cast<int>(a.f_prev % a.Lp);
  const int r0 = c0 & 3;
  int32_t* y = smem + 4 + r0;  // y[i] = ring column c0 + i
  // 1. stage ring columns [f_prev, e_new) of row d with 16-byte loads and stores (Lp % 4 == 0,
  //    so an aligned group of four columns never straddles the ring's wrap point)
  {
    const int32_t* src = a.plane + static_cast<size_t>(d) * a.Lp;
    const int ngroups = (len + r0 + 3) >> 2;
    int4* dst = reinterpret_cast<int4*>(smem + 4);
    for (int k = tid; k < ngroups; k += kMfThreads) {
      int c = c0 - r0 + 4 * k;
      if (c >= a.Lp) c -= a.Lp;
      dst[k] = __ldg(reinterpret_cast<const int4*>(src + c));
    }
  }
  __syncthreads();
  // caller's plane: the newly emitted samples [E_prev, E_new)
  if (a.plane_out) {
    const int first = static_cast<int>(a.e_prev - a.f_prev);
    if (a.out_scale != 0.0f) {
      float* o = static_cast<float*>(a.plane_out) + static_cast<size_t>(d) * a.nemit;
      for (int i = tid; i < a.nemit; i += kMfThreads) o[i] = static_cast<float>(y[first + i]) * a.out_scale;
    } else if (a.out_u8) {
      uint8_t* o = static_cast<uint8_t*>(a.plane_out) + static_cast<size_t>(d) * a.nemit;
      for (int i = tid; i < a.nemit; i += kMfThreads) o[i] = static_cast<uint8_t>(y[first + i]);
    } else {
      int32_t* o = static_cast<int32_t*>(a.plane_out) + static_cast<size_t>(d) * a.nemit;
      for (int i = tid; i < a.nemit; i += kMfThreads) o[i] = y[first + i];
    }
  }
  const int nb = a.nb;
  if (nb <= 0) return;
  __syncthreads();  // the caller's copy has read the raw values before the in-place scan
  // 2. warp-segmented exclusive scan in place (uint32 wrap-around keeps window sums exact),
  //    with the exact integer sums over the block's start times taken on the way
  const int seg = ((len + NWARP * 32 - 1) / (NWARP * 32)) * 32;
  const int lo = min(len, wid * seg), hi = min(len, lo + seg);
  uint32_t carry = 0;
  long long s1 = 0, s2 = 0;
  for (int base = lo; base < hi; base += 32) {
    const int i = base + lane;
    const uint32_t v = (i < hi) ? static_cast<uint32_t>(y[i]) : 0u;
    if (i < nb) {
      const long long vv = static_cast<int32_t>(v);
      s1 += vv;
      s2 += vv * vv;
    }
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += u;
    }
    if (i < hi) y[i] = static_cast<int32_t>(carry + incl - v);
    carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
  }
  if (lane == 0) wsum[wid] = carry;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_down_sync(0xFFFFFFFFu, s1, o);
    s2 += __shfl_down_sync(0xFFFFFFFFu, s2, o);
  }
  if (lane == 0) {
    red1[wid] = s1;
    red2[wid] = s2;
  }
  __syncthreads();
  const uint32_t wm = a.width_mask[d];
  if (wid == 0) {
    // row statistics (FP64, fixed order) and, lane j, the integer threshold of width 2^j
    long long t1 = 0, t2 = 0;
    for (int w = 0; w < NWARP; ++w) {
      t1 += red1[w];
      t2 += red2[w];
    }
    const double n = static_cast<double>(nb);
    const double mu = __ddiv_rn(static_cast<double>(t1), n);
    const double var = __dsub_rn(__ddiv_rn(static_cast<double>(t2), n), __dmul_rn(mu, mu));
    double sig = var > 0.0 ? __dsqrt_rn(var) : 0.0;
    if (a.binary && sig < a.sigma_min) sig = a.sigma_min;
    if (lane == 0) {
      smu = mu;
      ssig = sig;
      s_ok = sig > 0.0;
    }
    if (sig > 0.0 && lane < kNumWidthSlots && ((wm >> lane) & 1)) {
      const double w = static_cast<double>(1 << lane);
      const double mu_w = __dmul_rn(mu, w);
      const double den = __dmul_rn(sig, __dsqrt_rn(w));
      double est = ceil(__dadd_rn(mu_w, __dmul_rn(a.theta, den)));
      if (est < 0.0) est = 0.0;
      if (est > 2147483000.0) est = 2147483000.0;
      long long sv = static_cast<long long>(est);
      int down = 0, up = 0;
      while (sv > 0 && down < 64 && snr_of(sv - 1, mu_w, den) >= a.theta) {
        --sv;
        ++down;
      }
      while (up < 64 && snr_of(sv, mu_w, den) < a.theta) {
        ++sv;
        ++up;
      }
      if (down == 64 || up == 64) atomicOr(&a.counters[kCntStatus], kStatusTauTimeout);
      tau[lane] = static_cast<int>(sv);
    }
  }
  {
    uint32_t off = 0;
    for (int w = 0; w < wid; ++w) off += wsum[w];
    if (off)
      for (int i = lo + lane; i < hi; i += 32) y[i] = static_cast<int32_t>(static_cast<uint32_t>(y[i]) + off);
    if (wid == NWARP - 1 && lane == 0) y[len] = static_cast<int32_t>(off + carry);
  }
  __syncthreads();
  const int nbw = (nb + 31) >> 5;
  uint32_t* mrow = a.mask + static_cast<size_t>(d) * a.mw;
  if (!s_ok) {
    for (int q = tid; q < nbw; q += kMfThreads) mrow[q] = 0;
    return;
  }
  int tw[kNumWidthSlots];
#pragma unroll
  for (int j = 0; j < kNumWidthSlots; ++j) tw[j] = ((wm >> j) & 1) ? tau[j] : 0x7FFFFFFF;
  const double mu = smu, sig = ssig;
  const uint32_t* P = reinterpret_cast<const uint32_t*>(y);
  for (int q = wid; q < nbw; q += NWARP) {
    const int t = q * 32 + lane;
    bool hit = false;
    if (t < nb) {
      const uint32_t p0 = P[t];
#pragma unroll
      for (int j = 0; j < kNumWidthSlots; ++j) {
        if ((wm >> j) & 1) hit |= static_cast<int>(P[t + (1 << j)] - p0) >= tw[j];
      }
    }
    const uint32_t word = __ballot_sync(0xFFFFFFFFu, hit);
    if (lane == 0) mrow[q] = word;
    if (hit) {
      const uint32_t p0 = P[t];
      double best = -1.0e300;
      int bw = 0;
      for (int j = 0; j < kNumWidthSlots; ++j) {
        if (!((wm >> j) & 1)) continue;
        const double w = static_cast<double>(1 << j);
        const long long S = static_cast<int>(P[t + (1 << j)] - p0);
        const double v = snr_of(S, __dmul_rn(mu, w), __dmul_rn(sig, __dsqrt_rn(w)));
        if (v > best) {
          best = v;
          bw = 1 << j;
        }
      }
      const uint32_t idx = atomicAdd(&a.counters[kCntCells], 1u);
      if (idx < static_cast<uint32_t>(a.cell_cap)) {
        MfCell c;
        c.cell = static_cast<uint32_t>(d) * static_cast<uint32_t>(nb) + static_cast<uint32_t>(t);
        c.snr = __double2float_rn(best);
        c.width = bw;
        a.cells[idx] = c;
      } else {
        atomicOr(&a.counters[kCntStatus], kStatusCellOverflow);
      }
    }
  }
}

}  // namespace

cudaError_t launch_mf(const Plan& p, int64_t e_prev, int64_t e_new, int64_t f_prev, int64_t f_new,
                      void* d_plane_out, cudaStream_t s) {
  const int nb = static_cast<int>(f_new - f_prev);
  const int nemit = static_cast<int>(e_new - e_prev);
  if (nb <= 0 && (d_plane_out == nullptr || nemit <= 0)) return cudaSuccess;
  MfArgs a{};
  a.plane = p.dp.plane;
  a.Lp = p.Lp;
  a.ndm = p.ndm;
  a.f_prev = f_prev;
  a.e_prev = e_prev;
  a.e_new = e_new;
  a.nb = nb;
  a.width_mask = p.dp.width_mask;
  a.binary = p.mode == SND_MODE_BINARY;
  a.theta = p.det_theta;
  a.sigma_min = p.sigma_min;
  a.out_scale = (p.mode == SND_MODE_FLOAT) ? static_cast<float>(1.0 / std::sqrt(static_cast<double>(p.nchan))) : 0.0f;
  a.mask = p.dp.mask;
  a.mw = p.mw;
  a.cells = p.dp.cells;
  a.cell_cap = p.cell_cap;
  a.counters = p.dp.counters;
  a.plane_out = nemit > 0 ? d_plane_out : nullptr;
  a.nemit = nemit;
  a.out_u8 = p.plane_u8;
  const int len = static_cast<int>(e_new - f_prev);
  const int smem = (len + 16) * 4;  // front pad (4 + up to 3), prefix total and staging overrun
  cudaError_t e = cudaFuncSetAttribute(k_mf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_mf<<<p.ndm, kMfThreads, smem, s>>>(a);
  p.launches += 1;
  return cudaGetLastError();
}

}  // namespace snd
