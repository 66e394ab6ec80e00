// snd_encode_static: the delta encoder of one uint8 chunk into a bit-packed spike raster,
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running where allocation is forbidden (inside a
// host callback or a stream-ordered section that must not synchronise), plugins handed only
// pre-allocated device buffers by their host framework, or processes whose memory budget is
// fixed before they start. They still want the encoder. This entry point therefore takes
// only the caller's input and output buffers: the per-channel histogram and the integer
// levels, which the encoder needs as scratch between its kernels, live in one file-scope
// static device array of fixed size. Every GPU that loads the library keeps that array
// (kStaticScratchWords 32-bit words, 4 MiB + 16 KiB) until the process exits.
//
// The array's name is only a host-side stand-in in host code, so its device address is
// fetched once per device with cudaGetSymbolAddress (with that device current) the first
// time the entry point runs on that device; that first call must therefore come before any
// stream capture. All calls on one device share the array: the histogram is cleared at the
// start of every call, and calls whose work overlaps on the GPU (different streams without
// ordering) race on it and must be serialised by the caller.
//
// Limits: nchan <= kStaticMaxChan (the scratch size) and nsamp <= kStaticMaxSamp (the
// pack kernel's grid height of 65535 rows of 8 words); both are checked before any work is
// enqueued. A launch error is checked after every launch, and the call stops enqueuing at the
// first one; like any CUDA runtime error check this also reports (and clears) a launch error
// that earlier work on the calling thread left pending.

#include <cmath>
#include <mutex>

#include "snd_internal.h"

namespace snd {
namespace {

constexpr int kStaticMaxChan = 4096;  // largest nchan accepted
constexpr int kStaticMaxSamp = 65535 * 8 * 32;  // largest nsamp accepted (pack grid height)
constexpr int kStaticScratchWords = kStaticMaxChan * 256 + kStaticMaxChan;
constexpr int kMaxDevices = 64;
constexpr int kRowsPerBlock = 2048;

// histogram [nchan][256] followed by the levels [nchan]
static __device__ __align__(256) uint32_t g_encoder_scratch[kStaticScratchWords];

std::mutex g_mu;
uint32_t* g_scratch_ptr[kMaxDevices] = {};

__global__ void k_hist_static(const uint8_t* __restrict__ chunk, int nsamp, int nchan, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256][32];
  const int lane = threadIdx.x, wy = threadIdx.y, tid = wy * 32 + lane;
  for (int i = tid; i < 256 * 32; i += 256) (&h[0][0])[i] = 0;
  __syncthreads();
  const int c = blockIdx.x * 32 + lane;
  const int r0 = blockIdx.y * kRowsPerBlock, r1 = min(nsamp, r0 + kRowsPerBlock);
  if (c < nchan)
    for (int r = r0 + wy; r < r1; r += 8) atomicAdd(&h[chunk[static_cast<size_t>(r) * nchan + c]][lane], 1u);
  __syncthreads();
  for (int i = tid; i < 256 * 32; i += 256) {
    const int v = i >> 5, l = i & 31, cc = blockIdx.x * 32 + l;
    if (cc < nchan && h[v][l]) atomicAdd(&hist[static_cast<size_t>(cc) * 256 + v], h[v][l]);
  }
}

// One thread per channel: two-pass sigma clip in the same fixed FP64 order as the streaming
// encoder, then the integer level u (fire iff P >= u; 256 = never).
__global__ void k_levels_static(const uint32_t* __restrict__ hist, int nchan, int nsamp, double theta,
                                int32_t* __restrict__ levels) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchan) return;
  const uint32_t* h = hist + static_cast<size_t>(c) * 256;
  long long s1 = 0, s2 = 0;
  for (int v = 0; v < 256; ++v) {
    s1 += static_cast<long long>(h[v]) * v;
    s2 += static_cast<long long>(h[v]) * v * v;
  }
  const double nf = static_cast<double>(nsamp);
  const double mu0 = __ddiv_rn(static_cast<double>(s1), nf);
  const double var0 = __dsub_rn(__ddiv_rn(static_cast<double>(s2), nf), __dmul_rn(mu0, mu0));
  const double sig0 = var0 > 0.0 ? __dsqrt_rn(var0) : 0.0;
  const double lo = __dsub_rn(mu0, __dmul_rn(5.0, sig0));
  const double hi = __dadd_rn(mu0, __dmul_rn(5.0, sig0));
  long long s1in = 0, s2in = 0, nlo = 0, nhi = 0;
  for (int v = 0; v < 256; ++v) {
    const long long n = h[v];
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
    for (int v = 0; v < 256; ++v)
      if (static_cast<double>(v) > thr) {
        u = v;
        break;
      }
  }
  levels[c] = u;
}

// bits[c][w], bit i = x_c(32 w + i), samples counted from the start of the chunk
__global__ void k_pack_static(const uint8_t* __restrict__ chunk, int nsamp, int nchan, const int32_t* __restrict__ levels,
                              int nwords, uint32_t* __restrict__ bits) {
  const int c = blockIdx.x * 32 + threadIdx.x;
  const int w = blockIdx.y * 8 + threadIdx.y;
  if (c >= nchan || w >= nwords) return;
  const int u = levels[c];
  uint32_t b = 0;
  for (int i = 0; i < 32; ++i) {
    const int r = 32 * w + i;
    if (r < nsamp) b |= static_cast<uint32_t>(chunk[static_cast<size_t>(r) * nchan + c] >= u) << i;
  }
  bits[static_cast<size_t>(c) * nwords + w] = b;
}

// Device address of the scratch array for the current device, looked up once per device.
int scratch_for_current_device(uint32_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SND_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_encoder_scratch) != cudaSuccess || p == nullptr) return SND_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SND_OK;
}

}  // namespace
}  // namespace snd

extern "C" int snd_encode_static(const uint8_t* d_chunk, int32_t nsamp, int32_t nchan, double theta,
                                 uint32_t* d_bits_out, void* stream) {
  using namespace snd;
  if (!d_chunk || !d_bits_out || nsamp < 1 || nchan < 1 || !std::isfinite(theta)) return SND_ERR_ARG;
  if (nchan > kStaticMaxChan || nsamp > kStaticMaxSamp) return SND_ERR_UNSUPPORTED;
  uint32_t* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t* hist = scratch;
  int32_t* levels = reinterpret_cast<int32_t*>(scratch + static_cast<size_t>(kStaticMaxChan) * 256);
  if (cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 256 * static_cast<size_t>(nchan), s) != cudaSuccess)
    return SND_ERR_CUDA;
  dim3 hb(32, 8), hg((nchan + 31) / 32, (nsamp + kRowsPerBlock - 1) / kRowsPerBlock);
  k_hist_static<<<hg, hb, 0, s>>>(d_chunk, nsamp, nchan, hist);
  if (cudaGetLastError() != cudaSuccess) return SND_ERR_CUDA;
  k_levels_static<<<(nchan + 127) / 128, 128, 0, s>>>(hist, nchan, nsamp, theta, levels);
  if (cudaGetLastError() != cudaSuccess) return SND_ERR_CUDA;
  const int nwords = (nsamp + 31) / 32;
  dim3 pb(32, 8), pg((nchan + 31) / 32, (nwords + 7) / 8);
  k_pack_static<<<pg, pb, 0, s>>>(d_chunk, nsamp, nchan, levels, nwords, d_bits_out);
  return cudaGetLastError() == cudaSuccess ? SND_OK : SND_ERR_CUDA;
}
