// CPU oracle of the Spiking Neural Dedispersion (SND) hot path (arXiv 2606.15361), in plain
// C++17 with OpenMP over trial-DM rows (and over channels in the encoder).
//
// TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's CPU baseline /
// reference arm load this library. It shares no code, header, table or constant generator
// with the CUDA library: it is a second, independent statement of the same definitions as
// the numpy oracle in this package, written for speed of checking (it can run the full
// 1024-channel / 2048-DM stream), not for speed of the method. Every step is the plain
// definition; the only parallelism is over independent trial-DM rows, channels or mask rows.
//
// Readings of the paper (the same as the numpy oracle's):
//  * K_DM = 4.148808e3 MHz^2 s pc^-1 cm^3; the reference channel is the highest frequency;
//    delta = floor(x + 1/2) with x = ((K*d) * (1/f_c^2 - 1/f_ref^2)) / dt in FP64.
//  * Encoder statistics per chunk from the 256-bin histogram in a fixed FP64 order; the level
//    u is the smallest integer above mu + theta*sigma (256 = never fires; sigma = 0 never fires).
//  * Every tree shift is a difference of the globally rounded delays, so channel c is read at
//    t + delta_c(d) and the tree is evaluated per DM at one output time.
//  * Mode A: 1[s >= K_L] at leaves, 1[s >= K_I] above; Mode B: min(s, N) at every node, the
//    root included; Mode C: s (the caller scales the root by 1/sqrt(N_f)).
//  * Matched filter: mean / population std of the block's start times from int64 sums,
//    sigma_min in binary mode only, forward windows, FP64 S/N in the order
//    (S - mu*W) / (sigma*sqrt(W)), max over widths with ties to the smaller width, >= Theta.
//  * Candidates: closing = dilation (outside 0) then erosion (outside 1) with a square element;
//    8-connected labels; islands of >= N_min closed pixels; peak = largest float32 S/N over the
//    island's original-mask pixels, ties to the smaller DM index then the smaller t; sorted by
//    (t, DM index); islands are cut at block edges.
//  * Streaming in the ring-buffer form: E = max(0, T - D), F = max(0, E - (Wmax - 1)).
//
// This file must be compiled without floating-point contraction (-ffp-contract=off).

#include <omp.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <deque>
#include <new>
#include <vector>

namespace {

constexpr double kDm = 4.148808e3;  // MHz^2 s pc^-1 cm^3
constexpr int kBinary = 0, kGraded = 1, kFloat = 2;

int argmax_freq(const double* f, int n) {
  int r = 0;
  for (int c = 1; c < n; ++c)
    if (f[c] > f[r]) r = c;
  return r;
}

int argmin_freq(const double* f, int n) {
  int r = 0;
  for (int c = 1; c < n; ++c)
    if (f[c] < f[r]) r = c;
  return r;
}

// Methods, "Input encoding": two-pass sigma clip of one channel from its histogram.
void channel_stats(const uint8_t* v, int64_t n, int64_t stride, double out[4]) {
  out[0] = out[1] = out[2] = out[3] = 0.0;
  if (n <= 0) return;
  int64_t h[256] = {0};
  for (int64_t i = 0; i < n; ++i) h[v[i * stride]]++;
  int64_t s1 = 0, s2 = 0;
  for (int val = 0; val < 256; ++val) {
    s1 += static_cast<int64_t>(val) * h[val];
    s2 += static_cast<int64_t>(val) * val * h[val];
  }
  const double nf = static_cast<double>(n);
  const double mu0 = static_cast<double>(s1) / nf;
  const double var0 = static_cast<double>(s2) / nf - mu0 * mu0;
  const double sigma0 = var0 > 0.0 ? std::sqrt(var0) : 0.0;
  const double lo = mu0 - 5.0 * sigma0, hi = mu0 + 5.0 * sigma0;
  int64_t s1in = 0, s2in = 0, n_lo = 0, n_hi = 0;
  for (int val = 0; val < 256; ++val) {
    const int64_t c = h[val];
    if (c == 0) continue;
    const double fv = static_cast<double>(val);
    if (fv < lo) {
      n_lo += c;
    } else if (fv > hi) {
      n_hi += c;
    } else {
      s1in += static_cast<int64_t>(val) * c;
      s2in += static_cast<int64_t>(val) * val * c;
    }
  }
  const double s1c = (static_cast<double>(s1in) + static_cast<double>(n_lo) * lo) + static_cast<double>(n_hi) * hi;
  const double s2c =
      (static_cast<double>(s2in) + static_cast<double>(n_lo) * (lo * lo)) + static_cast<double>(n_hi) * (hi * hi);
  const double mu = s1c / nf;
  const double var = s2c / nf - mu * mu;
  out[0] = mu;
  out[1] = var > 0.0 ? std::sqrt(var) : 0.0;
  out[2] = mu0;
  out[3] = sigma0;
}

int level_from_stats(double mu, double sigma, double theta) {
  if (!(sigma > 0.0)) return 256;
  const double thr = mu + theta * sigma;
  for (int u = 0; u < 256; ++u)
    if (static_cast<double>(u) > thr) return u;
  return 256;
}

// One trial DM's tree, evaluated depth first over whole output series: node (lev, idx)
// writes its value v[j] for output times t_start + j, j < nout.
struct TreeEval {
  const uint8_t* x;       // raster x[c][t - x_t0], row length xlen
  int64_t xlen, x_t0;
  const int32_t* delay;   // delta_c(d) of this DM, [nchan]
  int nchan, C, B, mode, KL, KI, cap;
  int64_t t_start;
  int nout;
  std::vector<std::vector<std::pair<int, int>>> levels;  // [lev] -> (lo, hi) child ranges
  std::vector<std::vector<int32_t>> scratch;             // one child buffer per level

  // the mode's rule on a whole node series (threshold k in Mode A)
  void rule(int32_t* __restrict v, int n, int k) const {
    if (mode == kBinary) {
      for (int j = 0; j < n; ++j) v[j] = v[j] >= k ? 1 : 0;
    } else if (mode == kGraded) {
      const int32_t N = cap;
      for (int j = 0; j < n; ++j) v[j] = v[j] < N ? v[j] : N;
    }
  }

  void node(int lev, int idx, int32_t* __restrict v) {
    const int lo = levels[lev][idx].first, hi = levels[lev][idx].second;
    const int n = nout;
    for (int j = 0; j < n; ++j) v[j] = 0;
    if (lev == 0) {
      // leaf: s = sum of the cluster's channels, each read at t + delta_c(d)
      for (int c = lo; c < hi; ++c) {
        const uint8_t* __restrict row = x + static_cast<int64_t>(c) * xlen + (t_start - x_t0) + delay[c];
        for (int j = 0; j < n; ++j) v[j] += row[j];
      }
      rule(v, n, KL);
      return;
    }
    int32_t* __restrict tmp = scratch[lev - 1].data();
    for (int i = lo; i < hi; ++i) {
      node(lev - 1, i, tmp);
      for (int j = 0; j < n; ++j) v[j] += tmp[j];
    }
    rule(v, n, KI);
  }
};

// Methods, "Leaf clusters" / "Tree levels": level 0 = runs of C channels, level l+1 = runs
// of B nodes of level l; the last run of a level may be shorter; one node at the top.
std::vector<std::vector<std::pair<int, int>>> tree_levels(int nchan, int C, int B) {
  std::vector<std::vector<std::pair<int, int>>> lv(1);
  for (int lo = 0; lo < nchan; lo += C) lv[0].push_back({lo, std::min(lo + C, nchan)});
  while (lv.back().size() > 1) {
    const int n = static_cast<int>(lv.back().size());
    std::vector<std::pair<int, int>> up;
    for (int lo = 0; lo < n; lo += B) up.push_back({lo, std::min(lo + B, n)});
    lv.push_back(up);
  }
  return lv;
}

bool raster_covers(int64_t xlen, int64_t x_t0, const int32_t* delay, int nchan, int64_t t_start, int nout) {
  if (nout <= 0) return true;
  for (int c = 0; c < nchan; ++c) {
    const int64_t a = (t_start - x_t0) + delay[c];
    if (a < 0 || a + nout > xlen) return false;
  }
  return true;
}

// Methods, "Matched filtering": one row's block. y holds the row from the block's first start
// time on (at least nb + max width - 1 samples).
void row_mf(const int64_t* y, int nb, const std::vector<int>& widths, double theta, double sigma_floor,
            uint8_t* mask, double* snr, int32_t* wid, double* mu_out, double* sigma_out) {
  for (int t = 0; t < nb; ++t) {
    mask[t] = 0;
    snr[t] = NAN;
    wid[t] = 0;
  }
  if (nb <= 0) return;
  int64_t s1 = 0, s2 = 0;
  for (int t = 0; t < nb; ++t) {
    s1 += y[t];
    s2 += y[t] * y[t];
  }
  const double mu = static_cast<double>(s1) / static_cast<double>(nb);
  const double var = static_cast<double>(s2) / static_cast<double>(nb) - mu * mu;
  double sigma = var > 0.0 ? std::sqrt(var) : 0.0;
  if (sigma_floor >= 0.0 && sigma < sigma_floor) sigma = sigma_floor;
  if (mu_out) *mu_out = mu;
  if (sigma_out) *sigma_out = sigma;
  if (!(sigma > 0.0)) return;
  int wmax = 1;
  for (int w : widths) wmax = std::max(wmax, w);
  std::vector<int64_t> cs(static_cast<size_t>(nb) + wmax, 0);
  for (int t = 0; t < nb + wmax - 1; ++t) cs[t + 1] = cs[t] + y[t];
  std::vector<int> ws(widths);
  std::sort(ws.begin(), ws.end());
  for (int t = 0; t < nb; ++t) {
    double best = -INFINITY;
    int bw = 0;
    for (int w : ws) {
      const double s = static_cast<double>(cs[t + w] - cs[t]);
      const double val = (s - mu * static_cast<double>(w)) / (sigma * std::sqrt(static_cast<double>(w)));
      if (val > best) {
        best = val;
        bw = w;
      }
    }
    snr[t] = best;
    wid[t] = bw;
    mask[t] = best >= theta ? 1 : 0;
  }
}

// Methods, "Candidate detection": closing with a size x size square (dilation with outside 0,
// then erosion with outside 1).
void closing(const uint8_t* m, int h, int w, int size, uint8_t* out) {
  const int r = size / 2;
  std::vector<uint8_t> dil(static_cast<size_t>(h) * w, 0);
#pragma omp parallel for schedule(dynamic, 8)
  for (int i = 0; i < h; ++i)
    for (int j = 0; j < w; ++j) {
      uint8_t v = 0;
      for (int di = -r; di <= r && !v; ++di)
        for (int dj = -r; dj <= r; ++dj) {
          const int a = i + di, b = j + dj;
          if (a >= 0 && a < h && b >= 0 && b < w && m[static_cast<size_t>(a) * w + b]) {
            v = 1;
            break;
          }
        }
      dil[static_cast<size_t>(i) * w + j] = v;
    }
#pragma omp parallel for schedule(dynamic, 8)
  for (int i = 0; i < h; ++i)
    for (int j = 0; j < w; ++j) {
      uint8_t v = 1;
      for (int di = -r; di <= r && v; ++di)
        for (int dj = -r; dj <= r; ++dj) {
          const int a = i + di, b = j + dj;
          const bool inside = a >= 0 && a < h && b >= 0 && b < w;
          if (inside && !dil[static_cast<size_t>(a) * w + b]) {
            v = 0;
            break;
          }
        }
      out[static_cast<size_t>(i) * w + j] = v;
    }
}

struct Cand {
  int32_t dm_index, width, npix, pad;
  float dm, snr;
  int64_t t;
};

// Closing, 8-connected breadth-first labelling (labels in row-major order of their first
// pixel), the N_min filter and the peak of every island; sorted by (t, DM index).
void block_candidates(const uint8_t* mask, const double* snr, const int32_t* width, int h, int w, const double* dms,
                      int64_t t_base, int size, int n_min, std::vector<Cand>& out) {
  if (static_cast<int64_t>(h) * w == 0) return;
  std::vector<uint8_t> closed(static_cast<size_t>(h) * w, 0);
  closing(mask, h, w, size, closed.data());
  std::vector<int32_t> label(static_cast<size_t>(h) * w, 0);
  std::vector<Cand> found;
  int n = 0;
  std::deque<std::pair<int, int>> q;
  for (int i = 0; i < h; ++i)
    for (int j = 0; j < w; ++j) {
      const size_t at = static_cast<size_t>(i) * w + j;
      if (!closed[at] || label[at]) continue;
      ++n;
      label[at] = n;
      q.clear();
      q.push_back({i, j});
      int64_t npix = 0;
      bool have = false;
      float bsnr = 0.0f;
      int bd = 0, bt = 0;
      while (!q.empty()) {
        const auto [a, b] = q.front();
        q.pop_front();
        ++npix;
        const size_t ab = static_cast<size_t>(a) * w + b;
        if (mask[ab]) {
          const float s = static_cast<float>(snr[ab]);
          // key (snr32, -d, -t): larger S/N, then smaller d, then smaller t
          if (!have || s > bsnr || (s == bsnr && (a < bd || (a == bd && b < bt)))) {
            have = true;
            bsnr = s;
            bd = a;
            bt = b;
          }
        }
        for (int da = -1; da <= 1; ++da)
          for (int db = -1; db <= 1; ++db) {
            const int aa = a + da, bb = b + db;
            if (aa < 0 || aa >= h || bb < 0 || bb >= w) continue;
            const size_t k = static_cast<size_t>(aa) * w + bb;
            if (closed[k] && !label[k]) {
              label[k] = n;
              q.push_back({aa, bb});
            }
          }
      }
      if (npix < n_min || !have) continue;
      Cand c{};
      c.dm_index = bd;
      c.dm = static_cast<float>(dms[bd]);
      c.t = t_base + bt;
      c.snr = bsnr;
      c.width = width[static_cast<size_t>(bd) * w + bt];
      c.npix = static_cast<int32_t>(npix);
      found.push_back(c);
    }
  std::stable_sort(found.begin(), found.end(), [](const Cand& a, const Cand& b) {
    return a.t != b.t ? a.t < b.t : a.dm_index < b.dm_index;
  });
  out.insert(out.end(), found.begin(), found.end());
}

std::vector<int> row_widths(const double* freqs, int nchan, double dt, double dm, double alpha) {
  const int r = argmax_freq(freqs, nchan), lo = argmin_freq(freqs, nchan);
  const double inv_lo = 1.0 / (freqs[lo] * freqs[lo]), inv_r = 1.0 / (freqs[r] * freqs[r]);
  const double sweep = ((kDm * dm) * (inv_lo - inv_r)) / dt;
  const double lim = alpha * sweep;
  std::vector<int> w = {1, 2, 4, 8};
  for (int x = 16; x <= 1024; x *= 2)
    if (static_cast<double>(x) <= lim) w.push_back(x);
  return w;
}

struct Config {
  int32_t mode, cluster, branching, k_leaf, k_internal, cap, closing, n_min;
  double enc_theta, det_theta, sigma_min, mf_alpha;
};

// Methods, "Pipeline overview", in the ring-buffer form: the stream keeps the encoded raster
// from the first sample still needed (x_t0 = E) and the last Wmax - 1 plane samples of every
// row that the matched filter has not scored yet.
struct Stream {
  Config cfg{};
  int nchan = 0, ndm = 0;
  double dt = 0;
  std::vector<double> freqs, dms;
  std::vector<int32_t> delays;            // [ndm][nchan]
  std::vector<std::vector<int>> widths;   // per row
  int D = 0, wmax = 1;
  int64_t T = 0, E = 0, F = 0, x_t0 = 0;
  std::vector<std::vector<uint8_t>> x;    // [nchan][samples from x_t0]
  std::vector<std::vector<int64_t>> tail; // [ndm][E - F]
  std::vector<Cand> cands;
  std::vector<int32_t> last_levels;
};

}  // namespace

extern "C" {

int osnd_max_threads() { return omp_get_max_threads(); }
void osnd_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }

// Methods, "Incoherent dedispersion": delta_c(d), [ndm][nchan]. Returns 0, or -1 when a delay
// is negative, not finite or beyond 1e9 samples.
int osnd_delay_table(const double* freqs, int nchan, double dt, const double* dms, int ndm, int32_t* out) {
  const int r = argmax_freq(freqs, nchan);
  const double inv_r = 1.0 / (freqs[r] * freqs[r]);
  for (int d = 0; d < ndm; ++d)
    for (int c = 0; c < nchan; ++c) {
      const double inv_c = 1.0 / (freqs[c] * freqs[c]);
      const double x = ((kDm * dms[d]) * (inv_c - inv_r)) / dt;
      const double v = std::floor(x + 0.5);
      if (!(v >= 0.0) || v > 1.0e9) return -1;
      out[static_cast<size_t>(d) * nchan + c] = static_cast<int32_t>(v);
    }
  return 0;
}

// Methods, "Input encoding": (mu, sigma, mu0, sigma0) of n samples spaced `stride` bytes apart.
void osnd_channel_stats(const uint8_t* v, int64_t n, int64_t stride, double* out4) { channel_stats(v, n, stride, out4); }

// x[c][t] = 1[P_c(t) >= u_c] for a uint8 chunk [nsamp][nchan]; levels[c] = u_c.
void osnd_encode_chunk(const uint8_t* chunk, int nsamp, int nchan, double theta, uint8_t* x, int32_t* levels) {
#pragma omp parallel for schedule(static)
  for (int c = 0; c < nchan; ++c) {
    double st[4];
    channel_stats(chunk + c, nsamp, nchan, st);
    const int u = level_from_stats(st[0], st[1], theta);
    levels[c] = u;
    for (int t = 0; t < nsamp; ++t)
      x[static_cast<size_t>(c) * nsamp + t] = chunk[static_cast<size_t>(t) * nchan + c] >= u ? 1 : 0;
  }
}

// Methods, "The Spiking Neural Dedispersion algorithm": root values of the selected DM rows
// over [t_start, t_start + nout), from the raster x[c][t - x_t0] (row length xlen) and the
// delay table [ndm][nchan]. out is [nrows][nout]. Returns -1 if the raster is too short.
int osnd_snd_rows(const uint8_t* x, int nchan, int64_t xlen, int64_t x_t0, const int32_t* delays, const int32_t* rows,
                  int nrows, int64_t t_start, int nout, int mode, int C, int B, int KL, int KI, int cap,
                  int32_t* out) {
  if (nout <= 0 || nrows <= 0) return 0;
  for (int i = 0; i < nrows; ++i)
    if (!raster_covers(xlen, x_t0, delays + static_cast<size_t>(rows[i]) * nchan, nchan, t_start, nout)) return -1;
  const auto lv = tree_levels(nchan, C, B);
#pragma omp parallel
  {
    TreeEval te;
    te.x = x;
    te.xlen = xlen;
    te.x_t0 = x_t0;
    te.nchan = nchan;
    te.C = C;
    te.B = B;
    te.mode = mode;
    te.KL = KL;
    te.KI = KI;
    te.cap = cap;
    te.t_start = t_start;
    te.nout = nout;
    te.levels = lv;
    te.scratch.assign(lv.size(), std::vector<int32_t>(nout));
#pragma omp for schedule(dynamic, 1)
    for (int i = 0; i < nrows; ++i) {
      te.delay = delays + static_cast<size_t>(rows[i]) * nchan;
      te.node(static_cast<int>(lv.size()) - 1, 0, out + static_cast<size_t>(i) * nout);
    }
  }
  return 0;
}

// Methods, "The neuromorphic dedispersion neuron": direct dedispersion
// y_d(t) = sum_c x_c(t + delta_c(d)) of the selected rows.
int osnd_brute_rows(const uint8_t* x, int nchan, int64_t xlen, int64_t x_t0, const int32_t* delays, const int32_t* rows,
                    int nrows, int64_t t_start, int nout, int32_t* out) {
  if (nout <= 0 || nrows <= 0) return 0;
  for (int i = 0; i < nrows; ++i)
    if (!raster_covers(xlen, x_t0, delays + static_cast<size_t>(rows[i]) * nchan, nchan, t_start, nout)) return -1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < nrows; ++i) {
    const int32_t* dl = delays + static_cast<size_t>(rows[i]) * nchan;
    int32_t* __restrict y = out + static_cast<size_t>(i) * nout;
    const int n = nout;
    for (int j = 0; j < n; ++j) y[j] = 0;
    for (int c = 0; c < nchan; ++c) {
      const uint8_t* __restrict row = x + static_cast<int64_t>(c) * xlen + (t_start - x_t0) + dl[c];
      for (int j = 0; j < n; ++j) y[j] += row[j];
    }
  }
  return 0;
}

// Widths of one row (Methods, "Matched filtering"), written to w_out (at least 11 slots);
// returns how many.
int osnd_row_widths(const double* freqs, int nchan, double dt, double dm, double alpha, int32_t* w_out) {
  const auto w = row_widths(freqs, nchan, dt, dm, alpha);
  for (size_t i = 0; i < w.size(); ++i) w_out[i] = w[i];
  return static_cast<int>(w.size());
}

// One row's matched filter (sigma_floor < 0: none); ms_out = (mu, sigma).
void osnd_row_mf(const int64_t* y, int nb, const int32_t* widths, int nw, double theta, double sigma_floor, uint8_t* mask,
                 double* snr, int32_t* wid, double* ms_out) {
  std::vector<int> ws(widths, widths + nw);
  row_mf(y, nb, ws, theta, sigma_floor, mask, snr, wid, ms_out, ms_out ? ms_out + 1 : nullptr);
}

void osnd_closing(const uint8_t* mask, int h, int w, int size, uint8_t* out) { closing(mask, h, w, size, out); }

// Candidates of one [h][w] block; out holds records of 32 bytes (dm_index, width, npix, pad,
// dm float, snr float, t int64). Returns the number found (all of them are written only when
// it is at most cap).
int osnd_block_candidates(const uint8_t* mask, const double* snr, const int32_t* width, int h, int w, const double* dms,
                          int64_t t_base, int size, int n_min, void* out, int cap) {
  std::vector<Cand> c;
  block_candidates(mask, snr, width, h, w, dms, t_base, size, n_min, c);
  if (static_cast<int>(c.size()) <= cap)
    std::copy(c.begin(), c.end(), static_cast<Cand*>(out));
  return static_cast<int>(c.size());
}

void* osnd_stream_new(const double* freqs, int nchan, double dt, const double* dms, int ndm, const void* cfgp) {
  Stream* s = new (std::nothrow) Stream();
  if (!s) return nullptr;
  s->cfg = *static_cast<const Config*>(cfgp);
  s->nchan = nchan;
  s->ndm = ndm;
  s->dt = dt;
  s->freqs.assign(freqs, freqs + nchan);
  s->dms.assign(dms, dms + ndm);
  s->delays.assign(static_cast<size_t>(ndm) * nchan, 0);
  if (osnd_delay_table(freqs, nchan, dt, dms, ndm, s->delays.data()) != 0) {
    delete s;
    return nullptr;
  }
  for (int32_t v : s->delays) s->D = std::max(s->D, static_cast<int>(v));
  s->widths.resize(ndm);
  for (int d = 0; d < ndm; ++d) {
    s->widths[d] = row_widths(freqs, nchan, dt, dms[d], s->cfg.mf_alpha);
    for (int w : s->widths[d]) s->wmax = std::max(s->wmax, w);
  }
  s->x.assign(nchan, {});
  s->tail.assign(ndm, {});
  return s;
}

void osnd_stream_free(void* sp) { delete static_cast<Stream*>(sp); }

int osnd_stream_max_delay(void* sp) { return static_cast<Stream*>(sp)->D; }
int osnd_stream_max_width(void* sp) { return static_cast<Stream*>(sp)->wmax; }

// Plane samples the next chunk of nsamp samples emits.
int64_t osnd_stream_nemit(void* sp, int nsamp) {
  const Stream& s = *static_cast<Stream*>(sp);
  const int64_t e_new = std::max<int64_t>(0, s.T + nsamp - s.D);
  return e_new - s.E;
}

// Push one chunk uint8[nsamp][nchan] through encoder -> tree -> matched filter -> candidates.
// plane_out (nullable) receives the emitted root values [ndm][nemit] (Mode C: root counts);
// levels_out (nullable) the chunk's encoder levels; info = (e_prev, e_new, f_prev, nb,
// candidates of this block). Returns 0, or -1 on an internal inconsistency.
int osnd_stream_push(void* sp, const uint8_t* chunk, int nsamp, int32_t* plane_out, int32_t* levels_out,
                     int64_t* info) {
  Stream& s = *static_cast<Stream*>(sp);
  const Config& cfg = s.cfg;
  const int nchan = s.nchan, ndm = s.ndm;
  // encoder
  std::vector<uint8_t> xn(static_cast<size_t>(nchan) * nsamp);
  std::vector<int32_t> lev(nchan);
  osnd_encode_chunk(chunk, nsamp, nchan, cfg.enc_theta, xn.data(), lev.data());
  if (levels_out) std::copy(lev.begin(), lev.end(), levels_out);
  for (int c = 0; c < nchan; ++c)
    s.x[c].insert(s.x[c].end(), xn.begin() + static_cast<size_t>(c) * nsamp,
                  xn.begin() + static_cast<size_t>(c + 1) * nsamp);
  // tree over the newly complete output times
  const int64_t e_new = std::max<int64_t>(0, s.T + nsamp - s.D);
  const int nout = static_cast<int>(e_new - s.E);
  std::vector<int32_t> y(static_cast<size_t>(ndm) * std::max(nout, 0));
  if (nout > 0) {
    const int64_t xlen = static_cast<int64_t>(s.x[0].size());
    std::vector<uint8_t> xr(static_cast<size_t>(nchan) * xlen);
    for (int c = 0; c < nchan; ++c) std::copy(s.x[c].begin(), s.x[c].end(), xr.begin() + static_cast<size_t>(c) * xlen);
    std::vector<int32_t> rows(ndm);
    for (int d = 0; d < ndm; ++d) rows[d] = d;
    const int rc = osnd_snd_rows(xr.data(), nchan, xlen, s.x_t0, s.delays.data(), rows.data(), ndm, s.E, nout,
                                 cfg.mode, cfg.cluster, cfg.branching, cfg.k_leaf, cfg.k_internal, cfg.cap, y.data());
    if (rc != 0) return -1;
    if (plane_out) std::copy(y.begin(), y.end(), plane_out);
  }
  // matched filter over the start times whose windows are complete
  const int64_t f_new = std::max<int64_t>(0, e_new - (s.wmax - 1));
  const int nb = static_cast<int>(f_new - s.F);
  const size_t ncand0 = s.cands.size();
  for (int d = 0; d < ndm; ++d)
    s.tail[d].insert(s.tail[d].end(), y.begin() + static_cast<size_t>(d) * std::max(nout, 0),
                     y.begin() + static_cast<size_t>(d + 1) * std::max(nout, 0));
  if (nb > 0) {
    std::vector<uint8_t> mask(static_cast<size_t>(ndm) * nb);
    std::vector<double> snr(static_cast<size_t>(ndm) * nb);
    std::vector<int32_t> wid(static_cast<size_t>(ndm) * nb);
    const double floor = cfg.mode == kBinary ? cfg.sigma_min : -1.0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int d = 0; d < ndm; ++d)
      row_mf(s.tail[d].data(), nb, s.widths[d], cfg.det_theta, floor, mask.data() + static_cast<size_t>(d) * nb,
             snr.data() + static_cast<size_t>(d) * nb, wid.data() + static_cast<size_t>(d) * nb, nullptr, nullptr);
    block_candidates(mask.data(), snr.data(), wid.data(), ndm, nb, s.dms.data(), s.F, cfg.closing, cfg.n_min,
                     s.cands);
    for (int d = 0; d < ndm; ++d) s.tail[d].erase(s.tail[d].begin(), s.tail[d].begin() + nb);
  }
  if (info) {
    info[0] = s.E;
    info[1] = e_new;
    info[2] = s.F;
    info[3] = nb;
    info[4] = static_cast<int64_t>(s.cands.size() - ncand0);
  }
  s.T += nsamp;
  s.E = e_new;
  s.F = f_new;
  const int64_t keep = s.E - s.x_t0;
  if (keep > 0) {
    for (int c = 0; c < nchan; ++c) s.x[c].erase(s.x[c].begin(), s.x[c].begin() + keep);
    s.x_t0 = s.E;
  }
  return 0;
}

// Accumulated candidates (block order, each block sorted by (t, DM index)); returns how many
// there are, writing them only when they fit in cap.
int osnd_stream_candidates(void* sp, void* out, int cap) {
  const Stream& s = *static_cast<Stream*>(sp);
  if (static_cast<int>(s.cands.size()) <= cap) std::copy(s.cands.begin(), s.cands.end(), static_cast<Cand*>(out));
  return static_cast<int>(s.cands.size());
}

}  // extern "C"
