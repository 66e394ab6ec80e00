"""Delta encoder with two-pass sigma-clip normalisation (Methods, "Input encoding").

The paper's steps, per channel: (1) mu0, sigma0 of the data; (2) clip P to
[mu0 - 5 sigma0, mu0 + 5 sigma0]; (3) mu, sigma of the clipped values; (4) apply them
to the original data: z = (P - mu)/sigma, x = 1[z > theta].

Readings:
* Statistics are per chunk, over the chunk's own samples; population (1/n) std;
  clipping clamps values, it does not drop them.
* For uint8 input the statistics are sums over the 256-bin histogram, in this fixed
  FP64 order (so that every implementation takes the same integer decision):
    S1 = sum v h[v], S2 = sum v^2 h[v]            (exact integers)
    mu0 = S1/n; sigma0 = sqrt(max(0, S2/n - mu0*mu0))
    lo = mu0 - 5*sigma0; hi = mu0 + 5*sigma0
    in-range bins lo <= v <= hi keep v; n_lo bins below clamp to lo, n_hi above to hi
    S1c = (S1in + n_lo*lo) + n_hi*hi;  S2c = (S2in + n_lo*(lo*lo)) + n_hi*(hi*hi)
    mu = S1c/n; sigma = sqrt(max(0, S2c/n - mu*mu))
* z > theta is taken as P > mu + theta*sigma (sigma > 0), i.e. P >= u where u is the
  smallest integer in [0, 255] above mu + theta*sigma; u = 256 (never fires) when no
  such integer exists or sigma == 0.
"""
from __future__ import annotations

import math

import numpy as np


def channel_stats(values) -> tuple:
    """(mu, sigma, mu0, sigma0) of one channel's uint8 samples, by the recipe above."""
    v = np.asarray(values, dtype=np.uint8)
    n = v.size
    if n == 0:
        return 0.0, 0.0, 0.0, 0.0
    h = np.bincount(v, minlength=256).astype(np.int64)
    vals = np.arange(256, dtype=np.int64)
    s1 = int(np.sum(vals * h))
    s2 = int(np.sum(vals * vals * h))
    nf = float(n)
    mu0 = float(s1) / nf
    var0 = float(s2) / nf - mu0 * mu0
    sigma0 = math.sqrt(var0) if var0 > 0.0 else 0.0
    lo = mu0 - 5.0 * sigma0
    hi = mu0 + 5.0 * sigma0
    s1in = 0
    s2in = 0
    n_lo = 0
    n_hi = 0
    for val in range(256):
        c = int(h[val])
        if c == 0:
            continue
        fv = float(val)
        if fv < lo:
            n_lo += c
        elif fv > hi:
            n_hi += c
        else:
            s1in += val * c
            s2in += val * val * c
    s1c = (float(s1in) + float(n_lo) * lo) + float(n_hi) * hi
    s2c = (float(s2in) + float(n_lo) * (lo * lo)) + float(n_hi) * (hi * hi)
    mu = s1c / nf
    var = s2c / nf - mu * mu
    sigma = math.sqrt(var) if var > 0.0 else 0.0
    return mu, sigma, mu0, sigma0


def level_from_stats(mu: float, sigma: float, theta: float) -> int:
    """Smallest integer u in [0, 255] with u > mu + theta*sigma; 256 if none or sigma == 0."""
    if not sigma > 0.0:
        return 256
    thr = mu + theta * sigma
    for u in range(256):
        if float(u) > thr:
            return u
    return 256


def chunk_levels(chunk, theta: float) -> np.ndarray:
    """int64[nchan] integer levels u_c of a ``uint8[nsamp][nchan]`` chunk."""
    chunk = np.asarray(chunk, dtype=np.uint8)
    out = np.empty(chunk.shape[1], dtype=np.int64)
    for c in range(chunk.shape[1]):
        mu, sigma, _, _ = channel_stats(chunk[:, c])
        out[c] = level_from_stats(mu, sigma, theta)
    return out


def encode_chunk(chunk, theta: float) -> tuple:
    """(x bool[nchan][nsamp], u int64[nchan]) with x_c(t) = 1[P_c(t) > mu_c + theta sigma_c]."""
    chunk = np.asarray(chunk, dtype=np.uint8)
    u = chunk_levels(chunk, theta)
    x = chunk.T.astype(np.int64) >= u[:, None]
    return x, u
