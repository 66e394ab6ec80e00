"""DM-scaled boxcar matched filter (Methods, "Matched filtering").

Widths at row k: W(d_k) = {1, 2, 4, 8} U {w in {16, 32, ..., 1024} : w <= alpha * tau_sweep(d_k)/dt}.
Per cell: SNR(k, t, W) = (sum_{t'=t}^{t+W-1} y(t') - mu_k W) / (sigma_k sqrt W).

Readings:
* tau_sweep(d)/dt is the continuous sweep in samples from the top channel to the lowest
  channel centre (oracle.delays.sweep_samples); the comparison is alpha*sweep in FP64.
* mu_k, sigma_k are the mean and population std of the row over the block's start times,
  from exact integer sums: mu = S1/n, sigma = sqrt(max(0, S2/n - mu*mu)).
* sigma_min floors sigma in binary mode only (Table S1 lists it for Mode A alone; the
  operating-point sweep says it is not applied to non-binary planes).
* The window is forward, [t, t+W-1]; a cell is scored only when all its windows are
  complete (the streaming block lags by Wmax-1 samples).
* The cell's S/N is the maximum over its widths, ties to the smaller width; the cell is in
  the mask iff that S/N >= Theta ("thresholding at Theta", read as >=). S/N is evaluated in
  FP64 in this order: (float(S) - mu*W) / (sigma*sqrt(W)).
* A row with sigma == 0 has no mask cells (S/N undefined).
* Float mode runs the filter on the root counts (S/N is invariant to the 1/sqrt(N_f) scale).
"""
from __future__ import annotations

import math

import numpy as np

from .delays import sweep_samples

BASE_WIDTHS = (1, 2, 4, 8)
EXT_WIDTHS = (16, 32, 64, 128, 256, 512, 1024)


def row_widths(freqs, dt: float, dm: float, alpha: float) -> list:
    lim = float(alpha) * sweep_samples(freqs, dt, dm)
    return list(BASE_WIDTHS) + [w for w in EXT_WIDTHS if float(w) <= lim]


def max_width(freqs, dt: float, dms, alpha: float) -> int:
    return max(max(row_widths(freqs, dt, d, alpha)) for d in dms)


def row_stats(y_block, sigma_floor=None) -> tuple:
    """(mu, sigma) of the integer samples in ``y_block`` (the block's start times)."""
    y = np.asarray(y_block, dtype=np.int64)
    n = y.size
    s1 = int(y.sum())
    s2 = int((y * y).sum())
    mu = float(s1) / float(n)
    var = float(s2) / float(n) - mu * mu
    sigma = math.sqrt(var) if var > 0.0 else 0.0
    if sigma_floor is not None and sigma < sigma_floor:
        sigma = float(sigma_floor)
    return mu, sigma


def row_mf(y_concat, nb: int, widths, theta: float, sigma_floor=None) -> tuple:
    """Score start times 0..nb-1 of one row. ``y_concat`` holds the row from the first start
    time on and must extend nb + max(widths) - 1 samples. Returns (mask bool[nb],
    snr float64[nb] (NaN where undefined), width int64[nb], mu, sigma)."""
    y = np.asarray(y_concat, dtype=np.int64)
    mask = np.zeros(nb, dtype=bool)
    snr = np.full(nb, np.nan)
    wid = np.zeros(nb, dtype=np.int64)
    if nb == 0:
        return mask, snr, wid, 0.0, 0.0
    if y.size < nb + max(widths) - 1:
        raise ValueError("row too short for its widths")
    mu, sigma = row_stats(y[:nb], sigma_floor)
    if not sigma > 0.0:
        return mask, snr, wid, mu, sigma
    cs = np.concatenate(([0], np.cumsum(y)))
    best = np.full(nb, -np.inf)
    for w in sorted(widths):
        s = (cs[w:w + nb] - cs[0:nb]).astype(np.float64)
        val = (s - mu * float(w)) / (sigma * math.sqrt(float(w)))
        upd = val > best
        best[upd] = val[upd]
        wid[upd] = w
    snr[:] = best
    mask = best >= theta
    return mask, snr, wid, mu, sigma
