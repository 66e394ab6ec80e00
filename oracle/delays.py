"""Dispersion delays (Methods, "Incoherent dedispersion").

The paper gives Delta t_ij = K_DM * DM * (f_i^-2 - f_j^-2) with K_DM ~ 4.149e6 MHz^2 ms,
and the integer delay delta_c(d) = round(Delta t_{c,ref}(d) / Delta t).

Readings (the paper leaves them open):
* K_DM = 4.148808e3 MHz^2 s pc^-1 cm^3 (same constant to four digits).
* The reference channel is the highest-frequency channel, so delta >= 0 and the
  output time is the arrival time at the top of the band.
* Rounding is half-up, floor(x + 1/2), in FP64, with x evaluated in this exact
  order: inv2_c = 1/(f_c*f_c); x = ((K_DM*d) * (inv2_c - inv2_ref)) / dt.
"""
from __future__ import annotations

import numpy as np

K_DM = 4.148808e3


def reference_channel(freqs) -> int:
    """Index of the highest channel frequency (first one if tied)."""
    return int(np.argmax(np.asarray(freqs, dtype=np.float64)))


def _inv2(freqs) -> np.ndarray:
    f = np.asarray(freqs, dtype=np.float64)
    return 1.0 / (f * f)


def delay_table(freqs, dt: float, dms) -> np.ndarray:
    """int64[ndm][nchan]: delta_c(d) = floor(K*d*(f_c^-2 - f_ref^-2)/dt + 1/2)."""
    inv2 = _inv2(freqs)
    r = reference_channel(freqs)
    diff = inv2 - inv2[r]
    d = np.asarray(dms, dtype=np.float64)
    x = ((K_DM * d)[:, None] * diff[None, :]) / float(dt)
    return np.floor(x + 0.5).astype(np.int64)


def sweep_samples(freqs, dt: float, dm: float) -> float:
    """Continuous dispersive sweep across the band, in samples, from the reference
    (highest) channel to the lowest channel centre: K*d*(f_min^-2 - f_ref^-2)/dt."""
    inv2 = _inv2(freqs)
    r = reference_channel(freqs)
    lo = int(np.argmin(np.asarray(freqs, dtype=np.float64)))
    return ((K_DM * float(dm)) * (inv2[lo] - inv2[r])) / float(dt)
