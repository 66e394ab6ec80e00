"""Multi-rate bands and cross-band candidate merging (Methods, "Multi-rate extension";
Eq. scrunch).

A DM range is split into bands by the scrunch factor S whose scrunched interval does not
exceed the intra-channel smearing at the band's lowest DM:
    S * dt <= tau_smear(d) = K_DM * d * df / f_c^3      (Eq. scrunch, used as printed)
with df the channel bandwidth and f_c the centre frequency. Each band runs its own tree on
a time-scrunched stream with sample interval S*dt. Afterwards, candidates closer than
20 pc cm^-3 in DM and 200 ms in time are merged, keeping the highest S/N.

Readings:
* Every trial DM d runs at S(d) = the largest power of two with S*dt <= tau_smear(d)
  (S >= 1, at most s_max); a band is the set of trial DMs with one S, in grid order.
* df = |f_1 - f_0| (uniform channel spacing), f_c = (max f + min f)/2, all in MHz.
* Scrunching averages S consecutive uint8 samples with round-half-up,
  (sum + S//2) // S, so the band keeps the uint8 encoder (statistics per scrunched chunk).
* A band candidate at scrunched sample t_S has native time t_S * S.
* Merging is single-linkage: candidates joined by any chain of pairs within both windows
  form one cluster; its representative is the largest S/N (float32), ties to the smaller DM
  index, then the smaller time. The merged list is sorted by (t, DM index).
"""
from __future__ import annotations

import numpy as np

from . import delays as delays_mod
from . import stream as stream_mod


def smear_seconds(freqs, dm: float) -> float:
    f = np.asarray(freqs, dtype=np.float64)
    df = abs(float(f[1] - f[0])) if f.size > 1 else 1.0
    fc = 0.5 * (float(f.max()) + float(f.min()))
    return ((delays_mod.K_DM * float(dm)) * df) / (fc * fc * fc)


def scrunch_factor(freqs, dt: float, dm: float, s_max: int = 64) -> int:
    tau = smear_seconds(freqs, dm)
    s = 1
    while s * 2 <= s_max and float(s * 2) * dt <= tau:
        s *= 2
    return s


def bands(freqs, dt: float, dms, s_max: int = 64) -> list:
    """[(S, [global DM indices in grid order])] in increasing S."""
    by = {}
    for i, d in enumerate(dms):
        by.setdefault(scrunch_factor(freqs, dt, d, s_max), []).append(i)
    return [(s, by[s]) for s in sorted(by)]


def scrunch(chunk, s: int) -> np.ndarray:
    """uint8[n][nchan] -> uint8[n/s][nchan]: mean of s consecutive samples, half up."""
    x = np.asarray(chunk, dtype=np.int64)
    n = x.shape[0] // s
    tot = x[: n * s].reshape(n, s, x.shape[1]).sum(axis=1)
    return ((tot + s // 2) // s).astype(np.uint8)


def merge(cands, dms, dt: float, dm_window: float = 20.0, t_window_s: float = 0.2) -> list:
    """Single-linkage merge of candidates (dm_index, dm, t_native, snr, width, npix)."""
    n = len(cands)
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    tw = t_window_s / dt
    for i in range(n):
        for j in range(i + 1, n):
            if abs(float(dms[cands[i][0]]) - float(dms[cands[j][0]])) <= dm_window and \
                    abs(cands[i][2] - cands[j][2]) <= tw:
                a, b = find(i), find(j)
                if a != b:
                    parent[max(a, b)] = min(a, b)
    best = {}
    for i, c in enumerate(cands):
        r = find(i)
        key = (np.float32(c[3]), -c[0], -c[2])
        if r not in best or key > best[r][0]:
            best[r] = (key, c)
    out = [v[1] for v in best.values()]
    out.sort(key=lambda c: (c[2], c[0]))
    return out


class MultiRateStream:
    """Per-band OracleStreams on scrunched chunks; candidates mapped to native time and the
    global DM index."""

    def __init__(self, freqs, dt: float, dms, cfg: stream_mod.Config, s_max: int = 64):
        self.freqs = np.asarray(freqs, dtype=np.float64)
        self.dt = float(dt)
        self.dms = np.asarray(dms, dtype=np.float64)
        self.bands = bands(self.freqs, self.dt, self.dms, s_max)
        self.streams = [stream_mod.OracleStream(self.freqs, s * self.dt, self.dms[idx], cfg)
                        for s, idx in self.bands]
        self.pending = []

    @property
    def s_max(self) -> int:
        return max(s for s, _ in self.bands)

    def push(self, chunk) -> list:
        chunk = np.asarray(chunk, dtype=np.uint8)
        if chunk.shape[0] % self.s_max:
            raise ValueError("chunk length must be a multiple of the largest scrunch factor")
        out = []
        for (s, idx), st in zip(self.bands, self.streams):
            r = st.push(scrunch(chunk, s))
            for c in r["candidates"]:
                out.append((idx[c[0]], np.float32(self.dms[idx[c[0]]]), int(c[2]) * s, c[3], c[4] * s, c[5]))
        self.pending += out
        return out

    def candidates(self) -> list:
        """Merge and return everything found since the last call."""
        got = merge(self.pending, self.dms, self.dt)
        self.pending = []
        return got
