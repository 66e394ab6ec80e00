"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module draws inputs only. It holds none of the SND arithmetic: no delay
table, no encoder, no tree, no matched filter. Bursts are placed with the
continuous cold-plasma sweep of the signal model (a property of the simulated
sky, not of the search), evaluated in seconds and never rounded to samples.

Filterbank layout is SIGPROC order: ``uint8[nsamp][nchan]`` (time-major).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Dispersion constant of the simulated signal, MHz^2 s pc^-1 cm^3.
K_SKY = 4.148808e3


def channel_freqs(nchan: int, f_top: float = 416.0, bandwidth: float = 16.0) -> np.ndarray:
    """Channel-centre frequencies in MHz, channel 0 highest (Northern Cross band 400-416 MHz)."""
    c = np.arange(nchan, dtype=np.float64)
    return f_top - (c + 0.5) * (bandwidth / nchan)


def dm_grid(ndm: int, dm_max: float, dm_min: float = 0.0) -> np.ndarray:
    """Uniform trial-DM grid (pc cm^-3), row 0 = dm_min."""
    return np.linspace(dm_min, dm_max, ndm, dtype=np.float64)


@dataclass(frozen=True)
class Burst:
    t0: float          # arrival time at the top of the band, in samples (absolute stream time)
    dm: float          # pc cm^-3
    fwhm: float        # samples
    snr: float         # ideal matched-filter S/N over all channels


def draw_bursts(seed: int, n: int, *, dm_range, fwhm_range, snr_range, t_range,
                log_fwhm: bool = False, log_snr: bool = False,
                min_sep: float = 0.0) -> list[Burst]:
    """Draw ``n`` bursts. ``t_range`` bounds t0 (samples); bursts closer than ``min_sep``
    samples to an earlier one are redrawn (bounded number of attempts)."""
    rng = np.random.default_rng([seed, 0xB0B5])
    out: list[Burst] = []
    attempts = 0
    while len(out) < n and attempts < 100 * max(n, 1):
        attempts += 1
        t0 = rng.uniform(*t_range)
        if any(abs(t0 - b.t0) < min_sep for b in out):
            continue
        dm = rng.uniform(*dm_range)
        if log_fwhm:
            fwhm = float(np.exp(rng.uniform(np.log(fwhm_range[0]), np.log(fwhm_range[1]))))
        else:
            fwhm = rng.uniform(*fwhm_range)
        if log_snr:
            snr = float(np.exp(rng.uniform(np.log(snr_range[0]), np.log(snr_range[1]))))
        else:
            snr = rng.uniform(*snr_range)
        out.append(Burst(float(t0), float(dm), float(fwhm), float(snr)))
    out.sort(key=lambda b: b.t0)
    return out


def _noise(seed: int, chunk_index: int, nsamp: int, nchan: int, mean: float, sigma: float) -> np.ndarray:
    rng = np.random.default_rng([seed, chunk_index])
    x = rng.standard_normal((nsamp, nchan), dtype=np.float32)
    x *= np.float32(sigma)
    x += np.float32(mean)
    return x


def filterbank_chunk(seed: int, chunk_index: int, t_start: int, nsamp: int, freqs: np.ndarray,
                     dt: float, bursts=(), mean: float = 128.0, sigma: float = 16.0) -> np.ndarray:
    """One chunk ``uint8[nsamp][nchan]`` of noise ``rint(N(mean, sigma))`` clipped to 0..255,
    covering absolute samples ``[t_start, t_start + nsamp)``, with bursts added before rounding.

    A burst is a Gaussian in time in every channel, centred at ``t0 + sweep_c`` where
    ``sweep_c = K DM (f_c^-2 - f_top^-2) / dt`` (continuous samples), with per-channel
    amplitude ``a*sigma`` and ``a = snr / sqrt(nchan * sum(g^2))`` so that the ideal
    matched S/N over all channels equals ``snr``.
    """
    freqs = np.asarray(freqs, dtype=np.float64)
    nchan = freqs.size
    x = _noise(seed, chunk_index, nsamp, nchan, mean, sigma)
    f_top = freqs.max()
    t_abs = np.arange(t_start, t_start + nsamp, dtype=np.float64)
    for b in bursts:
        sw = K_SKY * b.dm * (freqs ** -2 - f_top ** -2) / dt   # samples, per channel
        half = 4.0 * b.fwhm + 2.0
        lo = b.t0 + sw.min() - half
        hi = b.t0 + sw.max() + half
        if hi < t_start or lo >= t_start + nsamp:
            continue
        s2 = b.fwhm / (2.0 * np.sqrt(2.0 * np.log(2.0)))
        gk = np.arange(-int(np.ceil(half)), int(np.ceil(half)) + 1, dtype=np.float64)
        norm = np.sqrt(np.sum(np.exp(-0.5 * (gk / s2) ** 2) ** 2))
        amp = b.snr / (np.sqrt(nchan) * norm) * sigma
        for c in range(nchan):
            centre = b.t0 + sw[c]
            i0 = max(int(np.floor(centre - half)) - t_start, 0)
            i1 = min(int(np.ceil(centre + half)) + 1 - t_start, nsamp)
            if i1 <= i0:
                continue
            g = np.exp(-0.5 * ((t_abs[i0:i1] - centre) / s2) ** 2)
            x[i0:i1, c] += (amp * g).astype(np.float32)
    np.rint(x, out=x)
    np.clip(x, 0.0, 255.0, out=x)
    return x.astype(np.uint8)


def bernoulli_raster(seed: int, nchan: int, nsamp: int, p: float) -> np.ndarray:
    """Independent Bernoulli(p) spikes, ``bool[nchan][nsamp]`` (for tree statistics tests)."""
    rng = np.random.default_rng([seed, 0x5EED])
    return rng.random((nchan, nsamp)) < p


# ---------------------------------------------------------------------------
# Named workloads (Northern Cross shapes)
# ---------------------------------------------------------------------------

NC_DT = 1.38e-4  # s


@dataclass(frozen=True)
class Workload:
    name: str
    seed: int
    nchan: int
    ndm: int
    dm_max: float
    chunk: int
    nchunks: int
    branching: int
    nbursts: int

    @property
    def nsamp(self) -> int:
        return self.chunk * self.nchunks

    def freqs(self) -> np.ndarray:
        return channel_freqs(self.nchan)

    def dms(self) -> np.ndarray:
        return dm_grid(self.ndm, self.dm_max)

    def sweep_max(self) -> float:
        f = self.freqs()
        return K_SKY * self.dm_max * (f.min() ** -2 - f.max() ** -2) / NC_DT

    def bursts(self) -> list[Burst]:
        sw = self.sweep_max()
        if self.name.startswith("nc64"):
            return draw_bursts(self.seed, self.nbursts, dm_range=(10.0, 90.0),
                               fwhm_range=(1e-3 / NC_DT, 1e-3 / NC_DT), snr_range=(8.0, 20.0),
                               t_range=(sw + 200.0, self.nsamp - 200.0), min_sep=400.0)
        if self.name.startswith("nc4096"):
            # a short stream: bursts arrive (at the top of the band) within the plane range
            # the stream emits, [0, nsamp - sweep), away from its ends
            t_end = self.nsamp - sw
            return draw_bursts(self.seed, self.nbursts, dm_range=(20.0, self.dm_max - 20.0),
                               fwhm_range=(1.0, 10e-3 / NC_DT), snr_range=(6.0, 50.0),
                               t_range=(1500.0, t_end - 1500.0), log_fwhm=True, log_snr=True,
                               min_sep=0.05 / NC_DT)
        return draw_bursts(self.seed, self.nbursts, dm_range=(20.0, min(1980.0, self.dm_max)),
                           fwhm_range=(1.0, 10e-3 / NC_DT), snr_range=(6.0, 50.0),
                           t_range=(sw + 200.0, self.nsamp - 200.0), log_fwhm=True, log_snr=True,
                           min_sep=0.05 / NC_DT)

    def chunk_data(self, i: int, bursts=None) -> np.ndarray:
        b = self.bursts() if bursts is None else bursts
        return filterbank_chunk(self.seed, i, i * self.chunk, self.chunk, self.freqs(), NC_DT, b)


# 64 channels 400-416 MHz, 128 DMs over 0-100, 16384 samples, B=2, 3 bursts.
NC64 = Workload("nc64_128dm", seed=1, nchan=64, ndm=128, dm_max=100.0, chunk=16384, nchunks=1,
                branching=2, nbursts=3)
# Full Northern Cross beam: 1024 channels, 2048 DMs over 0-2000, 2^18 samples in 16 chunks.
NC1024 = Workload("nc1024_2048dm", seed=2, nchan=1024, ndm=2048, dm_max=2000.0, chunk=16384,
                  nchunks=16, branching=8, nbursts=200)
# Stress-scale beam: 4096 channels 400-416 MHz, 8192 DMs over 0-3000, 1 s chunks of 7246
# samples (eight of them: the stream emits plane samples from the sixth chunk on), B = 4.
NC4096 = Workload("nc4096_8192dm", seed=500, nchan=4096, ndm=8192, dm_max=3000.0, chunk=7246,
                  nchunks=8, branching=4, nbursts=12)
