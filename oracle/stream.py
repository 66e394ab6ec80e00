"""Chunked streaming of the whole hot path (Methods, "Pipeline overview").

The paper overlaps consecutive chunks by delta_max + 1 samples and discards overlap
candidates. Reading: the equivalent ring-buffer form is used. With stream time starting
at 0 and chunk i covering samples [T_i, T_i + n_i):
* plane samples t in [E_{i-1}, E_i) are emitted after chunk i, E_i = max(0, T_i + n_i - D),
  D = max delay, so every emitted sample has its full history;
* the matched filter scores start times [F_{i-1}, F_i), F_i = max(0, E_i - (Wmax - 1)),
  so every boxcar window is complete; row statistics are taken over that block;
* candidate detection runs per matched-filter block.
Encoder statistics are per chunk (oracle.encoder).
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

from . import candidates as cand_mod
from . import delays as delays_mod
from . import encoder as enc_mod
from . import mf as mf_mod
from . import tree as tree_mod

BINARY, GRADED, FLOAT = tree_mod.BINARY, tree_mod.GRADED, tree_mod.FLOAT


@dataclass(frozen=True)
class Config:
    mode: int
    cluster: int = 4
    branching: int = 8
    k_leaf: int = 2
    k_internal: int = 2
    cap: int = 255
    enc_theta: float = 1.5
    det_theta: float = 7.0
    sigma_min: float = 0.20
    mf_alpha: float = 0.1
    closing: int = 9
    n_min: int = 10


def defaults(mode: int, **kw) -> Config:
    """Operating points of Supplementary Table S1 (C = 4 from its tree block)."""
    if mode == BINARY:
        c = Config(mode, k_leaf=2, k_internal=2, enc_theta=1.5, sigma_min=0.20)
    elif mode == GRADED:
        c = Config(mode, k_leaf=0, k_internal=0, cap=255, enc_theta=0.75)
    else:
        c = Config(mode, k_leaf=0, k_internal=0, enc_theta=1.5)
    return replace(c, **kw)


class OracleStream:
    """Feeds chunks through encoder -> SND tree -> matched filter -> candidates."""

    def __init__(self, freqs, dt: float, dms, cfg: Config):
        self.freqs = np.asarray(freqs, dtype=np.float64)
        self.dt = float(dt)
        self.dms = np.asarray(dms, dtype=np.float64)
        self.cfg = cfg
        self.nchan = self.freqs.size
        self.delays = delays_mod.delay_table(self.freqs, self.dt, self.dms)
        self.D = int(self.delays.max()) if self.delays.size else 0
        self.widths = [mf_mod.row_widths(self.freqs, self.dt, d, cfg.mf_alpha) for d in self.dms]
        self.wmax = max(max(w) for w in self.widths)
        self.T = 0
        self.E = 0
        self.F = 0
        self.x = np.zeros((self.nchan, 0), dtype=bool)
        self.x_t0 = 0
        self.tail = np.zeros((self.dms.size, 0), dtype=np.int64)

    def push(self, chunk) -> dict:
        cfg = self.cfg
        chunk = np.asarray(chunk, dtype=np.uint8)
        n = chunk.shape[0]
        x_new, levels = enc_mod.encode_chunk(chunk, cfg.enc_theta)
        self.x = np.concatenate([self.x, x_new], axis=1)
        e_new = max(0, self.T + n - self.D)
        nout = e_new - self.E
        y = tree_mod.snd_rows(self.x, self.x_t0, self.delays, range(self.dms.size), self.E, nout,
                              cfg.mode, cfg.cluster, cfg.branching, cfg.k_leaf, cfg.k_internal,
                              cfg.cap)
        concat = np.concatenate([self.tail, y], axis=1)
        f_new = max(0, e_new - (self.wmax - 1))
        nb = f_new - self.F
        ndm = self.dms.size
        mask = np.zeros((ndm, nb), dtype=bool)
        snr = np.full((ndm, nb), np.nan)
        wid = np.zeros((ndm, nb), dtype=np.int64)
        floor = cfg.sigma_min if cfg.mode == BINARY else None
        if nb > 0:
            for d in range(ndm):
                m, s, w, _, _ = mf_mod.row_mf(concat[d], nb, self.widths[d], cfg.det_theta, floor)
                mask[d], snr[d], wid[d] = m, s, w
            cands = cand_mod.block_candidates(mask, snr, wid, self.dms, self.F, cfg.closing,
                                              cfg.n_min)
        else:
            cands = []
        out = dict(levels=levels, e_prev=self.E, e_new=e_new, plane=y, f_prev=self.F, nb=nb,
                   mask=mask, snr=snr, width=wid, candidates=cands)
        if cfg.mode == FLOAT:
            out["plane_float"] = tree_mod.float_scale(y, self.nchan)
        self.tail = concat[:, nb:]
        self.T += n
        self.E = e_new
        self.F = f_new
        keep = self.E - self.x_t0
        if keep > 0:
            self.x = self.x[:, keep:]
            self.x_t0 = self.E
        return out
