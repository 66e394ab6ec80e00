"""Float-mode precision study: the labelled z payload and stored partial sums (Methods,
"Input encoding" and "Tree activation modes", Mode C).

Mode C propagates real partial sums. With the paper's 0/1 spike payload every partial sum
is an integer count, so any storage type that holds the integers up to the node's channel
count is exact (FP16 up to 2048). To measure what a narrow storage type costs, the spike
also carries its value: the labelled payload x_c(t) = z_c(t) * 1[P_c(t) >= u_c], with
z_c = (P_c - mu_c)/sigma_c and the encoder's per-chunk clipped statistics and level u_c.

Readings:
* z is evaluated in FP64 from the same (mu, sigma) that give u_c (oracle.encoder recipe),
  then rounded once to the storage type.
* Every node below the root (leaves included) is stored: its value is rounded to the
  storage type (float16 or float32) before its parent reads it. A node adds its children
  in index order in FP32, starting from 0 (a leaf's children are its C channel payloads).
* The root is the FP32 sum of its children, not rounded to the storage type; the plane is
  fp32(root) * fp32(1/sqrt(N_f)), as in Mode C.
* The FP64 reference is the exact definition: sum over all channels of the FP64 payload at
  t + delta_c(d), divided by sqrt(N_f) (tree and direct sum agree in exact arithmetic).
Test infrastructure only; the product path never imports this module.
"""
from __future__ import annotations

import math

import numpy as np

from . import delays as delays_mod
from . import encoder as enc_mod
from . import tree as tree_mod


def payload_table(chunk, theta: float, unit: bool = False):
    """(z64 float64[nchan][256], u int64[nchan]): the FP64 payload of every uint8 value
    per channel (0 below the level u_c), from the chunk's clipped statistics. With
    ``unit`` the payload of a spike is 1: the paper's own 0/1 raster."""
    chunk = np.asarray(chunk, dtype=np.uint8)
    nchan = chunk.shape[1]
    z = np.zeros((nchan, 256), dtype=np.float64)
    u = np.zeros(nchan, dtype=np.int64)
    v = np.arange(256, dtype=np.float64)
    for c in range(nchan):
        mu, sigma, _, _ = enc_mod.channel_stats(chunk[:, c])
        u[c] = enc_mod.level_from_stats(mu, sigma, theta)
        if u[c] < 256:
            z[c, u[c]:] = 1.0 if unit else (v[u[c]:] - mu) / sigma
    return z, u


def payload(chunk, table) -> np.ndarray:
    """x[c][t] = table[c][P_c(t)] for a ``uint8[nsamp][nchan]`` chunk (any table dtype)."""
    chunk = np.asarray(chunk, dtype=np.uint8)
    return table[np.arange(chunk.shape[1])[:, None], chunk.T.astype(np.int64)]


def gather(x, x_t0: int, delays_row, t_start: int, nout: int) -> np.ndarray:
    """a[c][j] = x_c(t_start + j + delta_c), keeping x's dtype."""
    delays_row = np.asarray(delays_row, dtype=np.int64)
    idx = (t_start - x_t0) + delays_row[:, None] + np.arange(nout, dtype=np.int64)[None, :]
    if idx.size and (idx.min() < 0 or idx.max() >= x.shape[1]):
        raise IndexError("payload raster does not cover the requested output times")
    return x[np.arange(x.shape[0])[:, None], idx]


def stored_root(a, levels, store) -> np.ndarray:
    """FP32 root of one DM row from aligned payloads a[c][t] (already in `store`), with every
    non-root node rounded to `store` and children added in order in FP32."""
    f32 = np.float32
    nlev = len(levels)

    def node(children, is_root):
        acc = np.zeros(children[0].shape, dtype=f32)
        for ch in children:
            acc = (acc + ch.astype(f32)).astype(f32)
        return acc if is_root else acc.astype(store)

    vals = [node([a[c] for c in range(lo, hi)], nlev == 1) for lo, hi in levels[0]]
    for li, lev in enumerate(levels[1:], start=1):
        vals = [node(vals[lo:hi], li == nlev - 1) for lo, hi in lev]
    return vals[0].astype(f32)


def plane_scale(nchan: int) -> np.float32:
    return np.float32(1.0 / math.sqrt(float(nchan)))


class ZStream:
    """Streams chunks through the labelled-payload tree; emits, per chunk, the stored-sum
    plane (`store` = np.float16 or np.float32) and the FP64 reference, for the same rows
    and emission rule as the main path (E = max(0, samples consumed - D))."""

    def __init__(self, freqs, dt: float, dms, cluster: int, branching: int, theta: float, store, rows=None,
                 unit: bool = False):
        self.unit = bool(unit)
        self.freqs = np.asarray(freqs, dtype=np.float64)
        self.delays = delays_mod.delay_table(self.freqs, float(dt), np.asarray(dms, dtype=np.float64))
        self.D = int(self.delays.max()) if self.delays.size else 0
        self.nchan = self.freqs.size
        self.levels = tree_mod.tree_levels(self.nchan, cluster, branching)
        self.theta = float(theta)
        self.store = store
        self.rows = list(range(self.delays.shape[0])) if rows is None else list(rows)
        self.T = self.E = 0
        self.x_t0 = 0
        self.xs = np.zeros((self.nchan, 0), dtype=store)
        self.x64 = np.zeros((self.nchan, 0), dtype=np.float64)

    def push(self, chunk) -> dict:
        chunk = np.asarray(chunk, dtype=np.uint8)
        z64, u = payload_table(chunk, self.theta, self.unit)
        self.xs = np.concatenate([self.xs, payload(chunk, z64.astype(self.store))], axis=1)
        self.x64 = np.concatenate([self.x64, payload(chunk, z64)], axis=1)
        e_new = max(0, self.T + chunk.shape[0] - self.D)
        nout = e_new - self.E
        sc = plane_scale(self.nchan)
        y = np.zeros((len(self.rows), nout), dtype=np.float32)
        y64 = np.zeros((len(self.rows), nout), dtype=np.float64)
        for i, d in enumerate(self.rows):
            a = gather(self.xs, self.x_t0, self.delays[d], self.E, nout)
            y[i] = (stored_root(a, self.levels, self.store) * sc).astype(np.float32)
            y64[i] = gather(self.x64, self.x_t0, self.delays[d], self.E, nout).sum(axis=0) / math.sqrt(self.nchan)
        out = dict(e_prev=self.E, e_new=e_new, plane=y, plane64=y64, levels=u)
        self.T += chunk.shape[0]
        self.E = e_new
        keep = self.E - self.x_t0
        if keep > 0:
            self.xs = self.xs[:, keep:]
            self.x64 = self.x64[:, keep:]
            self.x_t0 = self.E
        return out


def error_per_dm(y, y64) -> dict:
    """Per DM trial: max |y - y64| and that over the row's max |y64| (the plane's error
    against FP64 on the scale of the row's signal)."""
    y = np.asarray(y, dtype=np.float64)
    y64 = np.asarray(y64, dtype=np.float64)
    err = np.abs(y - y64).max(axis=1) if y.size else np.zeros(y.shape[0])
    scale = np.abs(y64).max(axis=1) if y.size else np.ones(y.shape[0])
    return dict(max_abs=err, max_rel_to_peak=err / np.where(scale > 0, scale, 1.0))
