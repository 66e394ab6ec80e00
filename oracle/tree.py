"""SND dedispersion tree and direct dedispersion (Methods, "The neuromorphic
dedispersion neuron" and "The Spiking Neural Dedispersion algorithm").

Direct dedispersion: y_d(t) = sum_c x_c(t + delta_c(d)).

SND, per trial DM d and output time t, with a_c = x_c(t + delta_c(d)):
* leaves are contiguous clusters of C channels (index order; the last may be shorter):
  s = sum_{c in leaf} a_c;
* each higher level combines contiguous runs of B nodes of the level below (the last
  run may be shorter) until one node (the root) remains: s = sum of child values;
* Mode A (binary): v = 1[s >= K_L] at leaves, 1[s >= K_I] above ("meets or exceeds");
  Mode B (graded): v = min(s, N) at every node, root included;
  Mode C (float): v = s; the root is divided by sqrt(N_f).

Reading of the per-level delays: every inter-node shift is a difference of the globally
rounded per-channel delays, so the shifts telescope and every channel is read at exactly
t + delta_c(d). The tree is therefore evaluated per DM without deduplication here: node
sharing between trial DMs (unique patterns) changes cost, never values. With these
delays the DM-time plane does not depend on B in float mode, nor in graded mode while no
non-root node exceeds N (the paper's B-invariance statement).
"""
from __future__ import annotations

import numpy as np

BINARY, GRADED, FLOAT = 0, 1, 2


def tree_levels(nchan: int, cluster: int, branching: int) -> list:
    """Level 0: list of (lo, hi) channel ranges; level l >= 1: list of (lo, hi) ranges of
    node indices of level l-1. The last level has exactly one node."""
    if nchan < 1 or cluster < 1 or branching < 2:
        raise ValueError("need nchan >= 1, cluster >= 1, branching >= 2")
    levels = [[(lo, min(lo + cluster, nchan)) for lo in range(0, nchan, cluster)]]
    while len(levels[-1]) > 1:
        n = len(levels[-1])
        levels.append([(lo, min(lo + branching, n)) for lo in range(0, n, branching)])
    return levels


def _rule(s: np.ndarray, mode: int, k: int, cap: int) -> np.ndarray:
    if mode == BINARY:
        return (s >= k).astype(np.int64)
    if mode == GRADED:
        return np.minimum(s, cap)
    return s


def gather(x, x_t0: int, delays_row, t_start: int, nout: int) -> np.ndarray:
    """a[c][j] = x_c(t_start + j + delta_c), from a raster x[c][t - x_t0]."""
    delays_row = np.asarray(delays_row, dtype=np.int64)
    idx = (t_start - x_t0) + delays_row[:, None] + np.arange(nout, dtype=np.int64)[None, :]
    if idx.size and (idx.min() < 0 or idx.max() >= x.shape[1]):
        raise IndexError("raster does not cover the requested output times")
    return x[np.arange(x.shape[0])[:, None], idx].astype(np.int64)


def snd_root(a: np.ndarray, levels, mode: int, k_leaf: int, k_internal: int, cap: int) -> np.ndarray:
    """Root value per output time for one DM, from the aligned inputs a[c][t]."""
    vals = [_rule(a[lo:hi].sum(axis=0), mode, k_leaf, cap) for lo, hi in levels[0]]
    for lev in levels[1:]:
        vals = [_rule(np.sum(vals[lo:hi], axis=0), mode, k_internal, cap) for lo, hi in lev]
    return vals[0]


def snd_rows(x, x_t0: int, delays, rows, t_start: int, nout: int, mode: int, cluster: int,
             branching: int, k_leaf: int = 0, k_internal: int = 0, cap: int = 255) -> np.ndarray:
    """int64[len(rows)][nout]: SND root values (float mode: root counts before the
    1/sqrt(N_f) scaling) for the selected DM rows over [t_start, t_start + nout)."""
    levels = tree_levels(x.shape[0], cluster, branching)
    out = np.zeros((len(rows), nout), dtype=np.int64)
    for i, d in enumerate(rows):
        a = gather(x, x_t0, delays[d], t_start, nout)
        out[i] = snd_root(a, levels, mode, k_leaf, k_internal, cap)
    return out


def brute_rows(x, x_t0: int, delays, rows, t_start: int, nout: int) -> np.ndarray:
    """int64[len(rows)][nout]: direct dedispersion y_d(t) = sum_c x_c(t + delta_c(d))."""
    out = np.zeros((len(rows), nout), dtype=np.int64)
    for i, d in enumerate(rows):
        out[i] = gather(x, x_t0, delays[d], t_start, nout).sum(axis=0)
    return out


def float_scale(counts, nchan: int) -> np.ndarray:
    """Mode C root normalisation: y = s / sqrt(N_f), in FP64."""
    return np.asarray(counts, dtype=np.float64) / np.sqrt(float(nchan))


def level_fire_counts(x, x_t0: int, delays, rows, t_start: int, nout: int, mode: int, cluster: int,
                      branching: int, k_leaf: int = 0, k_internal: int = 0, cap: int = 255) -> list:
    """Per tree level (0 = leaves), the number of (node, DM row, output time) with a nonzero
    node value over the selected rows and times: the per-level fire counts behind the
    per-level mean fire rates of the paper's dynamic-power model (Supplementary Table S2)."""
    levels = tree_levels(x.shape[0], cluster, branching)
    counts = [0] * len(levels)
    for d in rows:
        a = gather(x, x_t0, delays[d], t_start, nout)
        vals = [_rule(a[lo:hi].sum(axis=0), mode, k_leaf, cap) for lo, hi in levels[0]]
        counts[0] += int(sum(int((v != 0).sum()) for v in vals))
        for li, lev in enumerate(levels[1:], start=1):
            vals = [_rule(np.sum(vals[lo:hi], axis=0), mode, k_internal, cap) for lo, hi in lev]
            counts[li] += int(sum(int((v != 0).sum()) for v in vals))
    return counts
