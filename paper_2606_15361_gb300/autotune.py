"""Autotuner for a beam's tree: branching factor B, leaf cluster size C, and the direct tree
kernel's tile shape (warps per CTA, i.e. output words per CTA for its 32-DM tile) and
channel-group size (channels staged per round).

The tile shape and the channel-group size never change a result. B and C change the plane
only where a node rule can bind: in float mode every node holds an exact integer count, so
the plane does not depend on B or C (the tree equals direct dedispersion; Methods, "Tree
activation modes"), and the same holds in graded mode when the cap cannot bind (graded_cap
>= number of channels). There the tuner may also pick (B, C); elsewhere it keeps the caller's.

Every candidate is timed by the per-stage CUDA events (snd_profile) on seeded noise chunks,
in `repeats` separate runs of `steps` chunks. The pick is the candidate with the smallest
median pipeline time per chunk, and it replaces the default (the first candidate: the
caller's B and C, default tile shape) only when its median beats the default's by more than
the spread (max - min over the repeats) of both, so run-to-run noise cannot flip the choice.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import MODE_BINARY, MODE_FLOAT, MODE_GRADED, Plan, options

BRANCHING = (2, 4, 8, 16)
CLUSTER = (2, 3, 4, 5, 6, 7)
WARPS = (8, 4, 2)
ROUND = (128, 64)


def tunable(mode: int, nchan: int, graded_cap: int = 255) -> bool:
    """Whether B and C may be changed without changing the plane."""
    return mode == MODE_FLOAT or (mode == MODE_GRADED and graded_cap >= nchan)


def _time(p, data, fill: int, steps: int, repeats: int):
    for i in range(fill):
        p.execute(data[i % 2])
    tot, tree = [], []
    for r in range(repeats):
        p.profile(True)
        p.profile_read()
        for i in range(steps):
            p.execute(data[(r + i) % 2])
        prof = p.profile_read()
        p.profile(False)
        tot.append(sum(v[0] for v in prof.values()) / steps)
        tree.append(prof["tree"][0] / steps)
    return tot, tree


def autotune(freqs, dt: float, dms, mode: int, chunk: int, opts=None, branching=BRANCHING, cluster=CLUSTER,
             warps=WARPS, rounds=ROUND, warmup: int = 2, steps: int = 3, repeats: int = 3, seed: int = 0,
             device="cuda") -> dict:
    """Returns {"branching", "cluster", "tree_warps", "tree_round", "ms_per_chunk",
    "tree_ms_per_chunk", "spread_ms", "significant", "trials": [...]}. branching[0] must be the
    caller's B; B and C stay the caller's (branching None: untouched) unless the beam is
    tunable."""
    import torch
    freqs = np.asarray(freqs, dtype=np.float64)
    base = opts if opts is not None else options(mode)
    tune_bc = tunable(mode, freqs.size, base.graded_cap)
    # the first candidate is the default: branching[0] (the caller's B), the caller's C, and
    # the default tile shape (first of warps and rounds)
    bs = tuple(branching) if tune_bc else tuple(branching[:1])
    cs = (base.cluster_size,) + (tuple(c for c in cluster if c != base.cluster_size) if tune_bc else ())
    gen = torch.Generator(device=device).manual_seed(seed)
    data = [torch.randn((chunk, freqs.size), generator=gen, device=device).mul_(16).add_(128).round_()
            .clamp_(0, 255).to(torch.uint8) for _ in range(2)]
    trials = []
    for b, c, w, rnd in itertools.product(bs, cs, warps, rounds):
        o = options(mode)
        for f, _ in o._fields_:
            setattr(o, f, getattr(base, f))
        o.cluster_size, o.tree_warps, o.tree_round = c, w, rnd
        o.max_chunk = max(o.max_chunk, chunk)
        try:
            p = Plan(freqs, dt, dms, b, mode, o, device=device)
        except Exception:  # a shape the kernels do not support (e.g. shared memory)
            continue
        st = p.stats()
        fill = warmup + (st.max_delay + chunk - 1) // chunk
        tot, tree = _time(p, data, fill, steps, repeats)
        trials.append(dict(branching=b, cluster=c, tree_warps=w, tree_round=rnd, tree_kernel=int(st.tree_kernel),
                           ms_per_chunk=float(np.median(tot)), tree_ms_per_chunk=float(np.median(tree)),
                           spread_ms=float(max(tot) - min(tot))))
        del p
        torch.cuda.empty_cache()
    if not trials:
        raise RuntimeError("no tree shape of this beam could be planned")
    default = trials[0]
    best = min(trials, key=lambda t: t["ms_per_chunk"])
    margin = max(default["spread_ms"], best["spread_ms"])
    significant = best is not default and best["ms_per_chunk"] < default["ms_per_chunk"] - margin
    pick = best if significant else default
    out = dict(pick, significant=bool(significant), trials=trials)
    if not tune_bc:
        out["branching"] = None
    return out


__all__ = ["autotune", "tunable", "BRANCHING", "CLUSTER", "WARPS", "ROUND", "MODE_BINARY"]
