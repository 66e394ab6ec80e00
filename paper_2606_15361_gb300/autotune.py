"""Autotuner for the tree shape of a beam: branching factor B and leaf cluster size C.

In float mode every node holds an exact integer count, so the plane does not depend on B
or C (the tree equals direct dedispersion; Methods, "Tree activation modes"); the same holds
in graded mode when the cap cannot bind (graded_cap >= number of channels). There the tuner
may pick any (B, C): it times each candidate's pipeline on seeded noise chunks with the
per-stage CUDA events (snd_profile) and keeps the fastest. Binary mode's quorum rules
depend on B and C, so a binary beam keeps the caller's values.
"""
from __future__ import annotations

import numpy as np

from . import MODE_BINARY, MODE_FLOAT, MODE_GRADED, Plan, options

BRANCHING = (2, 4, 8, 16)
CLUSTER = (2, 3, 4, 5, 6, 7)


def tunable(mode: int, nchan: int, graded_cap: int = 255) -> bool:
    return mode == MODE_FLOAT or (mode == MODE_GRADED and graded_cap >= nchan)


def autotune(freqs, dt: float, dms, mode: int, chunk: int, opts=None, branching=BRANCHING, cluster=CLUSTER,
             warmup: int = 2, steps: int = 3, seed: int = 0, device="cuda") -> dict:
    """{"branching", "cluster", "ms_per_chunk", "tree_ms_per_chunk", "trials": [...]} for the
    fastest (B, C); untunable beams return the caller's (B, C) untimed."""
    import torch
    freqs = np.asarray(freqs, dtype=np.float64)
    base = opts if opts is not None else options(mode)
    if not tunable(mode, freqs.size, base.graded_cap):
        return dict(branching=None, cluster=base.cluster_size, ms_per_chunk=None, tree_ms_per_chunk=None, trials=[])
    gen = torch.Generator(device=device).manual_seed(seed)
    data = [torch.randn((chunk, freqs.size), generator=gen, device=device).mul_(16).add_(128).round_()
            .clamp_(0, 255).to(torch.uint8) for _ in range(2)]
    trials = []
    for b in branching:
        for c in cluster:
            o = options(mode)
            for f, _ in o._fields_:
                setattr(o, f, getattr(base, f))
            o.cluster_size = c
            o.max_chunk = max(o.max_chunk, chunk)
            try:
                p = Plan(freqs, dt, dms, b, mode, o, device=device)
            except Exception:  # a shape the kernels do not support (e.g. shared memory)
                continue
            d = p.stats().max_delay
            # fill the ring so every timed chunk emits `chunk` samples per row
            for i in range(warmup + (d + chunk - 1) // chunk):
                p.execute(data[i % 2])
            p.profile(True)
            p.profile_read()
            for i in range(steps):
                p.execute(data[i % 2])
            prof = p.profile_read()
            p.profile(False)
            tot = sum(v[0] for v in prof.values()) / steps
            trials.append(dict(branching=b, cluster=c, ms_per_chunk=tot, tree_ms_per_chunk=prof["tree"][0] / steps))
            del p
            torch.cuda.empty_cache()
    best = min(trials, key=lambda t: t["ms_per_chunk"])
    return dict(best, trials=trials)


__all__ = ["autotune", "tunable", "BRANCHING", "CLUSTER", "MODE_BINARY"]
