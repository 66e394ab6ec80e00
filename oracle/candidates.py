"""Candidate detection (Methods, "Candidate detection").

Steps: threshold the S/N plane at Theta; binary closing with a 9x9 structuring element;
8-connected component labelling of the closed mask; drop islands with fewer than N_min
pixels; one candidate per island with (DM, t, S/N) from its peak pixel.

Readings (the paper is silent on them):
* Closing = dilation with the square element (outside the block counts as 0) followed by
  erosion with the same element (outside counts as 1), so closing only adds pixels.
* N_min counts pixels of the closed mask.
* The peak is the largest S/N over the island's original-mask pixels, compared in float32;
  ties go to the smaller DM index, then the smaller t. An island with no original-mask
  pixel (not expected for a closing) yields no candidate.
* Candidates are sorted by (t, DM index). Islands are cut at the edges of a streaming
  block (the closing sees only the block).

Parity note: beyond the closing/labelling pins (scipy.ndimage and brute force on tiny
masks) the candidate identity has no printed values to check against.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def closing(mask, size: int = 9) -> np.ndarray:
    m = np.asarray(mask, dtype=bool)
    r = size // 2
    h, w = m.shape
    pad0 = np.zeros((h + 2 * r, w + 2 * r), dtype=bool)
    pad0[r:r + h, r:r + w] = m
    dil = np.zeros_like(m)
    for di in range(-r, r + 1):
        for dj in range(-r, r + 1):
            dil |= pad0[r + di:r + di + h, r + dj:r + dj + w]
    pad1 = np.ones((h + 2 * r, w + 2 * r), dtype=bool)
    pad1[r:r + h, r:r + w] = dil
    ero = np.ones_like(m)
    for di in range(-r, r + 1):
        for dj in range(-r, r + 1):
            ero &= pad1[r + di:r + di + h, r + dj:r + dj + w]
    return ero


def label8(mask) -> tuple:
    """Breadth-first 8-connected labelling. Returns (labels int64 (0 = background), n,
    list of per-label pixel arrays). Labels are numbered in row-major order of their
    first pixel."""
    m = np.asarray(mask, dtype=bool)
    h, w = m.shape
    labels = np.zeros((h, w), dtype=np.int64)
    pixels = []
    n = 0
    for i, j in zip(*np.nonzero(m)):
        if labels[i, j]:
            continue
        n += 1
        labels[i, j] = n
        q = deque([(int(i), int(j))])
        pix = []
        while q:
            a, b = q.popleft()
            pix.append((a, b))
            for da in (-1, 0, 1):
                for db in (-1, 0, 1):
                    aa, bb = a + da, b + db
                    if 0 <= aa < h and 0 <= bb < w and m[aa, bb] and not labels[aa, bb]:
                        labels[aa, bb] = n
                        q.append((aa, bb))
        pixels.append(np.array(pix, dtype=np.int64))
    return labels, n, pixels


def block_candidates(mask, snr, width, dms, t_base: int, size: int = 9, n_min: int = 10) -> list:
    """Candidates of one block: list of (dm_index, dm float32, t, snr float32, width, npix),
    sorted by (t, dm_index). ``mask``/``snr``/``width`` are [ndm][nb] arrays."""
    mask = np.asarray(mask, dtype=bool)
    if mask.size == 0:
        return []
    closed = closing(mask, size)
    _, n, pixels = label8(closed)
    out = []
    snr32 = np.asarray(snr, dtype=np.float64).astype(np.float32)
    for pix in pixels:
        npix = len(pix)
        if npix < n_min:
            continue
        best = None
        for d, t in pix:
            if not mask[d, t]:
                continue
            key = (snr32[d, t], -d, -t)
            if best is None or key > best[0]:
                best = (key, d, t)
        if best is None:
            continue
        _, d, t = best
        out.append((int(d), np.float32(dms[d]), int(t_base + t), np.float32(snr32[d, t]),
                    int(width[d, t]), int(npix)))
    out.sort(key=lambda c: (c[2], c[0]))
    return out
