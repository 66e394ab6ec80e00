"""Learned candidate sifter: DM-time snippet extraction and a small CNN classifier, forward
and backward in FP64 (test infrastructure only; the product path never imports this).

The paper leaves a learned classifier to future work ("Discussion"). Readings, shared with
the GPU implementation:
* Snippet: 64 trial-DM rows x 256 samples of the float plane centred on a candidate
  (rows dm_index - 32 .. + 31, samples t - 128 .. t + 127). Cells outside the plane are
  missing. The snippet is standardised with the mean and population std of its present
  cells (std 0 -> 1); missing cells are 0 after standardisation.
* Network (input 1 x 64 x 256):
    conv1 1->16, conv2 16->32, conv3 32->64: 3x3, stride 1, zero padding 1, bias, ReLU,
      each followed by 2x2 max pooling (stride 2; ties go to the first of (0,0), (0,1),
      (1,0), (1,1) in row-major order);
    fc1 64*8*32 -> 128 with bias and ReLU (features flattened channel-major, then row,
      then column); fc2 128 -> 1 with bias: the logit.
  Loss: mean binary cross-entropy on the logit, log(1 + e^z) - y z.
* Parameters live in one flat vector in this order: W1[16][1][3][3], b1, W2[32][16][3][3],
  b2, W3[64][32][3][3], b3, Wf1[128][16384], bf1, Wf2[1][128], bf2.
* `act` (optional) rounds each post-ReLU convolution output before pooling, so that the
  pooling decisions (an argmax) can be taken in the precision an implementation stores its
  activations in; None keeps FP64 throughout.
"""
from __future__ import annotations

import numpy as np

H, W = 64, 256
CONV = ((1, 16, 64, 256), (16, 32, 32, 128), (32, 64, 16, 64))  # (cin, cout, h, w) of each conv input
FEAT = 64 * 8 * 32
HID = 128


def param_shapes():
    shapes = []
    for cin, cout, _, _ in CONV:
        shapes += [(cout, cin, 3, 3), (cout,)]
    shapes += [(HID, FEAT), (HID,), (1, HID), (1,)]
    return shapes


def num_params() -> int:
    return int(sum(np.prod(s) for s in param_shapes()))


def unpack(theta):
    out, o = [], 0
    for s in param_shapes():
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def snippet(plane, dm_index: int, t: int) -> np.ndarray:
    """float64[64][256] standardised snippet of a float plane [ndm][ncols] around (dm_index, t)."""
    plane = np.asarray(plane, dtype=np.float64)
    ndm, ncols = plane.shape
    rows = np.arange(dm_index - 32, dm_index + 32)
    cols = np.arange(t - 128, t + 128)
    rv = (rows >= 0) & (rows < ndm)
    cv = (cols >= 0) & (cols < ncols)
    present = rv[:, None] & cv[None, :]
    vals = np.zeros((H, W))
    vals[np.ix_(rv, cv)] = plane[np.ix_(rows[rv], cols[cv])]
    n = int(present.sum())
    if n == 0:
        return np.zeros((H, W))
    mu = vals[present].sum() / n
    var = ((vals[present] - mu) ** 2).sum() / n
    sd = np.sqrt(var) if var > 0 else 1.0
    return np.where(present, (vals - mu) / sd, 0.0)


def conv3x3(x, w, b):
    """x[n][cin][h][w], w[cout][cin][3][3] -> y[n][cout][h][w]: sum over cin, dy, dx of
    w[o][i][dy][dx] * x[i][r + dy - 1][c + dx - 1] (zero outside) + b[o]."""
    n, cin, h, wd = x.shape
    xp = np.zeros((n, cin, h + 2, wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    y = np.zeros((n, w.shape[0], h, wd))
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("oi,nirc->norc", w[:, :, dy, dx], xp[:, :, dy:dy + h, dx:dx + wd])
    return y + b[None, :, None, None]


def conv3x3_backward(x, w, dy):
    """Gradients of conv3x3 with respect to x, w and b, given dL/dy."""
    n, cin, h, wd = x.shape
    xp = np.zeros((n, cin, h + 2, wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            win = xp[:, :, ky:ky + h, kx:kx + wd]
            dw[:, :, ky, kx] = np.einsum("norc,nirc->oi", dy, win)
            dxp[:, :, ky:ky + h, kx:kx + wd] += np.einsum("oi,norc->nirc", w[:, :, ky, kx], dy)
    return dxp[:, :, 1:-1, 1:-1], dw, dy.sum(axis=(0, 2, 3))


def maxpool2(x):
    """2x2 / stride 2 max pooling; returns (y, argmax in 0..3, first maximum in row-major order)."""
    n, c, h, w = x.shape
    q = x.reshape(n, c, h // 2, 2, w // 2, 2).transpose(0, 1, 2, 4, 3, 5).reshape(n, c, h // 2, w // 2, 4)
    a = np.argmax(q, axis=-1)
    return np.take_along_axis(q, a[..., None], axis=-1)[..., 0], a


def maxpool2_backward(dy, a, shape):
    n, c, h, w = shape
    dq = np.zeros((n, c, h // 2, w // 2, 4))
    np.put_along_axis(dq, a[..., None], dy[..., None], axis=-1)
    return dq.reshape(n, c, h // 2, w // 2, 2, 2).transpose(0, 1, 2, 4, 3, 5).reshape(n, c, h, w)


def forward(theta, x, act=None):
    """Logits z[n] for snippets x[n][64][256]; also returns the cache for backward."""
    p = unpack(theta)
    a = np.asarray(x, dtype=np.float64)[:, None]
    cache = []
    for li in range(3):
        w, b = p[2 * li], p[2 * li + 1]
        y = conv3x3(a, w, b)
        r = np.maximum(y, 0.0)
        if act is not None:
            r = act(r)
        pooled, am = maxpool2(r)
        cache.append((a, y, r.shape, am))
        a = pooled
    f = a.reshape(a.shape[0], -1)
    hpre = f @ p[6].T + p[7]
    h = np.maximum(hpre, 0.0)
    z = h @ p[8][0] + p[9][0]
    return z, (cache, f, hpre, h)


def loss(z, y) -> float:
    z = np.asarray(z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.mean(np.logaddexp(0.0, z) - y * z))


def gradients(theta, x, y, act=None):
    """(loss, flat gradient) of the mean BCE loss by backpropagation (the rounding `act`,
    if given, is treated as the identity in the backward pass)."""
    p = unpack(theta)
    z, (cache, f, hpre, h) = forward(theta, x, act)
    y = np.asarray(y, dtype=np.float64)
    n = z.shape[0]
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / n
    g = [None] * 10
    g[8] = (dz @ h)[None, :]
    g[9] = np.array([dz.sum()])
    dh = np.outer(dz, p[8][0]) * (hpre > 0)
    g[6] = dh.T @ f
    g[7] = dh.sum(axis=0)
    da = (dh @ p[6]).reshape(n, 64, 8, 32)
    for li in (2, 1, 0):
        a, ypre, rshape, am = cache[li]
        dr = maxpool2_backward(da, am, rshape)
        dypre = dr * (ypre > 0)
        dx, g[2 * li], g[2 * li + 1] = conv3x3_backward(a, p[2 * li], dypre)
        da = dx[:, 0] if li == 0 else dx
    return loss(z, y), pack(g)


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)) and zero biases, from numpy's generator."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in param_shapes():
        if len(s) == 1:
            parts.append(np.zeros(s))
        else:
            fan_in = int(np.prod(s[1:]))
            bound = np.sqrt(6.0 / fan_in)
            parts.append(rng.uniform(-bound, bound, size=s))
    return pack(parts)
