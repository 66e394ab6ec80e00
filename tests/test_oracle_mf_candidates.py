"""Pins for oracle.mf and oracle.candidates: brute-force window sums, the printed sigma_min
worked example, closing/labelling against scipy.ndimage, and hand-made islands."""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

import synth
from oracle import candidates, delays, mf
from tests.golden import load


def test_widths_rule():
    f = synth.channel_freqs(1024)
    assert mf.row_widths(f, 1.38e-4, 0.0, 0.1) == [1, 2, 4, 8]
    assert mf.row_widths(f, 1.38e-4, 2000.0, 0.1) == [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024]
    # boundary: 16 enters exactly when alpha * sweep reaches 16
    sw1 = delays.sweep_samples(f, 1.38e-4, 1.0)
    dm16 = 16.0 / (0.1 * sw1)
    assert 16 not in mf.row_widths(f, 1.38e-4, dm16 * 0.999, 0.1)
    assert 16 in mf.row_widths(f, 1.38e-4, dm16 * 1.001, 0.1)


def test_window_sums_brute_force():
    rng = np.random.default_rng(0)
    y = rng.integers(0, 9, 300)
    nb, widths = 250, [1, 2, 4, 8, 16, 32]
    m, s, w, mu, sigma = mf.row_mf(y, nb, widths, 2.0)
    assert abs(mu - y[:nb].mean()) < 1e-12 and abs(sigma - y[:nb].std()) < 1e-12
    for t in range(nb):
        best, bw = -np.inf, 0
        for W in widths:
            v = (sum(int(a) for a in y[t:t + W]) - mu * W) / (sigma * math.sqrt(W))
            if v > best:
                best, bw = v, W
        assert abs(s[t] - best) < 1e-12 and w[t] == bw and m[t] == (best >= 2.0)


def test_sigma_min_worked_example():
    g = load.printed()
    # binary row, mean ~ 0: one fire in a W = 64 boxcar, then ~25 fires in the same window
    y = np.zeros(64 * 200, dtype=np.int64)
    y[100] = 1
    _, s, _, mu, sigma = mf.row_mf(y, y.size - 63, [64], 100.0, g["sigma_min_example"])
    assert sigma == g["sigma_min_example"]
    assert abs(s[50] - g["snr_one_fire_w64"]) < 0.05
    y2 = np.zeros_like(y)
    y2[1000:1025] = 1
    _, s2, _, _, _ = mf.row_mf(y2, y2.size - 63, [64], 100.0, g["sigma_min_example"])
    assert abs(s2[1000] - g["snr_25_fires_w64"]) < 0.5


def test_eq_snr_a_on_exact_rates():
    # a row whose noise part has exactly rate p_n and a W-sample segment with rate p_s:
    # with exact row statistics the filter reproduces Eq. snr_A.
    from oracle import analytic
    W, n = 64, 64 * 400
    y = np.zeros(n + W, dtype=np.int64)
    y[::50] = 1                       # p_n = 1/50 over the block
    nb = n
    mu, sigma = mf.row_stats(y[:nb])
    seg = 20 * W
    y[seg:seg + W] = 0
    y[seg:seg + W:2] = 1              # p_s = 1/2 inside the segment
    mu, sigma = mf.row_stats(y[:nb])
    _, s, _, _, _ = mf.row_mf(y, nb, [W], 1e9)
    pred = analytic.snr_binary(W, 0.5, mu) * math.sqrt(mu * (1 - mu)) / sigma
    assert abs(s[seg] - pred) < 1e-9


def test_width_tie_goes_to_smaller():
    y = np.array([0, 0, 0, 0, 5, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0], dtype=np.int64)
    # at t = 4, W = 1 and W = 2 contain the same sum; with mu = 0 the larger W scores lower,
    # so force equality with a zero-sigma-free constant row segment instead
    m, s, w, mu, sigma = mf.row_mf(y, 12, [1, 2], -1e9)
    assert w[4] == 1
    flat = np.full(30, 3, dtype=np.int64)
    m, s, w, mu, sigma = mf.row_mf(flat, 10, [1, 2, 4], 0.0)
    assert sigma == 0.0 and not m.any() and np.isnan(s).all()


@pytest.mark.parametrize("seed", range(4))
def test_closing_matches_scipy(seed):
    rng = np.random.default_rng(seed)
    m = rng.random((40, 70)) < 0.03
    se = np.ones((9, 9), bool)
    ref = ndi.binary_erosion(ndi.binary_dilation(m, se, border_value=0), se, border_value=1)
    got = candidates.closing(m, 9)
    assert (got == ref).all() and (got >= m).all()


@pytest.mark.parametrize("seed", range(4))
def test_label8_matches_scipy(seed):
    rng = np.random.default_rng(10 + seed)
    m = rng.random((30, 50)) < 0.25
    lab, n, pix = candidates.label8(m)
    ref, nref = ndi.label(m, structure=np.ones((3, 3), bool))
    assert n == nref
    for k in range(1, n + 1):
        # same partition: each of our islands maps to exactly one scipy island of equal size
        vals = np.unique(ref[lab == k])
        assert vals.size == 1 and (ref == vals[0]).sum() == (lab == k).sum() == len(pix[k - 1])


def test_block_candidates_hand_example():
    ndm, nb = 30, 60
    mask = np.zeros((ndm, nb), bool)
    snr = np.zeros((ndm, nb))
    width = np.ones((ndm, nb), np.int64)
    # island A: two runs in one row with a 3-sample gap -> closed into one island;
    # its two best pixels tie in S/N -> the smaller t wins (same DM)
    mask[10, 20:24] = True
    mask[10, 27:30] = True
    snr[10, 20:24] = 8.0
    snr[10, 27:30] = 8.0
    snr[10, 22] = snr[10, 28] = 9.0
    width[10, 22] = 4
    # island B: a single pixel stays a single pixel -> dropped by n_min = 2
    mask[20, 45] = True
    snr[20, 45] = 50.0
    dms = np.arange(ndm, dtype=np.float64) * 2.0
    closed = candidates.closing(mask, 9)
    assert closed[10, 20:30].all() and closed.sum() == 11
    out = candidates.block_candidates(mask, snr, width, dms, 1000, 9, 2)
    assert len(out) == 1
    d, dm, t, s, w, npix = out[0]
    assert (d, t, w, npix) == (10, 1022, 4, 10) and s == np.float32(9.0) and dm == np.float32(20.0)
    # n_min counts closed pixels: the single pixel survives with n_min = 1; sorted by t
    out = candidates.block_candidates(mask, snr, width, dms, 1000, 9, 1)
    assert [(c[0], c[2], c[5]) for c in out] == [(10, 1022, 10), (20, 1045, 1)]
    # ties between DMs at equal S/N go to the smaller DM index
    mask2 = np.zeros((ndm, nb), bool)
    mask2[12, 30] = mask2[11, 31] = True
    snr2 = np.zeros((ndm, nb))
    snr2[12, 30] = snr2[11, 31] = 7.5
    out = candidates.block_candidates(mask2, snr2, width, dms, 0, 9, 1)
    assert len(out) == 1 and (out[0][0], out[0][2]) == (11, 31)


def test_closing_touches_block_border():
    # erosion treats outside as 1, so an island within 4 pixels of the block edge grows to it
    m = np.zeros((30, 60), bool)
    m[27, 30] = True
    c = candidates.closing(m, 9)
    assert c[27:30, 30].all() and c.sum() == 3
