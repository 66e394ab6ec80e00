"""Pins for the C++/OpenMP oracle (oracle/cpp/snd_oracle.cpp via oracle.cxx).

It is pinned two ways: to the paper's invariants and printed values directly (delay sweep,
brute-force equality, DM = 0 channel sum, the OR/AND cascades, B-invariance, Eq. cascade
rates, Table 1 via Eq. cascade, the sigma_min worked example, scipy's closing and labels),
and cell by cell / candidate by candidate to the numpy oracle on whole streams in all three
modes (ragged chunks included)."""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

import synth
from oracle import analytic, candidates, cxx, delays, encoder, mf, stream, tree
from tests.golden import load

BINARY, GRADED, FLOAT = stream.BINARY, stream.GRADED, stream.FLOAT


def _setup(nchan, ndm, nout, p, seed, dm_max=60.0):
    f = synth.channel_freqs(nchan)
    dms = np.linspace(0, dm_max, ndm)
    tab = cxx.delay_table(f, 1.38e-4, dms)
    D = int(tab.max())
    x = synth.bernoulli_raster(seed, nchan, nout + D, p).astype(np.uint8)
    return x, tab, D


def test_delay_table_bitwise_and_printed_sweep():
    g = load.printed()
    f = synth.channel_freqs(1024)
    dms = np.linspace(0, 3000, 257)
    a = cxx.delay_table(f, synth.NC_DT, dms)
    b = delays.delay_table(f, synth.NC_DT, dms)
    assert (a == b).all()
    # the DM 3000 sweep spans ~42,500 native samples (Methods, "Hardware mapping")
    assert abs(int(a[-1].max()) - g["sweep_dm3000_samples"]) / g["sweep_dm3000_samples"] < 0.01
    # half-up rounding at 0.4 / 0.6 / 2.6 samples of the lowest channel
    sw1 = delays.sweep_samples(f, synth.NC_DT, 1.0)
    for frac, want in ((0.4, 0), (0.6, 1), (2.6, 3)):
        t = cxx.delay_table(f, synth.NC_DT, [frac / sw1])
        assert t[0].max() == want


def test_encoder_matches_clip_definition_and_numpy():
    rng = np.random.default_rng(3)
    chunk = np.clip(np.rint(rng.normal(128, 16, (4000, 40))), 0, 255).astype(np.uint8)
    chunk[:, 5] = 7                    # constant channel: never fires
    chunk[::3, 6] = 250                # two-valued
    x, lev = cxx.encode_chunk(chunk, 1.5)
    xn, levn = encoder.encode_chunk(chunk, 1.5)
    assert (lev == levn).all() and (x.astype(bool) == xn).all()
    assert lev[5] == 256 and not x[5].any()
    for c in (0, 6, 17):
        v = chunk[:, c].astype(np.float64)
        lo, hi = v.mean() - 5 * v.std(), v.mean() + 5 * v.std()
        q = np.clip(v, lo, hi)
        mu, sigma, mu0, sigma0 = cxx.channel_stats(chunk[:, c])
        assert abs(mu - q.mean()) < 1e-10 and abs(sigma - q.std()) < 1e-10
        assert abs(mu0 - v.mean()) < 1e-10 and abs(sigma0 - v.std()) < 1e-10


def test_encoder_rate_matches_discretised_gaussian_tail():
    rng = np.random.default_rng(5)
    n = 200000
    chunk = np.clip(np.rint(rng.normal(128, 16, (n, 2))), 0, 255).astype(np.uint8)
    x, lev = cxx.encode_chunk(chunk, 1.5)
    # P(round(N(128,16)) >= u) from the Gaussian CDF, the rate the integer level implies
    p = 0.5 * math.erfc(((lev[0] - 0.5) - 128.0) / (16.0 * math.sqrt(2.0)))
    rate = x[0].mean()
    assert abs(rate - p) < 5 * math.sqrt(p * (1 - p) / n)
    g = load.printed()
    assert abs(analytic.p_fire(1.5) - g["p_fire_1p5"]) < 5e-4


@pytest.mark.parametrize("nchan,C,B", [(64, 4, 2), (37, 3, 4), (16, 1, 2), (50, 7, 3), (5, 8, 2), (70, 10, 3)])
def test_float_and_uncapped_graded_equal_brute_force(nchan, C, B):
    x, tab, D = _setup(nchan, 12, 600, 0.3, nchan + C)
    rows = range(tab.shape[0])
    s = cxx.snd_rows(x, 0, tab, rows, 0, 600, FLOAT, C, B)
    b = cxx.brute_rows(x, 0, tab, rows, 0, 600)
    assert (s == b).all()
    g = cxx.snd_rows(x, 0, tab, rows, 0, 600, GRADED, C, B, cap=nchan)
    assert (g == b).all()
    # brute force written out by hand for one row
    d = 7
    want = [sum(int(x[c, t + tab[d, c]]) for c in range(nchan)) for t in range(600)]
    assert list(b[d]) == want


def test_dm0_row_is_channel_sum_and_conservation():
    x, tab, D = _setup(32, 9, 500, 0.2, 5)
    n = x.shape[1]
    s = cxx.snd_rows(x, 0, tab, [0], 0, n, FLOAT, 4, 2)
    assert (s[0] == x.sum(axis=0)).all()
    pad = np.concatenate([np.zeros((32, D), np.uint8), x, np.zeros((32, D), np.uint8)], axis=1)
    s = cxx.snd_rows(pad, -D, tab, range(9), -D, n + D, FLOAT, 4, 2)
    assert (s.sum(axis=1) == int(x.sum())).all()


def test_binary_or_and_cascades_and_hand_example():
    x, tab, D = _setup(64, 10, 700, 0.05, 11)
    b = cxx.brute_rows(x, 0, tab, range(10), 0, 700)
    s = cxx.snd_rows(x, 0, tab, range(10), 0, 700, BINARY, 4, 2, 1, 1)
    assert (s == (b >= 1)).all()
    x2, tab2, D2 = _setup(64, 10, 700, 0.97, 12)
    b2 = cxx.brute_rows(x2, 0, tab2, range(10), 0, 700)
    s2 = cxx.snd_rows(x2, 0, tab2, range(10), 0, 700, BINARY, 4, 4, 4, 4)
    assert (s2 == (b2 == 64)).all() and s2.any()
    # the numpy oracle's hand-computed 4-channel example
    xh = np.array([[1, 0, 1, 0, 0], [0, 1, 1, 0, 0], [0, 1, 0, 1, 0], [0, 0, 1, 1, 0]], dtype=np.uint8)
    th = np.array([[0, 1, 1, 2]], dtype=np.int32)
    assert list(cxx.brute_rows(xh, 0, th, [0], 0, 3)[0]) == [4, 2, 2]
    assert list(cxx.snd_rows(xh, 0, th, [0], 0, 3, BINARY, 2, 2, 2, 2)[0]) == [1, 0, 0]
    assert list(cxx.snd_rows(xh, 0, th, [0], 0, 3, BINARY, 2, 2, 1, 2)[0]) == [1, 1, 1]
    assert list(cxx.snd_rows(xh, 0, th, [0], 0, 3, GRADED, 2, 2, cap=1)[0]) == [1, 1, 1]
    assert list(cxx.snd_rows(xh, 0, th, [0], 0, 3, GRADED, 2, 2, cap=3)[0]) == [3, 2, 2]


def test_b_invariance_and_graded_cap():
    x, tab, D = _setup(128, 16, 1200, 0.2, 21, dm_max=20.0)
    rows = range(16)
    ref_f = cxx.snd_rows(x, 0, tab, rows, 0, 1200, FLOAT, 4, 2)
    ref_g = cxx.snd_rows(x, 0, tab, rows, 0, 1200, GRADED, 4, 2, cap=255)
    for B in (4, 8, 16):
        assert (cxx.snd_rows(x, 0, tab, rows, 0, 1200, FLOAT, 4, B) == ref_f).all()
        assert (cxx.snd_rows(x, 0, tab, rows, 0, 1200, GRADED, 4, B, cap=255) == ref_g).all()
    b2 = cxx.snd_rows(x, 0, tab, rows, 0, 1200, BINARY, 4, 2, 1, 2)
    b8 = cxx.snd_rows(x, 0, tab, rows, 0, 1200, BINARY, 4, 8, 1, 2)
    assert (b2 != b8).any()
    ones = np.ones((64, 10), np.uint8)
    z = np.zeros((1, 64), np.int32)
    assert cxx.snd_rows(ones, 0, z, [0], 0, 10, GRADED, 4, 2, cap=255)[0, 0] == 64
    assert cxx.snd_rows(ones, 0, z, [0], 0, 10, GRADED, 4, 2, cap=5)[0, 0] == 5


@pytest.mark.parametrize("kl,ki", [(1, 2), (2, 2), (3, 1)])
def test_cascade_rate_matches_eq_cascade(kl, ki):
    nchan, C, B, p0 = 64, 4, 2, 0.1
    x, tab, D = _setup(nchan, 3, 40000, p0, 300 + 10 * kl + ki)
    lv = tree.tree_levels(nchan, C, B)
    fan = [l[0][1] - l[0][0] for l in lv[1:]]
    p_root = analytic.cascade(p0, C, fan, kl, ki)[-1]
    s = cxx.snd_rows(x, 0, tab, [2], 0, 40000, BINARY, C, B, kl, ki)
    se = math.sqrt(max(p_root * (1 - p_root), 1e-12) / 40000)
    assert abs(s.mean() - p_root) < 5 * se + 1e-12


def test_table1_rate_of_the_nc_tree():
    # Table 1's K_L = K_I = 2 row (p_noise 2.2e-4 on the Northern Cross tree) from a long
    # Bernoulli(p(1.5)) raster through the C++ tree with zero delays
    p0 = analytic.p_fire(1.5)
    row = [r for r in load.table1() if r[0] == 2 and r[1] == 2][0]
    x = synth.bernoulli_raster(77, 1024, 300000, p0).astype(np.uint8)
    z = np.zeros((1, 1024), np.int32)
    s = cxx.snd_rows(x, 0, z, [0], 0, 300000, BINARY, 4, 8, 2, 2)
    p = float(row[2])
    se = math.sqrt(p * (1 - p) / 300000)
    assert abs(s.mean() - p) < 5 * se + 0.05 * p


def test_matched_filter_brute_force_and_sigma_min_example():
    rng = np.random.default_rng(0)
    y = rng.integers(0, 9, 300)
    widths = [1, 2, 4, 8, 16, 32]
    m, s, w, mu, sigma = cxx.row_mf(y, 250, widths, 2.0)
    for t in range(250):
        best, bw = -np.inf, 0
        for W in widths:
            v = (sum(int(a) for a in y[t:t + W]) - mu * W) / (sigma * math.sqrt(W))
            if v > best:
                best, bw = v, W
        assert abs(s[t] - best) < 1e-12 and w[t] == bw and m[t] == (best >= 2.0)
    g = load.printed()
    y = np.zeros(64 * 200, dtype=np.int64)
    y[100] = 1
    _, s, _, _, sigma = cxx.row_mf(y, y.size - 63, [64], 100.0, g["sigma_min_example"])
    assert sigma == g["sigma_min_example"] and abs(s[50] - g["snr_one_fire_w64"]) < 0.05
    y2 = np.zeros_like(y)
    y2[1000:1025] = 1
    _, s2, _, _, _ = cxx.row_mf(y2, y2.size - 63, [64], 100.0, g["sigma_min_example"])
    assert abs(s2[1000] - g["snr_25_fires_w64"]) < 0.5
    f = synth.channel_freqs(1024)
    for dm in (0.0, 3.0, 57.0, 2000.0):
        assert cxx.row_widths(f, synth.NC_DT, dm, 0.1) == mf.row_widths(f, synth.NC_DT, dm, 0.1)


@pytest.mark.parametrize("size", [1, 3, 9])
def test_closing_and_labels_against_scipy(size):
    rng = np.random.default_rng(size)
    m = rng.random((40, 70)) < 0.06
    got = cxx.closing(m, size)
    st = np.ones((size, size), bool)
    dil = ndi.binary_dilation(m, st, border_value=0)
    ero = ndi.binary_erosion(dil, st, border_value=1)
    assert (got == ero).all()
    assert (got == candidates.closing(m, size)).all()


def test_block_candidates_match_numpy_on_random_blocks():
    rng = np.random.default_rng(9)
    for trial in range(6):
        h, w = 30 + trial, 90
        m = rng.random((h, w)) < 0.04
        snr = np.where(m, rng.integers(70, 90, (h, w)) / 10.0, np.nan)   # ties are common
        wid = rng.integers(1, 64, (h, w))
        dms = np.linspace(0, 50, h)
        a = cxx.block_candidates(m, snr, wid, dms, 1000 * trial, 9, 10)
        b = candidates.block_candidates(m, snr, wid, dms, 1000 * trial, 9, 10)
        key = lambda c: (c[0], c[2], float(c[3]), c[4], c[5])  # noqa: E731
        assert [key(c) for c in a] == [key(c) for c in b]


@pytest.mark.parametrize("mode", [BINARY, GRADED, FLOAT])
@pytest.mark.parametrize("B", [2, 8])
def test_stream_matches_numpy_oracle(mode, B):
    """Whole NC64 stream in ragged chunks: emitted ranges, levels, every plane cell and the
    candidate list equal the numpy oracle's."""
    w = synth.NC64
    data = w.chunk_data(0)
    cfg = stream.defaults(mode, branching=B)
    a = stream.OracleStream(w.freqs(), synth.NC_DT, w.dms(), cfg)
    b = cxx.Stream(w.freqs(), synth.NC_DT, w.dms(), cfg)
    ca, cb = [], []
    for lo, hi in [(0, 5000), (5000, 8013), (8013, 12000), (12000, 16384)]:
        ra, rb = a.push(data[lo:hi]), b.push(data[lo:hi])
        for k in ("e_prev", "e_new", "f_prev", "nb"):
            assert ra[k] == rb[k]
        assert (ra["levels"] == rb["levels"]).all()
        assert (ra["plane"] == rb["plane"]).all()
        if mode == FLOAT:
            assert (ra["plane_float"] == rb["plane_float"]).all()
        ca += ra["candidates"]
        cb += rb["candidates"]
    key = lambda c: (c[0], c[2], float(c[3]), c[4], c[5])  # noqa: E731
    assert [key(c) for c in ca] == [key(c) for c in cb]
    if mode != BINARY:
        assert len(ca) >= 2


def test_threads_do_not_change_results():
    x, tab, D = _setup(64, 40, 800, 0.2, 4)
    n0 = cxx.max_threads()
    try:
        cxx.set_threads(1)
        a = cxx.snd_rows(x, 0, tab, range(40), 0, 800, GRADED, 4, 2, cap=255)
        cxx.set_threads(max(2, n0))
        b = cxx.snd_rows(x, 0, tab, range(40), 0, 800, GRADED, 4, 2, cap=255)
    finally:
        cxx.set_threads(n0)
    assert (a == b).all()
