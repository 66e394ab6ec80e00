"""Pins for oracle.tree: brute-force equality, closed-form special cases, conservation,
B-invariance, the cascade recursion (Eq. cascade) and Table 1's printed noise rates."""
import itertools
import math

import numpy as np
import pytest

import synth
from oracle import analytic, delays, tree
from oracle.tree import BINARY, FLOAT, GRADED
from tests.golden import load


def _setup(nchan, ndm, nout, p, seed, dm_max=60.0):
    """Raster covering nout output samples plus the maximum delay: returns (x, tab, D)."""
    f = synth.channel_freqs(nchan)
    dms = np.linspace(0, dm_max, ndm)
    tab = delays.delay_table(f, 1.38e-4, dms)
    D = int(tab.max())
    x = synth.bernoulli_raster(seed, nchan, nout + D, p)
    return x, tab, D


def test_levels_nc_shape():
    g = load.printed()
    lv = tree.tree_levels(1024, 4, 8)
    assert [len(l) for l in lv] == [256, 32, 4, 1]
    assert len(lv) == g["nc_levels"]
    assert lv[-1][0] == (0, int(g["nc_root_fanin"]))
    lv = tree.tree_levels(10, 4, 2)   # ragged: leaves 4,4,2
    assert lv[0] == [(0, 4), (4, 8), (8, 10)]
    assert lv[1] == [(0, 2), (2, 3)] and lv[2] == [(0, 2)]
    assert tree.tree_levels(3, 4, 2) == [[(0, 3)]]


@pytest.mark.parametrize("nchan,C,B", [(64, 4, 2), (37, 3, 4), (16, 1, 2), (50, 7, 3), (5, 8, 2)])
def test_float_equals_brute_force(nchan, C, B):
    x, tab, D = _setup(nchan, 12, 600, 0.3, nchan + C)
    nout = 600
    rows = range(tab.shape[0])
    s = tree.snd_rows(x, 0, tab, rows, 0, nout, FLOAT, C, B)
    b = tree.brute_rows(x, 0, tab, rows, 0, nout)
    assert (s == b).all()
    g = tree.snd_rows(x, 0, tab, rows, 0, nout, GRADED, C, B, cap=nchan)
    assert (g == b).all()


def test_dm0_row_is_channel_sum_and_conservation():
    x, tab, D = _setup(32, 9, 500, 0.2, 5)
    n = x.shape[1]
    s = tree.snd_rows(x, 0, tab, [0], 0, n, FLOAT, 4, 2)
    assert (s[0] == x.sum(axis=0)).all()
    # spike conservation with zero padding on both sides
    pad = np.concatenate([np.zeros((32, D), bool), x, np.zeros((32, D), bool)], axis=1)
    s = tree.snd_rows(pad, -D, tab, range(9), -D, n + D, FLOAT, 4, 2)
    assert (s.sum(axis=1) == x.sum()).all()


def test_binary_or_and_cascades():
    x, tab, D = _setup(64, 10, 700, 0.05, 11)
    nout = 700
    b = tree.brute_rows(x, 0, tab, range(10), 0, nout)
    s = tree.snd_rows(x, 0, tab, range(10), 0, nout, BINARY, 4, 2, 1, 1)
    assert (s == (b >= 1)).all()
    x2, tab2, D2 = _setup(64, 10, 700, 0.97, 12)
    b2 = tree.brute_rows(x2, 0, tab2, range(10), 0, 700)
    s2 = tree.snd_rows(x2, 0, tab2, range(10), 0, 700, BINARY, 4, 4, 4, 4)
    assert (s2 == (b2 == 64)).all() and s2.any()


def test_hand_example():
    # 4 channels, C=2, B=2, one DM with delays 0,1,1,2; raster chosen by hand
    x = np.array([[1, 0, 1, 0, 0],
                  [0, 1, 1, 0, 0],
                  [0, 1, 0, 1, 0],
                  [0, 0, 1, 1, 0]], dtype=bool)
    tab = np.array([[0, 1, 1, 2]])
    # a_c(t) for t = 0,1,2: ch0 x[0][t], ch1 x[1][t+1], ch2 x[2][t+1], ch3 x[3][t+2]
    # t=0: 1,1,1,1 ; t=1: 0,1,0,1 ; t=2: 1,0,1,0
    assert (tree.brute_rows(x, 0, tab, [0], 0, 3)[0] == [4, 2, 2]).all()
    # leaves {0,1},{2,3}: t=0: 2,2 ; t=1: 1,1 ; t=2: 1,1
    assert (tree.snd_rows(x, 0, tab, [0], 0, 3, BINARY, 2, 2, 2, 2)[0] == [1, 0, 0]).all()
    assert (tree.snd_rows(x, 0, tab, [0], 0, 3, BINARY, 2, 2, 1, 2)[0] == [1, 1, 1]).all()
    assert (tree.snd_rows(x, 0, tab, [0], 0, 3, GRADED, 2, 2, cap=1)[0] == [1, 1, 1]).all()
    assert (tree.snd_rows(x, 0, tab, [0], 0, 3, GRADED, 2, 2, cap=3)[0] == [3, 2, 2]).all()


def test_b_invariance():
    x, tab, D = _setup(128, 16, 1200, 0.2, 21, dm_max=20.0)
    nout = 1200
    rows = range(16)
    ref_f = tree.snd_rows(x, 0, tab, rows, 0, nout, FLOAT, 4, 2)
    ref_g = tree.snd_rows(x, 0, tab, rows, 0, nout, GRADED, 4, 2, cap=255)
    for B in (4, 8, 16):
        assert (tree.snd_rows(x, 0, tab, rows, 0, nout, FLOAT, 4, B) == ref_f).all()
        assert (tree.snd_rows(x, 0, tab, rows, 0, nout, GRADED, 4, B, cap=255) == ref_g).all()
    # binary mode is not B-invariant in general
    b2 = tree.snd_rows(x, 0, tab, rows, 0, nout, BINARY, 4, 2, 1, 2)
    b8 = tree.snd_rows(x, 0, tab, rows, 0, nout, BINARY, 4, 8, 1, 2)
    assert (b2 != b8).any()


def test_graded_cap_binds_only_at_capped_nodes():
    # all channels fire: graded root = min(N_f, cap) only if lower nodes never exceed cap
    x = np.ones((64, 10), bool)
    tab = np.zeros((1, 64), np.int64)
    assert tree.snd_rows(x, 0, tab, [0], 0, 10, GRADED, 4, 2, cap=255)[0, 0] == 64
    # cap 5: leaves 4, level1 min(8,5)=5, level2 min(10,5)=5 ... root 5
    assert tree.snd_rows(x, 0, tab, [0], 0, 10, GRADED, 4, 2, cap=5)[0, 0] == 5


@pytest.mark.parametrize("kl,ki", [(1, 2), (2, 1), (2, 2), (3, 1), (1, 3)])
def test_cascade_rate_matches_eq_cascade(kl, ki):
    # one DM, disjoint channel sets per node -> root is Bernoulli(p_root) per time sample
    nchan, C, B, p0 = 64, 4, 2, 0.1
    x, tab, D = _setup(nchan, 3, 40000, p0, 100 + 10 * kl + ki)
    lv = tree.tree_levels(nchan, C, B)
    fan = [hi - lo for hi, lo in [(l[0][1], l[0][0]) for l in lv[1:]]]
    p_root = analytic.cascade(p0, C, fan, kl, ki)[-1]
    nout = 40000
    s = tree.snd_rows(x, 0, tab, [2], 0, nout, BINARY, C, B, kl, ki)
    rate = s.mean()
    se = math.sqrt(max(p_root * (1 - p_root), 1e-12) / nout)
    assert abs(rate - p_root) < 5 * se + 1e-12


def test_table1_printed_noise_rates():
    p0 = analytic.p_fire(1.5)
    lv = tree.tree_levels(1024, 4, 8)
    fan = [lv[i][0][1] - lv[i][0][0] for i in range(1, len(lv))]
    assert fan == [8, 8, 4]
    for kl, ki, p_txt, s_txt in load.table1():
        p = analytic.cascade(p0, 4, fan, kl, ki)[-1]
        if p_txt == "tiny":
            assert p < 1e-15
        else:
            pv = float(p_txt)
            digits = len(p_txt.split("e")[0].replace(".", "").lstrip("0"))
            assert abs(p - pv) <= 0.5 * 10 ** (math.floor(math.log10(pv)) - digits + 1) + 1e-18 \
                or (pv == 1.0 and p > 0.99)
        if s_txt not in ("-", "inf", ">1e7"):
            s = analytic.snr_binary(1, 1.0, p)
            assert abs(s - float(s_txt)) <= 0.05 + 0.002 * float(s_txt)
        if s_txt == ">1e7":
            assert analytic.snr_binary(1, 1.0, p) > 1e7


@pytest.mark.parametrize("mode,kl,ki", [(BINARY, 2, 2), (BINARY, 1, 2), (FLOAT, 0, 0), (GRADED, 0, 0)])
def test_level_fire_rates_match_eq_cascade(mode, kl, ki):
    """Per-level fire rates on a Bernoulli(p) raster with zero delays: binary levels follow Eq.
    cascade level by level; a float or graded node is nonzero iff any of its n channels fired,
    so its rate is 1 - (1 - p)^n (the OR cascade)."""
    nchan, C, B, p0, n = 64, 4, 2, 0.1, 30000
    x = synth.bernoulli_raster(900 + kl + 10 * mode, nchan, n, p0)
    tab = np.zeros((1, nchan), np.int64)
    counts = tree.level_fire_counts(x, 0, tab, [0], 0, n, mode, C, B, kl, ki)
    lv = tree.tree_levels(nchan, C, B)
    fan = [l[0][1] - l[0][0] for l in lv[1:]]
    if mode == BINARY:
        want = analytic.cascade(p0, C, fan, kl, ki)
    else:
        want = [1 - (1 - p0) ** (C * B ** l) for l in range(len(lv))]
    for l, (c, w) in enumerate(zip(counts, want)):
        nodes = len(lv[l])
        rate = c / (nodes * n)
        assert abs(rate - w) < 5 * math.sqrt(max(w * (1 - w), 1e-12) / (nodes * n)) + 1e-9, (l, rate, w)
