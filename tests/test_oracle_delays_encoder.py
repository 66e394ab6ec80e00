"""Pins for oracle.delays, oracle.encoder and oracle.analytic against values the paper
prints and against closed forms / library routines."""
import math

import numpy as np
import pytest

import synth
from oracle import analytic, delays, encoder
from tests.golden import load


def test_kdm_matches_printed_constant():
    g = load.printed()
    # 4.149e6 MHz^2 ms == 4.149e3 MHz^2 s, agreeing to the printed 4 digits
    assert abs(delays.K_DM * 1e3 - g["kdm_mhz2_ms"]) / g["kdm_mhz2_ms"] < 2e-4


def test_sweep_dm3000_matches_printed():
    g = load.printed()
    f = synth.channel_freqs(1024)
    s = delays.sweep_samples(f, 1.38e-4, 3000.0)
    assert abs(s - g["sweep_dm3000_samples"]) / g["sweep_dm3000_samples"] < 2e-3
    tab = delays.delay_table(f, 1.38e-4, [3000.0])
    assert abs(tab.max() - s) <= 0.5


def test_delay_table_structure():
    f = synth.channel_freqs(64)
    dms = np.linspace(0, 100, 33)
    tab = delays.delay_table(f, 1.38e-4, dms)
    assert tab.shape == (33, 64)
    assert (tab[0] == 0).all()                       # DM 0
    assert (tab[:, delays.reference_channel(f)] == 0).all()
    assert (np.diff(tab, axis=0) >= 0).all()         # monotone in DM
    assert (np.diff(tab, axis=1) >= 0).all()         # channel 0 highest -> delays grow with c
    # ascending frequency order gives the mirrored table
    tab2 = delays.delay_table(f[::-1], 1.38e-4, dms)
    assert (tab2 == tab[:, ::-1]).all()


def test_delay_rounding_half_up():
    # two channels, dt chosen so that x = 0.4 and 0.6 of a sample
    f = np.array([2.0, 1.0])
    base = delays.K_DM * (1.0 - 0.25)
    t = delays.delay_table(f, base / 0.4, [1.0])
    assert t[0, 1] == 0
    t = delays.delay_table(f, base / 0.6, [1.0])
    assert t[0, 1] == 1
    t = delays.delay_table(f, base / 2.6, [1.0])
    assert t[0, 1] == 3


def test_p_fire_printed():
    g = load.printed()
    assert abs(analytic.p_fire(1.5) - g["p_fire_1p5"]) < 5e-5
    assert abs(1024 * analytic.p_fire(0.75) - g["graded_baseline_counts"]) < 0.5


def _plain_stats(col):
    """The paper's four steps written with numpy clip/mean/std (different summation order)."""
    p = col.astype(np.float64)
    mu0, s0 = p.mean(), p.std()
    q = np.clip(p, mu0 - 5 * s0, mu0 + 5 * s0)
    return q.mean(), q.std()


@pytest.mark.parametrize("seed", range(6))
def test_encoder_recipe_matches_plain_definition(seed):
    rng = np.random.default_rng(seed)
    n = 5000 + 997 * seed
    col = np.clip(np.rint(rng.normal(128, 16, n)), 0, 255)
    # heavy right tail (RFI-like) so that clipping matters
    hot = rng.random(n) < 0.01
    col[hot] = 250 + rng.integers(0, 6, hot.sum())
    col = col.astype(np.uint8)
    mu, sigma, mu0, sigma0 = encoder.channel_stats(col)
    pm, ps = _plain_stats(col)
    assert abs(mu - pm) < 1e-10 * abs(pm)
    assert abs(sigma - ps) < 1e-10 * ps
    assert abs(mu0 - col.mean()) < 1e-10 * mu0
    for theta in (0.75, 1.5, 2.0):
        u = encoder.level_from_stats(mu, sigma, theta)
        fires = (col.astype(np.float64) - pm) / ps > theta
        assert (fires == (col >= u)).all()


def test_encoder_fire_rate_discretised_gaussian():
    # round(N(128,16)): fire iff P >= u, u = smallest integer above mu + theta*sigma ~ 152
    x = synth.filterbank_chunk(7, 0, 0, 200000, synth.channel_freqs(1), 1e-3)
    xs, u = encoder.encode_chunk(x, 1.5)
    rate = xs.mean()
    p_disc = 0.5 * math.erfc(((u[0] - 0.5) - 128.0) / 16.0 / math.sqrt(2))
    assert u[0] in (152, 153)          # mu + 1.5 sigma sits right at 152
    se = math.sqrt(p_disc * (1 - p_disc) / xs.size)
    assert abs(rate - p_disc) < 5 * se
    assert abs(rate - analytic.p_fire(1.5)) < 0.006     # the printed theory, within discretisation


def test_encoder_degenerate_channels():
    n = 100
    const = np.full((n, 1), 77, np.uint8)
    x, u = encoder.encode_chunk(const, 1.5)
    assert u[0] == 256 and not x.any()
    two = np.zeros((n, 1), np.uint8)
    two[::2] = 10
    x, u = encoder.encode_chunk(two, 0.5)
    # mu = 5, sigma = 5: threshold 7.5 -> u = 8, the 10s fire
    assert u[0] == 8 and x.sum() == 50
    neg = np.zeros((n, 1), np.uint8)
    neg[0] = 255
    x, u = encoder.encode_chunk(neg, -3.0)
    assert u[0] == 0 and x.all()       # negative threshold: every sample fires
    hi = np.zeros((n, 1), np.uint8)
    hi[:50] = 255
    x, u = encoder.encode_chunk(hi, 1.5)
    assert u[0] == 256                  # threshold above 255 -> never fires


def test_encoder_clip_matters():
    rng = np.random.default_rng(3)
    col = np.clip(np.rint(rng.normal(100, 5, 10000)), 0, 255).astype(np.uint8)
    col[:300] = 255
    mu, sigma, mu0, sigma0 = encoder.channel_stats(col)
    assert sigma < sigma0 and mu < mu0
