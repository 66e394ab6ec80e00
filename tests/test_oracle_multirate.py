"""Pins for oracle.multirate: the printed Northern Cross band edges (Supplementary Table S1)
follow from Eq. scrunch, scrunching is a rounded mean, merging is single-linkage."""
import os

import numpy as np

import synth
from oracle import multirate as mr
from oracle import stream

HERE = os.path.dirname(os.path.abspath(__file__))


def _printed_bands():
    rows = []
    for line in open(os.path.join(HERE, "golden", "multirate_bands.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            s, lo, hi = line.split()
            rows.append((int(s), float(lo), float(hi)))
    return rows


def test_nc_band_edges_match_table_s1():
    f = synth.channel_freqs(1024)
    dt = 1.38e-4
    printed = _printed_bands()
    prev_hi = None
    for s, lo, hi in printed:
        # mid-band DMs get the printed scrunch factor
        assert mr.scrunch_factor(f, dt, 0.5 * (lo + hi), s_max=16) == s
        if s > 1:
            # Eq. scrunch boundary s*dt = tau_smear(d) lies between the printed end of the lower
            # band and the printed start of this one (the table prints whole DMs)
            d_s = s * dt / (mr.smear_seconds(f, 1.0))
            assert prev_hi <= d_s <= lo + 0.5
            assert mr.scrunch_factor(f, dt, d_s + 0.01, s_max=16) == s
            assert mr.scrunch_factor(f, dt, d_s - 0.01, s_max=16) == s // 2
        prev_hi = hi


def test_scrunch_is_rounded_mean():
    x = np.array([[1, 200], [2, 201], [4, 0], [5, 255]], dtype=np.uint8)
    y = mr.scrunch(x, 2)
    assert y.tolist() == [[2, 201], [5, 128]]   # (1+2+1)//2=2, (200+201+1)//2=201, (4+5+1)//2=5, (255+1)//2=128
    assert (mr.scrunch(x, 1) == x).all()


def test_merge_single_linkage_and_peak():
    dms = np.arange(0.0, 100.0, 1.0)
    dt = 1e-3  # 200 ms = 200 samples
    c = [(10, 10.0, 1000, 8.0, 4, 12),   # A
         (25, 25.0, 1150, 9.0, 8, 12),   # within 20 DM / 200 samples of A
         (44, 44.0, 1300, 7.5, 8, 12),   # chained through the second one
         (90, 90.0, 1000, 30.0, 2, 12),  # far in DM: alone
         (12, 12.0, 5000, 6.0, 1, 12)]   # far in time: alone
    m = mr.merge(c, dms, dt)
    assert [(x[0], x[2]) for x in m] == [(90, 1000), (25, 1150), (12, 5000)]
    # ties on S/N: smaller DM index wins
    m2 = mr.merge([(5, 5.0, 0, 7.0, 1, 10), (3, 3.0, 100, 7.0, 1, 10)], dms, dt)
    assert len(m2) == 1 and m2[0][0] == 3


def test_single_band_equals_single_rate():
    w = synth.NC64
    dms = np.linspace(0.0, 10.0, 16)     # tau_smear < 2 dt for all: one band, S = 1
    cfg = stream.defaults(stream.GRADED, branching=2)
    m = mr.MultiRateStream(w.freqs(), synth.NC_DT, dms, cfg)
    assert [s for s, _ in m.bands] == [1]
    ref = stream.OracleStream(w.freqs(), synth.NC_DT, dms, cfg)
    data = w.chunk_data(0)
    m.push(data)
    r = ref.push(data)
    assert m.candidates() == mr.merge([(c[0], c[1], c[2], c[3], c[4], c[5]) for c in r["candidates"]], dms,
                                      synth.NC_DT)


def test_nc64_multirate_finds_bursts():
    w = synth.NC64
    cfg = stream.defaults(stream.FLOAT, branching=2)
    m = mr.MultiRateStream(w.freqs(), synth.NC_DT, w.dms(), cfg)
    assert [s for s, _ in m.bands] == [1, 2, 4, 8]
    m.push(w.chunk_data(0))
    got = m.candidates()
    found = sum(any(abs(c[1] - b.dm) <= 20 and abs(c[2] - b.t0) <= 200 for c in got) for b in w.bursts())
    assert found >= 2
