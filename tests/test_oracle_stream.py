"""Streaming bookkeeping of the oracle and a qualitative recovery check on the 64-channel
workload (all modes peak at the injected DM and time, cf. the mode comparison figure)."""
import numpy as np
import pytest

import synth
from oracle import encoder, stream, tree


def test_emitted_ranges_and_plane_consistency():
    w = synth.NC64
    data = w.chunk_data(0)
    cfg = stream.defaults(stream.GRADED, branching=2)
    s = stream.OracleStream(w.freqs(), synth.NC_DT, w.dms(), cfg)
    cuts = [0, 5000, 8000, 8013, 16384]
    xs, es, fs, nbs = [], [0], [0], []
    for a, b in zip(cuts[:-1], cuts[1:]):
        r = s.push(data[a:b])
        xs.append(encoder.encode_chunk(data[a:b], cfg.enc_theta)[0])
        assert r["e_prev"] == es[-1] and r["f_prev"] == fs[-1]
        es.append(r["e_new"])
        fs.append(r["f_prev"] + r["nb"])
        x = np.concatenate(xs, axis=1)
        ref = tree.snd_rows(x, 0, s.delays, [0, 7, 127], r["e_prev"], r["e_new"] - r["e_prev"],
                            cfg.mode, 4, 2, cap=255)
        assert (r["plane"][[0, 7, 127]] == ref).all()
    assert es[-1] == 16384 - s.D
    assert fs[-1] == max(0, es[-1] - (s.wmax - 1))


def test_float_plane_scaling():
    w = synth.NC64
    s = stream.OracleStream(w.freqs(), synth.NC_DT, w.dms()[:4], stream.defaults(stream.FLOAT))
    r = s.push(w.chunk_data(0)[:4000])
    assert np.allclose(r["plane_float"], r["plane"] / 8.0, rtol=0, atol=0)


@pytest.mark.parametrize("mode", [stream.GRADED, stream.FLOAT])
def test_bursts_recovered(mode):
    w = synth.NC64
    s = stream.OracleStream(w.freqs(), synth.NC_DT, w.dms(), stream.defaults(mode, branching=2))
    r = s.push(w.chunk_data(0))
    found = 0
    for b in w.bursts():
        for c in r["candidates"]:
            if abs(c[1] - b.dm) <= 10.0 and abs(c[2] - b.t0) <= 10:
                found += 1
                break
    assert found >= 2
