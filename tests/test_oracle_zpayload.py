"""Pins for oracle.zpayload (float-mode precision study): stored partial sums reduce to the
exact Mode C counts for the 0/1 payload up to 2048 channels per node, lose exactly what the
rounding rules say beyond it, and stay within the classical summation error bounds for the
labelled z payload."""
import math

import numpy as np

import synth
from oracle import delays as odelays
from oracle import encoder as oenc
from oracle import tree as otree
from oracle import zpayload as oz


def _rows_stored(x, delays, levels, store, nout):
    return np.stack([oz.stored_root(oz.gather(x, 0, delays[d], 0, nout), levels, store) for d in range(len(delays))])


def test_zero_one_payload_in_fp16_equals_mode_c_counts():
    """With the paper's 0/1 spikes every node holds an integer <= its channel count <= 2048,
    so FP16 storage reproduces the integer tree of Mode C exactly."""
    rng = np.random.default_rng(5)
    nchan, nsamp = 256, 900
    f = synth.channel_freqs(nchan)
    dms = np.linspace(0.0, 30.0, 6)
    dl = odelays.delay_table(f, 1.38e-4, dms)
    x = rng.random((nchan, nsamp)) < 0.3
    nout = nsamp - int(dl.max())
    for C, B in [(4, 2), (4, 8), (3, 5)]:
        levels = otree.tree_levels(nchan, C, B)
        counts = otree.snd_rows(x, 0, dl, range(len(dms)), 0, nout, otree.FLOAT, C, B)
        got = _rows_stored(x.astype(np.float16), dl, levels, np.float16, nout)
        assert (got.astype(np.float64) == counts).all()


def test_fp16_node_over_2048_channels_rounds():
    """A leaf of 2049 firing channels stores fp16(2049) = 2048 (ties to even); the FP32 root
    then reads 2048 + 1 = 2049 instead of the count 2050. FP32 storage keeps 2050."""
    a = np.ones((2050, 1), dtype=np.float16)
    levels = otree.tree_levels(2050, 2049, 2)
    assert [len(l) for l in levels] == [2, 1]
    assert oz.stored_root(a, levels, np.float16)[0] == 2049.0
    assert oz.stored_root(a.astype(np.float32), levels, np.float32)[0] == 2050.0


def test_rounding_points_by_hand():
    """Leaves [2048, 1] and [1, 0.5]: FP32 sums 2049 and 1.5, stored in FP16 as 2048 and 1.5;
    the root (not stored) is 2049.5. A root-level store would give 2050."""
    a = np.array([[2048.0], [1.0], [1.0], [0.5]], dtype=np.float16)
    levels = otree.tree_levels(4, 2, 2)
    assert oz.stored_root(a, levels, np.float16)[0] == np.float32(2049.5)
    # single level: the leaf is the root, kept in FP32
    assert oz.stored_root(a, otree.tree_levels(4, 4, 2), np.float16)[0] == np.float32(2050.5)


def test_exactly_representable_payload_is_exact():
    """Payloads on a 1/16 grid with node sums below 128 are exact in FP16 at every node, so
    the stored tree equals the FP64 sum (no term dropped, no index misplaced)."""
    rng = np.random.default_rng(9)
    nchan, nsamp = 96, 400
    x64 = rng.integers(0, 20, size=(nchan, nsamp)) / 16.0
    dl = odelays.delay_table(synth.channel_freqs(nchan), 1.38e-4, np.linspace(0, 20, 5))
    nout = nsamp - int(dl.max())
    levels = otree.tree_levels(nchan, 4, 3)
    got = _rows_stored(x64.astype(np.float16), dl, levels, np.float16, nout)
    exp = np.stack([oz.gather(x64, 0, dl[d], 0, nout).sum(axis=0) for d in range(len(dl))])
    assert (got.astype(np.float64) == exp).all()


def test_payload_table_against_encoder():
    rng = np.random.default_rng(2)
    chunk = np.clip(np.rint(rng.normal(128, 16, size=(3000, 5))), 0, 255).astype(np.uint8)
    chunk[:, 4] = 77  # constant channel: sigma = 0, never fires
    z, u = oz.payload_table(chunk, 1.5)
    assert (u == oenc.chunk_levels(chunk, 1.5)).all()
    assert u[4] == 256 and not z[4].any()
    for c in range(4):
        mu, sigma, _, _ = oenc.channel_stats(chunk[:, c])
        assert (z[c, :u[c]] == 0).all()
        assert z[c, u[c]] > 1.5 and z[c, u[c] - 1] == 0
        assert abs(z[c, 200] - (200 - mu) / sigma) <= 1e-12 * abs(z[c, 200])
        assert (np.diff(z[c, u[c]:]) > 0).all()


def _z_case(nchan=128, nsamp=2500, seed=4):
    rng = np.random.default_rng(seed)
    chunk = np.clip(np.rint(rng.normal(128, 16, size=(nsamp, nchan))), 0, 255).astype(np.uint8)
    z64, _ = oz.payload_table(chunk, 1.0)
    f = synth.channel_freqs(nchan)
    dl = odelays.delay_table(f, 1.38e-4, np.linspace(0, 60, 7))
    return chunk, z64, dl, nsamp - int(dl.max())


def test_fp32_storage_within_summation_bound():
    """Recursive FP32 summation: a payload passes through at most (C-1) + (B-1)(L-1) adds, so
    |y - y64| <= (that + 1) u32 * sum|x| (u32 = 2^-24), plus the final scale's rounding."""
    chunk, z64, dl, nout = _z_case()
    nchan = chunk.shape[1]
    C, B = 4, 2
    levels = otree.tree_levels(nchan, C, B)
    x32 = oz.payload(chunk, z64.astype(np.float32))
    x64 = oz.payload(chunk, z64)
    adds = (C - 1) + (B - 1) * (len(levels) - 1)
    u32 = 2.0 ** -24
    for d in range(len(dl)):
        y = oz.stored_root(oz.gather(x32, 0, dl[d], 0, nout), levels, np.float32).astype(np.float64)
        a64 = oz.gather(x64, 0, dl[d], 0, nout)
        exact = a64.sum(axis=0)
        bound = (adds + 1) * u32 * np.abs(a64).sum(axis=0) + 1e-300
        assert (np.abs(y - exact) <= bound).all()


def test_fp16_storage_within_bound_and_worse_than_fp32():
    """FP16 storage: the payload and each of the L-1 stored nodes on its path round with
    relative error <= 2^-11, so |y - y64| <= (L * 2^-11 + adds * 2^-24) sum|x| (first
    order); the z payload makes that error visible, larger than FP32 storage."""
    chunk, z64, dl, nout = _z_case()
    nchan = chunk.shape[1]
    C, B = 4, 2
    levels = otree.tree_levels(nchan, C, B)
    L = len(levels)
    adds = (C - 1) + (B - 1) * (L - 1)
    x16 = oz.payload(chunk, z64.astype(np.float16))
    x32 = oz.payload(chunk, z64.astype(np.float32))
    x64 = oz.payload(chunk, z64)
    e16 = e32 = 0.0
    for d in range(len(dl)):
        a64 = oz.gather(x64, 0, dl[d], 0, nout)
        exact = a64.sum(axis=0)
        y16 = oz.stored_root(oz.gather(x16, 0, dl[d], 0, nout), levels, np.float16).astype(np.float64)
        y32 = oz.stored_root(oz.gather(x32, 0, dl[d], 0, nout), levels, np.float32).astype(np.float64)
        bound = (L * 2.0 ** -11 * (1 + 2.0 ** -10) + adds * 2.0 ** -24) * np.abs(a64).sum(axis=0) + 1e-300
        assert (np.abs(y16 - exact) <= bound).all()
        e16 = max(e16, float(np.abs(y16 - exact).max()))
        e32 = max(e32, float(np.abs(y32 - exact).max()))
    assert e16 > 10 * e32 > 0


def test_zstream_emits_like_main_path_and_reports_error():
    w = synth.NC64
    data = w.chunk_data(0)
    s16 = oz.ZStream(w.freqs(), synth.NC_DT, w.dms(), 4, 2, 1.5, np.float16, rows=[0, 50, 127])
    r1 = s16.push(data[:9000])
    r2 = s16.push(data[9000:])
    D = int(odelays.delay_table(w.freqs(), synth.NC_DT, w.dms()).max())
    assert (r1["e_prev"], r1["e_new"], r2["e_new"]) == (0, 9000 - D, 16384 - D)
    err = oz.error_per_dm(r2["plane"], r2["plane64"])
    assert (err["max_rel_to_peak"] < 2e-3).all() and (err["max_abs"] > 0).all()
    # the DM = 0 row is the plain channel sum of the payload at each time (each chunk with its
    # own statistics)
    x = np.concatenate([oz.payload(part, oz.payload_table(part, 1.5)[0]) for part in (data[:9000], data[9000:])],
                       axis=1)
    t0, t1 = r2["e_prev"], r2["e_new"]
    assert np.allclose(r2["plane64"][0], x[:, t0:t1].sum(axis=0) / math.sqrt(64), rtol=1e-12, atol=0)


def test_unit_payload_is_the_paper_raster():
    """With the unit payload (the paper's 0/1 spikes) the stored-sum tree is the spike count:
    FP32 storage gives fp32(count) * fp32(1/sqrt(N_f)) for any tree, FP16 storage too while no
    stored node holds more than 2048 channels."""
    w = synth.NC64
    data = w.chunk_data(0)[:3000]
    freqs, dms = w.freqs(), w.dms()[:12]
    tab = odelays.delay_table(freqs, synth.NC_DT, dms)
    x = oenc.encode_chunk(data, 1.5)[0]
    D = int(tab.max())
    counts = otree.snd_rows(x, 0, tab, range(12), 0, 3000 - D, otree.FLOAT, 4, 2)
    for st in (np.float16, np.float32):
        r = oz.ZStream(freqs, synth.NC_DT, dms, 4, 2, 1.5, st, unit=True).push(data)
        exp = (counts.astype(np.float32) * oz.plane_scale(64)).astype(np.float32)
        assert r["e_new"] == 3000 - D and (r["plane"] == exp).all()


def test_unit_payload_fp16_rounds_nodes_above_2048():
    """4100 channels, B = 2: the root's first child holds 4096 channels and is stored. At
    theta = -2 almost every channel fires, so that child's count exceeds 2048 and FP16 storage
    rounds it to an even number (ties to even); FP32 storage keeps the exact count."""
    nchan = 4100
    freqs = synth.channel_freqs(nchan)
    dms = np.array([0.0, 3.0])
    rng = np.random.default_rng(4)
    data = np.clip(np.rint(rng.normal(128, 16, (300, nchan))), 0, 255).astype(np.uint8)
    r16 = oz.ZStream(freqs, synth.NC_DT, dms, 4, 2, -2.0, np.float16, unit=True).push(data)
    r32 = oz.ZStream(freqs, synth.NC_DT, dms, 4, 2, -2.0, np.float32, unit=True).push(data)
    sc = oz.plane_scale(nchan)
    count32 = np.rint(r32["plane"].astype(np.float64) / float(sc))
    exact = np.rint(r32["plane64"] * np.sqrt(float(nchan)))
    assert (count32 == exact).all() and exact.min() > 2048 + 4
    x = oenc.encode_chunk(data, -2.0)[0]
    tab = odelays.delay_table(freqs, synth.NC_DT, dms)
    n = r16["e_new"]
    a_first = otree.snd_rows(x[:4096], 0, tab[:, :4096], [0, 1], 0, n, otree.FLOAT, 4, 2)
    a_rest = otree.snd_rows(x[4096:], 0, tab[:, 4096:], [0, 1], 0, n, otree.FLOAT, 4, 2)
    want16 = (a_first.astype(np.float16).astype(np.float32) + a_rest.astype(np.float32)) * sc
    assert (r16["plane"] == want16.astype(np.float32)).all()
    assert (r16["plane"] != r32["plane"]).any()
