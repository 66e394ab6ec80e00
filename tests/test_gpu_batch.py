"""Many beams per step (snd_batch_*): a batch of ragged beams (own DM grids, chunk lengths,
modes and branching) gives every beam exactly the candidates of its own plan run alone,
eagerly and through a CUDA graph, and every batched beam's candidates equal the oracle's.
A step of all beams takes a fixed handful of launches (multi-beam encoder, persistent tree,
multi-beam matched filter, cooperative candidate stage), whatever the number of beams. The
autotuner's pick leaves a float beam's plane unchanged."""
import numpy as np
import pytest

import synth
from oracle import cxx
from oracle import stream as ostream

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_15361_gb300 as g  # noqa: E402
from paper_2606_15361_gb300 import autotune  # noqa: E402

# (nchan, ndm, dm_max, chunk, mode, B)
BEAMS = [
    (64, 128, 100.0, 4096, g.MODE_FLOAT, 2),
    (128, 77, 300.0, 3000, g.MODE_FLOAT, 8),
    (64, 200, 150.0, 5000, g.MODE_GRADED, 4),
    (96, 64, 80.0, 2048, g.MODE_BINARY, 2),
    (64, 128, 100.0, 4096, g.MODE_FLOAT, 2),   # same instantiation as beam 0: shares its launch
    (256, 300, 400.0, 6000, g.MODE_FLOAT, 4),
    (64, 50, 60.0, 1024, g.MODE_GRADED, 8),
]


def _beam_data(i, nchan, chunk, nsteps, dm_max):
    f = synth.channel_freqs(nchan)
    sw = synth.K_SKY * dm_max * (f.min() ** -2 - f.max() ** -2) / synth.NC_DT
    b = synth.draw_bursts(100 + i, 4, dm_range=(0.1 * dm_max, 0.9 * dm_max), fwhm_range=(2.0, 20.0),
                          snr_range=(12.0, 30.0), t_range=(sw + 100, nsteps * chunk - 200), min_sep=300.0)
    return [synth.filterbank_chunk(100 + i, s, s * chunk, chunk, f, synth.NC_DT, b) for s in range(nsteps)]


def _plans(det_theta=5.5):
    return [g.Plan(synth.channel_freqs(nc), synth.NC_DT, synth.dm_grid(nd, dmx), B, mode,
                   g.options(mode, det_theta=det_theta, max_chunk=chunk))
            for nc, nd, dmx, chunk, mode, B in BEAMS]


def _tuples(arr):
    return [(int(c["dm_index"]), int(c["t"]), float(c["snr"]), int(c["width"]), int(c["npix"])) for c in arr]


@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_each_plan_alone(graph):
    nsteps = 6
    data = [_beam_data(i, nc, chunk, nsteps, dmx) for i, (nc, nd, dmx, chunk, mode, B) in enumerate(BEAMS)]
    dev = [[torch.from_numpy(c).cuda() for c in d] for d in data]
    solo = _plans()
    batched = _plans()
    batch = g.Batch(batched, graph=graph)
    got_solo = [[] for _ in BEAMS]
    got_batch = [[] for _ in BEAMS]
    for s in range(nsteps):
        for i, p in enumerate(solo):
            p.execute(dev[i][s])
        batch.execute([dev[i][s] for i in range(len(BEAMS))])
        if s % 2 == 1:  # read candidates mid-stream too
            for i in range(len(BEAMS)):
                got_solo[i] += _tuples(solo[i].candidates()[0])
                got_batch[i] += _tuples(batched[i].candidates()[0])
    for i in range(len(BEAMS)):
        got_solo[i] += _tuples(solo[i].candidates()[0])
        got_batch[i] += _tuples(batched[i].candidates()[0])
        assert got_batch[i] == got_solo[i], f"beam {i}"
        sb, ss = batched[i].stats(), solo[i].stats()
        assert (sb.samples_in, sb.emitted, sb.scored) == (ss.samples_in, ss.emitted, ss.scored)
    assert sum(len(x) for x in got_batch) >= 10
    if graph:
        inst, upd = batch.graph_stats()
        assert inst >= 1 and inst + upd == nsteps


@pytest.mark.parametrize("graph", [False, True])
def test_every_batched_beam_matches_oracle(graph):
    """Every beam of the batch against the C++ oracle stream of its own configuration."""
    nsteps = 4
    data = [_beam_data(i, nc, chunk, nsteps, dmx) for i, (nc, nd, dmx, chunk, mode, B) in enumerate(BEAMS)]
    plans = _plans()
    batch = g.Batch(plans, graph=graph)
    refs = [cxx.Stream(synth.channel_freqs(nc), synth.NC_DT, synth.dm_grid(nd, dmx),
                       ostream.defaults(mode, branching=B, det_theta=5.5))
            for nc, nd, dmx, chunk, mode, B in BEAMS]
    exp = [[] for _ in BEAMS]
    for s in range(nsteps):
        batch.execute([torch.from_numpy(data[i][s]).cuda() for i in range(len(BEAMS))])
        for i in range(len(BEAMS)):
            exp[i] += refs[i].push(data[i][s], want_plane=False)["candidates"]
    total = 0
    for i in range(len(BEAMS)):
        got = _tuples(plans[i].candidates()[0])
        assert got == [(c[0], c[2], float(c[3]), c[4], c[5]) for c in exp[i]], f"beam {i}"
        total += len(got)
    assert total >= 10


def test_step_launch_count_is_fixed():
    """A steady step of 7 ragged beams in 3 modes: encoder (3), one tree launch per kernel
    instantiation, one matched-filter and one candidate launch, i.e. at most 3 + 4 + 2
    launches, and the same count with twice the beams."""
    nsteps = 5
    data = [_beam_data(i, nc, chunk, nsteps, dmx) for i, (nc, nd, dmx, chunk, mode, B) in enumerate(BEAMS)]
    dev = [[torch.from_numpy(c).cuda() for c in d] for d in data]
    counts = []
    for copies in (1, 2):
        plans = _plans() + (_plans() if copies == 2 else [])
        batch = g.Batch(plans)
        for s in range(nsteps - 1):
            batch.execute([dev[i % len(BEAMS)][s] for i in range(len(plans))])
        torch.cuda.synchronize()
        l0 = sum(p.stats().kernel_launches for p in plans)
        batch.execute([dev[i % len(BEAMS)][nsteps - 1] for i in range(len(plans))])
        torch.cuda.synchronize()
        counts.append(sum(p.stats().kernel_launches for p in plans) - l0)
    insts = len({(p.stats().tree_kernel, p.stats().mode, p.stats().tree_smem_bytes > 0) for p in _plans()})
    assert counts[0] == counts[1] and counts[0] <= 3 + 4 + 2, (counts, insts)


def test_autotune_pick_keeps_the_float_plane():
    f = synth.channel_freqs(256)
    dms = synth.dm_grid(256, 300.0)
    res = autotune.autotune(f, synth.NC_DT, dms, g.MODE_FLOAT, 4096, branching=(2, 8), cluster=(3, 4), steps=2,
                            warps=(8, 4), rounds=(128, 64))
    assert len(res["trials"]) == 16 and res["branching"] in (2, 8) and res["cluster"] in (3, 4)
    assert res["tree_warps"] in (8, 4) and res["tree_round"] in (128, 64)
    t0 = res["trials"][0]
    assert (t0["branching"], t0["cluster"], t0["tree_warps"], t0["tree_round"]) == (2, 4, 8, 128)
    if not res["significant"]:
        assert (res["branching"], res["cluster"], res["tree_warps"]) == (2, 4, 8)
    assert all(t["spread_ms"] >= 0 for t in res["trials"])
    assert not autotune.tunable(g.MODE_BINARY, 256) and not autotune.tunable(g.MODE_GRADED, 1024)
    chunks = [synth.filterbank_chunk(9, i, 0, 4096, f, synth.NC_DT, []) for i in range(3)]
    planes = []
    for B, C, w, r in ((8, 4, 0, 0), (res["branching"], res["cluster"], res["tree_warps"], res["tree_round"])):
        p = g.Plan(f, synth.NC_DT, dms, B, g.MODE_FLOAT,
                   g.options(g.MODE_FLOAT, cluster_size=C, max_chunk=4096, tree_warps=w, tree_round=r))
        rows = []
        for ch in chunks:
            ne = p.nemit_next(ch.shape[0])
            out = torch.empty((len(dms), max(ne, 1)), dtype=torch.float32, device="cuda")
            p.execute(torch.from_numpy(ch).cuda(), out)
            rows.append(out[:, :ne].cpu().numpy())
        planes.append(np.concatenate(rows, axis=1))
    assert planes[0].shape[1] > 0 and np.array_equal(planes[0], planes[1])


def test_autotune_untunable_binary_searches_tile_shape_only():
    f = synth.channel_freqs(128)
    dms = synth.dm_grid(64, 200.0)
    res = autotune.autotune(f, synth.NC_DT, dms, g.MODE_BINARY, 2048, branching=(4, 8), cluster=(3,), steps=1,
                            repeats=2, warps=(8, 2), rounds=(64,))
    assert res["branching"] is None and res["cluster"] == 4
    assert {(t["branching"], t["cluster"]) for t in res["trials"]} == {(4, 4)}
    assert len(res["trials"]) == 2
