"""Many beams per step (snd_batch_*): a batch of ragged beams (own DM grids, chunk lengths,
modes and branching) gives every beam exactly the candidates of its own plan run alone,
eagerly and through a CUDA graph; the single-beam plans are themselves checked against the
oracle in test_gpu_parity.py, and one batched beam is checked against the oracle here. The
autotuner's pick leaves a float beam's plane unchanged."""
import numpy as np
import pytest

import synth
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


def test_batched_beam_matches_oracle():
    """Beam 1 of a batch (128 channels, B = 8, float) against the FP64 oracle stream."""
    nsteps = 4
    data = [_beam_data(i, nc, chunk, nsteps, dmx) for i, (nc, nd, dmx, chunk, mode, B) in enumerate(BEAMS)]
    plans = _plans()
    batch = g.Batch(plans, graph=True)
    nc, nd, dmx, chunk, mode, B = BEAMS[1]
    cfg = ostream.defaults(ostream.FLOAT, branching=B, det_theta=5.5)
    ref = ostream.OracleStream(synth.channel_freqs(nc), synth.NC_DT, synth.dm_grid(nd, dmx), cfg)
    exp = []
    for s in range(nsteps):
        batch.execute([torch.from_numpy(data[i][s]).cuda() for i in range(len(BEAMS))])
        exp += ref.push(data[1][s])["candidates"]
    got = _tuples(plans[1].candidates()[0])
    assert got == [(c[0], c[2], float(c[3]), c[4], c[5]) for c in exp]


def test_autotune_pick_keeps_the_float_plane():
    f = synth.channel_freqs(256)
    dms = synth.dm_grid(256, 300.0)
    res = autotune.autotune(f, synth.NC_DT, dms, g.MODE_FLOAT, 4096, branching=(2, 8), cluster=(3, 4), steps=2)
    assert len(res["trials"]) == 4 and res["branching"] in (2, 8) and res["cluster"] in (3, 4)
    assert not autotune.tunable(g.MODE_BINARY, 256) and not autotune.tunable(g.MODE_GRADED, 1024)
    chunks = [synth.filterbank_chunk(9, i, 0, 4096, f, synth.NC_DT, []) for i in range(3)]
    planes = []
    for B, C in ((8, 4), (res["branching"], res["cluster"])):
        p = g.Plan(f, synth.NC_DT, dms, B, g.MODE_FLOAT, g.options(g.MODE_FLOAT, cluster_size=C, max_chunk=4096))
        rows = []
        for ch in chunks:
            ne = p.nemit_next(ch.shape[0])
            out = torch.empty((len(dms), max(ne, 1)), dtype=torch.float32, device="cuda")
            p.execute(torch.from_numpy(ch).cuda(), out)
            rows.append(out[:, :ne].cpu().numpy())
        planes.append(np.concatenate(rows, axis=1))
    assert planes[0].shape[1] > 0 and np.array_equal(planes[0], planes[1])
