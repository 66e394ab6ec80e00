"""GPU parity of the multi-rate search (snd_multirate_*) against oracle.multirate on the same
seeded inputs: same bands, and the merged candidate lists identical (global DM index,
native time, S/N float, width in native samples, pixel count)."""
import numpy as np
import pytest

import synth
from oracle import multirate as omr
from oracle import stream as ostream

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_15361_gb300 as g  # noqa: E402

MODES = {"binary": ostream.BINARY, "graded": ostream.GRADED, "float": ostream.FLOAT}


def _opts(mode, cfg, **kw):
    o = g.options(mode, cluster_size=cfg.cluster, k_leaf=max(cfg.k_leaf, 1), k_internal=max(cfg.k_internal, 1),
                  graded_cap=cfg.cap, enc_theta=cfg.enc_theta, det_theta=cfg.det_theta, sigma_min=cfg.sigma_min,
                  mf_alpha=cfg.mf_alpha, closing_size=cfg.closing, n_min_pixels=cfg.n_min)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _tuples(arr):
    return [(int(c["dm_index"]), int(c["t"]), float(c["snr"]), int(c["width"]), int(c["npix"])) for c in arr]


def _oracle_tuples(lst):
    return [(int(c[0]), int(c[2]), float(c[3]), int(c[4]), int(c[5])) for c in lst]


def run_both(freqs, dt, dms, mode, cfg, chunks, s_max=64, host=False, reads=None, graph=False, **optkw):
    plan = g.MultiRatePlan(freqs, dt, dms, cfg.branching, mode, _opts(mode, cfg, **optkw), s_max=s_max)
    plan.set_graph(graph)
    ref = omr.MultiRateStream(freqs, dt, dms, cfg, s_max=s_max)
    assert plan.scrunch == [s for s, _ in ref.bands]
    assert plan.band_ndm == [len(idx) for _, idx in ref.bands]
    reads = set(reads or [len(chunks) - 1])
    got, exp = [], []
    for i, ch in enumerate(chunks):
        if host:
            plan.execute_host(ch)
        else:
            plan.execute(torch.from_numpy(np.ascontiguousarray(ch)).cuda())
        ref.push(ch)
        if i in reads:
            c, rc = plan.candidates()
            assert rc == 0
            got.append(_tuples(c))
            exp.append(_oracle_tuples(ref.candidates()))
    assert got == exp
    return got


@pytest.mark.parametrize("mode", list(MODES))
def test_nc64_multirate_one_chunk(mode):
    w = synth.NC64
    cfg = ostream.defaults(MODES[mode], branching=2)
    got = run_both(w.freqs(), synth.NC_DT, w.dms(), MODES[mode], cfg, [w.chunk_data(0)])
    if mode != "binary":
        assert len(got[0]) >= 1


def test_nc64_multirate_bands_present():
    w = synth.NC64
    plan = g.MultiRatePlan(w.freqs(), synth.NC_DT, w.dms(), 2, ostream.GRADED, bind=False)
    assert len(plan.scrunch) >= 3 and plan.scrunch[0] == 1
    assert sum(plan.band_ndm) == len(w.dms())
    st = plan.band_plan(len(plan.scrunch) - 1).stats()
    assert st.ndm == plan.band_ndm[-1]


def test_nc64_multirate_streaming_and_reads():
    """Chunks of several lengths (multiples of the largest S) with candidate reads between them,
    through the host-chunk entry point."""
    w = synth.NC64
    data = w.chunk_data(0)
    cfg = ostream.defaults(ostream.FLOAT, branching=4)
    smax = max(omr.bands(w.freqs(), synth.NC_DT, w.dms())[-1][0], 1)
    cuts = [0, 256 * smax // 8, 5000 // smax * smax, 9000 // smax * smax, 16384]
    chunks = [data[a:b] for a, b in zip(cuts[:-1], cuts[1:])]
    run_both(w.freqs(), synth.NC_DT, w.dms(), ostream.FLOAT, cfg, chunks, host=True, reads=[1, 3])


def test_nc64_multirate_s_max_caps_bands():
    w = synth.NC64
    cfg = ostream.defaults(ostream.GRADED, branching=2)
    run_both(w.freqs(), synth.NC_DT, w.dms(), ostream.GRADED, cfg, [w.chunk_data(0)], s_max=2)


def test_multirate_chunk_must_be_multiple_of_s_max():
    w = synth.NC64
    plan = g.MultiRatePlan(w.freqs(), synth.NC_DT, w.dms(), 2, ostream.GRADED)
    smax = max(plan.scrunch)
    assert smax > 1
    x = torch.zeros((smax + 1, w.nchan), dtype=torch.uint8, device="cuda")
    with pytest.raises(g.SndError) as e:
        plan.execute(x)
    assert e.value.code == g.ERR["SND_ERR_CHUNK"]


def _burst_chunks(seed, nchan, dm_max, ndm, nchunks, nbursts, **kw):
    f = synth.channel_freqs(nchan)
    dms = synth.dm_grid(ndm, dm_max)
    sw = synth.K_SKY * dm_max * (f.min() ** -2 - f.max() ** -2) / synth.NC_DT
    b = synth.draw_bursts(seed, nbursts, dm_range=(5.0, 0.99 * dm_max), t_range=(sw + 100, nchunks * 16384 - 2000),
                          min_sep=300.0, **kw)
    chunks = [synth.filterbank_chunk(seed, i, i * 16384, 16384, f, synth.NC_DT, b) for i in range(nchunks)]
    return f, dms, chunks


@pytest.mark.parametrize("mode", ["graded", "float"])
def test_multirate_merges_across_bands_64ch(mode):
    """16 bursts 300 samples apart at DMs over all four bands: the merge joins candidates
    across bands and neighbouring bursts (oracle: 16 band candidates -> 12 merged, graded)."""
    f, dms, chunks = _burst_chunks(7, 64, 100.0, 128, 2, 16, fwhm_range=(2.0, 30.0), snr_range=(9.0, 25.0))
    cfg = ostream.defaults(MODES[mode], branching=2)
    got = run_both(f, synth.NC_DT, dms, MODES[mode], cfg, chunks)
    assert len(got[0]) >= 8


@pytest.mark.parametrize("mode", list(MODES))
def test_multirate_256ch_five_bands(mode):
    """256 channels, 256 DMs up to 1000 (bands S = 1..16), three chunks, B = 4; float mode
    replays every chunk through a CUDA graph."""
    f, dms, chunks = _burst_chunks(11, 256, 1000.0, 256, 3, 24, fwhm_range=(2.0, 60.0), snr_range=(9.0, 30.0),
                                   log_fwhm=True)
    cfg = ostream.defaults(MODES[mode], branching=4)
    got = run_both(f, synth.NC_DT, dms, MODES[mode], cfg, chunks, s_max=16, graph=(mode == "float"))
    if mode != "binary":
        assert len(got[0]) >= 10
