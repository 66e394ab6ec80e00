"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs. Binary and graded planes must match exactly, float planes to 1e-5 relative (the
only rounding is the final float32 scale of an exact integer count), candidate lists
exactly (same islands, peaks, S/N floats, widths and pixel counts)."""
import math
import zlib

import numpy as np
import pytest

import synth
from oracle import delays as odelays
from oracle import encoder as oenc
from oracle import mf as omf
from oracle import stream as ostream
from oracle import tree as otree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_15361_gb300 as g  # noqa: E402

FLOAT_RTOL = 1e-5
MODES = {"binary": ostream.BINARY, "graded": ostream.GRADED, "float": ostream.FLOAT}


def _opts(mode, cfg, flags=0, **kw):
    o = g.options(mode, cluster_size=cfg.cluster, k_leaf=max(cfg.k_leaf, 1), k_internal=max(cfg.k_internal, 1),
                  graded_cap=cfg.cap, enc_theta=cfg.enc_theta, det_theta=cfg.det_theta, sigma_min=cfg.sigma_min,
                  mf_alpha=cfg.mf_alpha, closing_size=cfg.closing, n_min_pixels=cfg.n_min, flags=flags)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _cand_tuples(arr):
    return [(int(c["dm_index"]), int(c["t"]), float(c["snr"]), int(c["width"]), int(c["npix"])) for c in arr]


def _oracle_cands(lst):
    return [(c[0], c[2], float(c[3]), c[4], c[5]) for c in lst]


def _compare_plane(mode, got, r, nchan):
    if mode == ostream.FLOAT:
        exp = r["plane_float"]
        g64 = got.astype(np.float64)
        bad = ~(((exp == 0) & (g64 == 0)) | (np.abs(g64 - exp) <= FLOAT_RTOL * np.abs(exp)))
        assert not bad.any(), f"{bad.sum()} float cells off, e.g. {g64[bad][:4]} vs {exp[bad][:4]}"
    else:
        exp = r["plane"]
        assert got.shape == exp.shape
        diff = got != exp
        assert not diff.any(), f"{diff.sum()} cells differ; first at {np.argwhere(diff)[:3]}"


def run_both(freqs, dt, dms, mode, cfg, chunks, flags=0, host=False, **optkw):
    """Stream `chunks` through the GPU plan and the oracle; compare every emitted plane and
    the final candidate lists. Returns the GPU candidates."""
    plan = g.Plan(freqs, dt, dms, cfg.branching, mode, _opts(mode, cfg, flags, **optkw))
    ref = ostream.OracleStream(freqs, dt, dms, cfg)
    all_exp = []
    for ch in chunks:
        nemit = plan.nemit_next(ch.shape[0])
        dtype = torch.float32 if mode == ostream.FLOAT else torch.int32
        out = torch.full((len(dms), max(nemit, 1)), -7, dtype=dtype, device="cuda")
        if host:
            got_n = plan.execute_host(ch, out)
        else:
            got_n = plan.execute(torch.from_numpy(np.ascontiguousarray(ch)).cuda(), out)
        assert got_n == nemit
        r = ref.push(ch)
        assert r["e_new"] - r["e_prev"] == nemit
        if nemit:
            _compare_plane(mode, out[:, :nemit].cpu().numpy(), r, len(freqs))
        all_exp += r["candidates"]
    cands, rc = plan.candidates()
    assert rc == 0
    assert _cand_tuples(cands) == _oracle_cands(all_exp)
    return cands


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("B", [2, 8])
def test_nc64_single_chunk(mode, B):
    w = synth.NC64
    cfg = ostream.defaults(MODES[mode], branching=B)
    c = run_both(w.freqs(), synth.NC_DT, w.dms(), MODES[mode], cfg, [w.chunk_data(0)])
    if mode != "binary":
        assert len(c) >= 2


@pytest.mark.parametrize("mode", list(MODES))
def test_nc64_reference_kernel(mode):
    w = synth.NC64
    cfg = ostream.defaults(MODES[mode], branching=2)
    run_both(w.freqs(), synth.NC_DT, w.dms(), MODES[mode], cfg, [w.chunk_data(0)], flags=g.FLAG_REFERENCE_TREE)


@pytest.mark.parametrize("mode", ["graded", "float"])
def test_nc64_host_chunks_overlapped_uploads(mode):
    """Ragged page-locked host chunks through snd_execute_host on a side stream with no
    synchronisation between calls: the two staging buffers alternate and each upload waits
    only for the chunk before last, so uploads overlap the previous chunk's kernels. Every
    plane and the candidates still match the oracle."""
    w = synth.NC64
    data = w.chunk_data(0)
    cuts = [0, 1300, 1301, 5000, 5037, 9000, 12000, 16384]
    chunks = [torch.from_numpy(np.ascontiguousarray(data[a:b])).pin_memory() for a, b in zip(cuts[:-1], cuts[1:])]
    cfg = ostream.defaults(MODES[mode], branching=2)
    plan = g.Plan(w.freqs(), synth.NC_DT, w.dms(), cfg.branching, MODES[mode], _opts(MODES[mode], cfg, 0))
    ref = ostream.OracleStream(w.freqs(), synth.NC_DT, w.dms(), cfg)
    side = torch.cuda.Stream()
    outs = []
    for ch in chunks:
        nemit = plan.nemit_next(ch.shape[0])
        dtype = torch.float32 if MODES[mode] == ostream.FLOAT else torch.int32
        out = torch.full((len(w.dms()), max(nemit, 1)), -7, dtype=dtype, device="cuda")
        side.wait_stream(torch.cuda.current_stream())  # the fill above runs on the default stream
        assert plan.execute_host(ch, out, stream=side) == nemit
        outs.append((out, nemit))
    torch.cuda.synchronize()
    all_exp = []
    for ch, (out, nemit) in zip(chunks, outs):
        r = ref.push(ch.numpy())
        assert r["e_new"] - r["e_prev"] == nemit
        if nemit:
            _compare_plane(MODES[mode], out[:, :nemit].cpu().numpy(), r, w.nchan)
        all_exp += r["candidates"]
    cands, rc = plan.candidates()
    assert rc == 0
    assert _cand_tuples(cands) == _oracle_cands(all_exp)
    assert len(cands) >= 1


@pytest.mark.parametrize("mode", list(MODES))
def test_nc64_streaming_ragged_chunks(mode):
    w = synth.NC64
    data = w.chunk_data(0)
    cuts = [0, 1300, 1301, 5000, 5037, 9000, 16384]
    chunks = [data[a:b] for a, b in zip(cuts[:-1], cuts[1:])]
    cfg = ostream.defaults(MODES[mode], branching=2)
    run_both(w.freqs(), synth.NC_DT, w.dms(), MODES[mode], cfg, chunks)


def test_host_chunk_path_matches():
    w = synth.NC64
    cfg = ostream.defaults(ostream.GRADED, branching=4)
    data = w.chunk_data(0)
    run_both(w.freqs(), synth.NC_DT, w.dms(), ostream.GRADED, cfg, [data[:8000], data[8000:]], host=True)


CASES = [
    # (name, nchan, C, B, ndm, dm_max, mode, kl, ki, cap, shuffle_dms, ascending_freqs)
    ("ragged-leaves", 37, 4, 3, 21, 80.0, ostream.BINARY, 2, 2, 255, False, False),
    ("c3-b5", 45, 3, 5, 17, 60.0, ostream.GRADED, 0, 0, 255, False, True),
    ("c1-b2", 16, 1, 2, 9, 90.0, ostream.FLOAT, 0, 0, 255, False, False),
    ("c7-b4", 50, 7, 4, 33, 40.0, ostream.BINARY, 3, 1, 255, True, False),
    ("quorum-k4", 64, 4, 4, 24, 70.0, ostream.BINARY, 4, 3, 255, False, False),
    ("or-cascade", 32, 4, 2, 8, 30.0, ostream.BINARY, 1, 1, 255, False, False),
    ("graded-cap5", 64, 4, 2, 19, 50.0, ostream.GRADED, 0, 0, 5, True, False),
    ("graded-cap200", 96, 4, 2, 11, 50.0, ostream.GRADED, 0, 0, 200, False, False),
    ("one-dm", 64, 4, 8, 1, 25.0, ostream.FLOAT, 0, 0, 255, False, False),
    ("one-leaf", 3, 4, 2, 5, 40.0, ostream.BINARY, 2, 2, 255, False, False),
    ("deep-b2", 512, 4, 2, 13, 30.0, ostream.GRADED, 0, 0, 255, False, False),
    ("deep-binary-k8", 512, 4, 2, 13, 30.0, ostream.BINARY, 3, 2, 255, False, False),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_edge_configurations(case):
    name, nchan, C, B, ndm, dm_max, mode, kl, ki, cap, shuf, asc = case
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    f = synth.channel_freqs(nchan)
    if asc:
        f = f[::-1].copy()
    dms = np.linspace(0.0, dm_max, ndm)
    if shuf:
        dms = rng.permutation(np.concatenate([dms, dms[:2]]))  # unsorted, with duplicates
    cfg = ostream.defaults(mode, cluster=C, branching=B, k_leaf=kl, k_internal=ki, cap=cap,
                           det_theta=5.0, n_min=3)
    D = int(odelays.delay_table(f, synth.NC_DT, dms).max())
    n = D + 6000
    bursts = [synth.Burst(D + 1500.0, float(dms.max()) * 0.6, 6.0, 40.0),
              synth.Burst(D + 4100.0, float(dms.max()) * 0.3, 20.0, 30.0)]
    data = synth.filterbank_chunk(11, 0, 0, n, f, synth.NC_DT, bursts)
    chunks = [data[: n // 3], data[n // 3: n // 3 + 777], data[n // 3 + 777:]]
    run_both(f, synth.NC_DT, dms, mode, cfg, chunks)


@pytest.mark.parametrize("size", [1, 3, 15, 31])
@pytest.mark.parametrize("ref", [False, True], ids=["fused", "separable"])
def test_closing_sizes(size, ref):
    """Closing element sides from 1 (no closing) to the largest allowed, through the fused
    tiled kernel and the four separable passes (reference flag), on a 64-channel beam with a
    low detection threshold so that many mask cells and islands meet the tile borders."""
    w = synth.NC64
    data = w.chunk_data(0)
    cfg = ostream.defaults(ostream.FLOAT, branching=2, det_theta=4.0, closing=size, n_min=3)
    flags = g.FLAG_REFERENCE_TREE if ref else 0
    c = run_both(w.freqs(), synth.NC_DT, w.dms(), ostream.FLOAT, cfg, [data[:9000], data[9000:]], flags=flags)
    assert len(c) >= 3


def test_capacity_overflow_reports_and_keeps_prefix():
    w = synth.NC64
    cfg = ostream.defaults(ostream.GRADED, branching=2)
    plan = g.Plan(w.freqs(), synth.NC_DT, w.dms(), 2, ostream.GRADED, _opts(ostream.GRADED, cfg, cand_capacity=1))
    plan.execute(torch.from_numpy(w.chunk_data(0)).cuda())
    cands, rc = plan.candidates(check=False)
    assert rc == g.ERR["SND_ERR_OVERFLOW"] and len(cands) == 1
    ref = ostream.OracleStream(w.freqs(), synth.NC_DT, w.dms(), cfg).push(w.chunk_data(0))["candidates"]
    assert len(ref) > 1


def test_chunk_too_long_rejected():
    w = synth.NC64
    plan = g.Plan(w.freqs(), synth.NC_DT, w.dms(), 2, ostream.FLOAT, g.options(ostream.FLOAT, max_chunk=1000))
    with pytest.raises(g.SndError) as e:
        plan.execute(torch.zeros((1001, 64), dtype=torch.uint8, device="cuda"))
    assert e.value.code == g.ERR["SND_ERR_CHUNK"]
    assert plan.execute(torch.zeros((1000, 64), dtype=torch.uint8, device="cuda")) == 0


@pytest.mark.parametrize("mode", ["binary", "graded"])
def test_uint8_plane_output(mode):
    """plane_dtype = 1 writes the same root values as uint8."""
    w = synth.NC64
    cfg = ostream.defaults(MODES[mode], branching=2)
    data = w.chunk_data(0)
    plan = g.Plan(w.freqs(), synth.NC_DT, w.dms(), 2, MODES[mode], _opts(MODES[mode], cfg, plane_dtype=1))
    ref = ostream.OracleStream(w.freqs(), synth.NC_DT, w.dms(), cfg)
    for ch in (data[:6000], data[6000:]):
        ne = plan.nemit_next(ch.shape[0])
        out = torch.full((len(w.dms()), max(ne, 1)), 77, dtype=torch.uint8, device="cuda")
        assert plan.execute(torch.from_numpy(np.ascontiguousarray(ch)).cuda(), out) == ne
        r = ref.push(ch)
        if ne:
            assert (out[:, :ne].cpu().numpy().astype(np.int64) == r["plane"]).all()
    c, rc = plan.candidates()
    assert rc == 0
