"""GPU parity of the labelled-payload Mode C tree (SND_MODE_ZFLOAT) with FP16 and FP32
partial-sum storage against oracle.zpayload: the planes must be bit-identical to the
oracle's stored-sum evaluation (same rounding points, same FP32 addition order), and their
error against the FP64 definition is reported per DM trial and bounded."""
import numpy as np
import pytest

import synth
from oracle import zpayload as oz

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_15361_gb300 as g  # noqa: E402

STORES = {"fp16": (np.float16, g.FLAG_FP16_PARTIALS), "fp32": (np.float32, 0)}


def run_z(freqs, dms, chunks, B, store, C=4, theta=1.5, rows=None, max_chunk=None):
    st, flag = STORES[store]
    o = g.options(g.MODE_ZFLOAT, cluster_size=C, enc_theta=theta, flags=flag)
    if max_chunk:
        o.max_chunk = max_chunk
    plan = g.Plan(freqs, synth.NC_DT, dms, B, g.MODE_ZFLOAT, o)
    ref = oz.ZStream(freqs, synth.NC_DT, dms, C, B, theta, st, rows=rows)
    rows = list(range(len(dms))) if rows is None else list(rows)
    errs = []
    for ch in chunks:
        nemit = plan.nemit_next(ch.shape[0])
        out = torch.full((len(dms), max(nemit, 1)), float("nan"), dtype=torch.float32, device="cuda")
        assert plan.execute(torch.from_numpy(np.ascontiguousarray(ch)).cuda(), out) == nemit
        r = ref.push(ch)
        assert r["e_new"] - r["e_prev"] == nemit
        if nemit:
            got = out[rows, :nemit].cpu().numpy()
            exp = r["plane"]
            bad = got.view(np.uint32) != exp.view(np.uint32)
            assert not bad.any(), f"{bad.sum()} cells differ, e.g. {got[bad][:4]} vs {exp[bad][:4]}"
            errs.append(oz.error_per_dm(got, r["plane64"]))
    c, rc = plan.candidates()
    assert rc == 0 and len(c) == 0
    return errs


@pytest.mark.parametrize("store", list(STORES))
@pytest.mark.parametrize("B", [2, 8])
def test_nc64_zfloat_bit_exact(store, B):
    w = synth.NC64
    data = w.chunk_data(0)
    errs = run_z(w.freqs(), w.dms(), [data[:7001], data[7001:]], B, store)
    worst = max(float(e["max_rel_to_peak"].max()) for e in errs)
    assert worst < (2e-3 if store == "fp16" else 1e-6)


@pytest.mark.parametrize("store", list(STORES))
def test_ragged_channels_and_cluster(store):
    """250 channels (ragged last leaf), C = 3, B = 5, several chunk lengths."""
    f = synth.channel_freqs(250)
    dms = synth.dm_grid(77, 300.0)
    chunks = [synth.filterbank_chunk(3, i, 0, n, f, synth.NC_DT, []) for i, n in enumerate([5000, 4096, 123, 9000])]
    run_z(f, dms, chunks, 5, store, C=3)


@pytest.mark.parametrize("store", list(STORES))
def test_deep_tree_b2_256ch(store):
    """256 channels, C = 1, B = 2: nine levels (the deepest kernel instantiation)."""
    f = synth.channel_freqs(256)
    dms = synth.dm_grid(40, 200.0)
    chunks = [synth.filterbank_chunk(5, i, 0, 6000, f, synth.NC_DT, []) for i in range(2)]
    run_z(f, dms, chunks, 2, store, C=1)


@pytest.mark.parametrize("store", list(STORES))
def test_nc1024_full_size_sampled_rows(store):
    """The full Northern Cross beam (1024 channels, 2048 DMs, B = 8, 16384-sample chunks), in
    the bench's launch configuration: sampled DM rows against the oracle, bit for bit."""
    w = synth.NC1024
    rows = sorted(set(np.linspace(0, w.ndm - 1, 24).astype(int).tolist()) | {1, 2046})
    chunks = [w.chunk_data(i) for i in range(3)]
    errs = run_z(w.freqs(), w.dms(), chunks, 8, store, rows=rows, max_chunk=w.chunk)
    e = errs[-1]
    # per DM trial error of the full-chunk plane against FP64 (printed for the record)
    print(f"\nzfloat {store} per-DM error vs FP64 over {len(rows)} sampled trials: max_abs "
          f"median {np.median(e['max_abs']):.3e} max {e['max_abs'].max():.3e}; max_rel_to_peak "
          f"median {np.median(e['max_rel_to_peak']):.3e} max {e['max_rel_to_peak'].max():.3e}")
    assert e["max_rel_to_peak"].max() < (2e-3 if store == "fp16" else 1e-6)


@pytest.mark.parametrize("store", list(STORES))
def test_unit_payload_4100_channels_rounds_above_2048(store):
    """The paper's own 0/1 payload (SND_FLAG_UNIT_PAYLOAD) on 4100 channels with B = 2: the
    root's first child holds 4096 channels and is stored. At theta = -2 almost every channel
    fires, so its count passes 2048 and FP16 storage rounds it (ties to even) exactly as the
    oracle's stored-sum tree does; FP32 storage keeps the count. Bit-identical planes."""
    nchan = 4100
    freqs = synth.channel_freqs(nchan)
    dms = np.linspace(0.0, 6.0, 5)
    rng = np.random.default_rng(41)
    data = np.clip(np.rint(rng.normal(128, 16, (1500, nchan))), 0, 255).astype(np.uint8)
    st, flag = STORES[store]
    o = g.options(g.MODE_ZFLOAT, cluster_size=4, enc_theta=-2.0, flags=flag | g.FLAG_UNIT_PAYLOAD, max_chunk=1000)
    plan = g.Plan(freqs, synth.NC_DT, dms, 2, g.MODE_ZFLOAT, o)
    ref = oz.ZStream(freqs, synth.NC_DT, dms, 4, 2, -2.0, st, unit=True)
    rounded = 0
    for ch in (data[:700], data[700:]):
        ne = plan.nemit_next(ch.shape[0])
        out = torch.full((len(dms), max(ne, 1)), float("nan"), dtype=torch.float32, device="cuda")
        assert plan.execute(torch.from_numpy(np.ascontiguousarray(ch)).cuda(), out) == ne
        r = ref.push(ch)
        if ne:
            got = out[:, :ne].cpu().numpy()
            assert (got.view(np.uint32) == r["plane"].view(np.uint32)).all()
            exact = (np.rint(r["plane64"] * np.sqrt(float(nchan))).astype(np.float32) *
                     oz.plane_scale(nchan)).astype(np.float32)
            rounded += int((got != exact).sum())
    assert (rounded > 0) == (store == "fp16")
