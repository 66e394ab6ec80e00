"""The direct tree kernel (csrc/tree_direct.cu) against the oracle, over the configurations it
takes: float at 64 to 4096 channels; graded with the exact level at the root, one or two capped
levels above it, and caps that bind below the root; binary with every leaf quorum K_L = 1..4,
K_I = 1..2, regular and ragged upper levels, and the fixed-logic state of B = 4 and 8. Each case streams ragged chunks with injected
bursts; every plane cell and the candidate list must equal the C++ oracle's, and the plan must
report the kernel that the case is meant to exercise. A last case checks that the leaf-sharing
kernel (SND_FLAG_LEAF_SHARING) and the direct kernel give the same planes on the 1024-channel
beam."""
import zlib

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

B_, G_, F_ = ostream.BINARY, ostream.GRADED, ostream.FLOAT

CASES = [
    # name, nchan, B, ndm, dm_max, mode, kl, ki, cap, expect_direct
    ("float-64-b2", 64, 2, 40, 80.0, F_, 0, 0, 255, True),
    ("float-128-b3", 128, 3, 33, 150.0, F_, 0, 0, 255, True),
    ("float-1024-b8", 1024, 8, 70, 900.0, F_, 0, 0, 255, True),
    ("float-4096-b4", 4096, 4, 36, 300.0, F_, 0, 0, 255, True),
    ("graded-256-root", 256, 2, 45, 200.0, G_, 0, 0, 255, True),
    ("graded-512-b2-u1", 512, 2, 31, 300.0, G_, 0, 0, 255, True),
    ("graded-1024-b2-u2", 1024, 2, 40, 500.0, G_, 0, 0, 255, True),
    ("graded-1024-b8-cap100", 1024, 8, 40, 600.0, G_, 0, 0, 100, True),
    ("graded-1024-b16-root", 1024, 16, 40, 600.0, G_, 0, 0, 255, True),
    ("graded-cap20-fallback", 256, 2, 20, 100.0, G_, 0, 0, 20, False),
    ("binary-64-b2", 64, 2, 40, 80.0, B_, 2, 2, 255, True),
    ("binary-256-b3-k1", 256, 3, 35, 200.0, B_, 1, 2, 255, True),
    ("binary-256-b8-k3", 256, 8, 35, 200.0, B_, 3, 1, 255, True),
    ("binary-1024-b2-k4", 1024, 2, 33, 400.0, B_, 4, 2, 255, True),
    ("binary-1024-b8-k2", 1024, 8, 64, 900.0, B_, 2, 2, 255, True),
    ("binary-4096-b2-k2", 4096, 2, 32, 200.0, B_, 2, 2, 255, True),
    # regular trees (B = 4, 8): the in-group levels as fixed logic; the root inside one group
    # (64 channels at B = 4), just above it (64 at B = 8), and ragged top levels
    ("binary-64-b4-root-in-group", 64, 4, 40, 80.0, B_, 2, 2, 255, True),
    ("binary-64-b8-k1", 64, 8, 40, 80.0, B_, 2, 1, 255, True),
    ("binary-192-b4-k1", 192, 4, 35, 150.0, B_, 1, 1, 255, True),
    ("binary-1024-b4-k3", 1024, 4, 40, 600.0, B_, 3, 2, 255, True),
    ("binary-3072-b8-k2", 3072, 8, 33, 300.0, B_, 2, 2, 255, True),
    ("binary-k3-internal-fallback", 256, 2, 20, 100.0, B_, 2, 3, 255, False),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_direct_kernel_cases(case):
    name, nchan, B, ndm, dm_max, mode, kl, ki, cap, expect_direct = case
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    f = synth.channel_freqs(nchan)
    dms = np.linspace(0.0, dm_max, ndm)
    cfg = ostream.defaults(mode, branching=B, k_leaf=kl, k_internal=ki, cap=cap, det_theta=5.0, n_min=3)
    D = int(cxx.delay_table(f, synth.NC_DT, dms).max())
    n = D + 7000
    bursts = [synth.Burst(1500.0 + 2500.0 * i, float(rng.uniform(0.2, 0.9) * dm_max), float(rng.uniform(2, 20)),
                          float(rng.uniform(25, 60))) for i in range(2)]
    data = synth.filterbank_chunk(zlib.crc32(name.encode()) & 0xFFFF, 0, 0, n, f, synth.NC_DT, bursts)
    cuts = [0, n // 3, n // 3 + 1111, n]
    o = g.options(mode, k_leaf=max(kl, 1), k_internal=max(ki, 1), graded_cap=cap, det_theta=5.0, n_min_pixels=3)
    plan = g.Plan(f, synth.NC_DT, dms, B, mode, o)
    assert plan.stats().tree_kernel == (1 if expect_direct else 0)
    ref = cxx.Stream(f, synth.NC_DT, dms, cfg)
    dtype = torch.float32 if mode == F_ else torch.int32
    exp_c = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        ch = np.ascontiguousarray(data[a:b])
        ne = plan.nemit_next(ch.shape[0])
        out = torch.full((ndm, max(ne, 1)), -7, dtype=dtype, device="cuda")
        assert plan.execute(torch.from_numpy(ch).cuda(), out) == ne
        r = ref.push(ch)
        assert r["e_new"] - r["e_prev"] == ne
        if ne:
            got = out[:, :ne].cpu().numpy()
            if mode == F_:
                exp = r["plane_float"]
                bad = ~(((exp == 0) & (got == 0)) | (np.abs(got.astype(np.float64) - exp) <= 1e-5 * np.abs(exp)))
                assert not bad.any(), np.argwhere(bad)[:4]
            else:
                diff = got != r["plane"]
                assert not diff.any(), f"{diff.sum()} cells differ, first at {np.argwhere(diff)[:4]}"
        exp_c += r["candidates"]
    got_c, rc = plan.candidates()
    assert rc == 0
    assert [(int(c["dm_index"]), int(c["t"]), float(c["snr"]), int(c["width"]), int(c["npix"])) for c in got_c] == \
        [(c[0], c[2], float(c[3]), c[4], c[5]) for c in exp_c]


@pytest.mark.parametrize("mode", ["binary", "graded", "float"])
def test_direct_equals_leaf_sharing_on_nc1024(mode):
    w = synth.NC1024
    m = {"binary": B_, "graded": G_, "float": F_}[mode]
    b = w.bursts()
    chunks = [torch.from_numpy(w.chunk_data(i, b)).cuda() for i in range(4)]
    outs = []
    for flags in (0, g.FLAG_LEAF_SHARING):
        plan = g.Plan(w.freqs(), synth.NC_DT, w.dms(), 8, m, g.options(m, max_chunk=w.chunk, flags=flags))
        assert plan.stats().tree_kernel == (0 if flags else 1)
        planes = []
        for c in chunks:
            ne = plan.nemit_next(c.shape[0])
            out = torch.empty((w.ndm, max(ne, 1)), dtype=torch.float32 if m == F_ else torch.int32, device="cuda")
            plan.execute(c, out)
            planes.append(out[:, :ne].cpu())
        cands, rc = plan.candidates()
        assert rc == 0
        outs.append((planes, cands))
    for a, c in zip(outs[0][0], outs[1][0]):
        assert torch.equal(a, c)
    assert (outs[0][1] == outs[1][1]).all()
