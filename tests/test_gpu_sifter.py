"""GPU checks of the learned sifter: the tcgen05 BF16 GEMM against an FP32 reference of
the same BF16 operands, snippet extraction against the oracle, the network's logits and
every parameter gradient against the FP64 oracle, and learning on a separable task."""
import numpy as np
import pytest

from oracle import sifter as osf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_15361_gb300 as g  # noqa: E402


def _bf16(shape, gen, pitch=None):
    rows, cols = shape
    pitch = pitch or cols
    t = torch.zeros((rows, pitch), dtype=torch.bfloat16)
    t[:, :cols] = torch.randn((rows, cols), generator=gen).to(torch.bfloat16)
    return t.cuda()


@pytest.mark.parametrize("m,n,k,pitch,splits", [
    (128, 32, 64, None, 1),
    (300, 16, 100, 104, 1),      # ragged M and K (zero fill past K), N below the tile
    (256, 144, 192, None, 1),
    (1000, 9, 640, None, 4),     # split K with atomic accumulation
    (64, 1024, 128, None, 1),
    (128, 200, 4096, None, 7),
    (89600, 64, 192, None, 1),   # 700 output tiles: persistent CTAs, both TMEM buffers reused
    (5000, 144, 4096, None, 5),  # many tiles and split K together
])
def test_gemm_tc_matches_fp32_reference(m, n, k, pitch, splits):
    gen = torch.Generator().manual_seed(m * 7 + n * 3 + k)
    a = _bf16((m, k), gen, pitch)
    b = _bf16((n, k), gen, pitch)
    c, err = g.gemm_bf16(a, b, k=k, splits=splits)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = a[:, :k].double().cpu() @ b[:, :k].double().cpu().T
    scale = a[:, :k].double().abs().cpu() @ b[:, :k].double().abs().cpu().T
    diff = (c.double().cpu() - ref).abs()
    # FP32 accumulation of exact BF16 products: |error| <= K * 2^-23 * sum |a b| (loose)
    assert (diff <= 1e-6 + k * 2.0 ** -23 * scale).all(), float((diff / (scale + 1e-30)).max())


def test_snippets_match_oracle():
    rng = np.random.default_rng(4)
    plane = rng.normal(3.0, 2.0, size=(150, 3000)).astype(np.float32)
    rows = np.array([75, 0, 149, 10, 31, 120], dtype=np.int32)
    cols = np.array([1500, 0, 2999, 127, 5, 2900], dtype=np.int64)
    dp = torch.from_numpy(plane).cuda()
    out = g.snippets(dp, torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()).cpu().numpy()
    for i in range(len(rows)):
        exp = osf.snippet(plane.astype(np.float64), int(rows[i]), int(cols[i]))
        assert np.abs(out[i] - exp).max() <= 1e-5 * max(1.0, np.abs(exp).max())


def _bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def test_logits_and_gradients_match_oracle():
    """Gradient check against the CPU oracle. The oracle sees the same BF16-rounded snippets
    and weights the tensor cores read, and takes its pooling argmax on BF16-rounded
    activations as the kernels do; what remains is the BF16 rounding of activations and
    gradients between layers (2^-9 relative each, a few layers deep), so each parameter
    tensor's gradient must agree in direction (cosine >= 0.9999) and size (relative L2 error
    <= 1e-2)."""
    rng = np.random.default_rng(11)
    n = 6
    theta = osf.init_params(5)
    shapes = osf.param_shapes()
    offs = np.concatenate([[0], np.cumsum([int(np.prod(s)) for s in shapes])])
    for t in (1, 3, 5, 7, 9):  # non-zero biases
        theta[offs[t]:offs[t + 1]] = rng.normal(0, 0.05, offs[t + 1] - offs[t])
    x = rng.normal(size=(n, 64, 256))
    x[:3, 28:36, 100:160] += 3.0  # give some samples a bright patch
    y = np.array([1, 1, 1, 0, 0, 0], dtype=np.float64)
    sf = g.Sifter(max_batch=64, training=True, seed=1)
    sf.set_params(theta.astype(np.float32))
    assert np.array_equal(sf.get_params(), theta.astype(np.float32))
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    z_gpu = sf.forward(xd).cpu().numpy().astype(np.float64)
    loss_gpu, g_gpu = sf.gradients(xd, yd)
    g_gpu = g_gpu.cpu().numpy().astype(np.float64)
    # oracle on the rounded operands (weights BF16, biases FP32)
    th = theta.astype(np.float32).astype(np.float64)
    for t in (0, 2, 4, 6):
        th[offs[t]:offs[t + 1]] = _bf16_round(th[offs[t]:offs[t + 1]])
    xr = _bf16_round(x.astype(np.float32))
    # the pooling argmax is taken on BF16 activations on both sides (the kernel stores them so)
    z_ref, _ = osf.forward(th, xr, act=_bf16_round)
    loss_ref, g_ref = osf.gradients(th, xr, y, act=_bf16_round)
    assert np.abs(z_gpu - z_ref).max() <= 2e-2 * (1.0 + np.abs(z_ref).max()), (z_gpu, z_ref)
    assert abs(float(loss_gpu.item()) - loss_ref) <= 2e-2 * max(1.0, loss_ref)
    stats = []
    for t, s in enumerate(shapes):
        a, b = g_gpu[offs[t]:offs[t + 1]], g_ref[offs[t]:offs[t + 1]]
        nb = np.linalg.norm(b)
        cos = float(a @ b / (np.linalg.norm(a) * nb + 1e-300)) if nb > 0 else 1.0
        rel = float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))
        stats.append((t, s, round(cos, 5), round(rel, 4)))
    print("\nper-tensor gradient agreement (index, shape, cosine, relative L2 error):", stats)
    for t, s, cos, rel in stats:
        assert cos >= 0.9999 and rel <= 1e-2, (t, s, cos, rel)
    # element-wise, fc1 and fc2: the error of each gradient element is bounded relative to the
    # absolute-sum scale of its own sum (sum over the batch of |delta| x |activation|, the
    # standard bound for a rounded sum), taken from the oracle's intermediates; |delta| gets
    # a floor for the logit's own error (the output gradient moves by at most 1/4 of it, the
    # slope of the sigmoid, taken twice for margin), and a pooled feature an absolute
    # allowance of 2^-7 of the largest feature (a feature near zero is the small difference
    # of large conv sums, so its rounding error is relative to those, not to itself). 2^-6
    # covers the BF16 rounding of one operand (2^-9), a one-ulp difference of a BF16
    # activation (2^-8) and the FP32 accumulation. Hidden units whose pre-activation is too
    # close to zero for the ReLU decision to be stable are left to the per-tensor check above.
    _, (_, f, hpre, h) = osf.forward(th, xr, act=_bf16_round)
    p = osf.unpack(th)
    dz = (1.0 / (1.0 + np.exp(-z_ref)) - y) / n
    adz = np.abs(dz) + 0.5 * np.abs(z_gpu - z_ref).max() / n + 1e-6
    adh = np.outer(adz, np.abs(p[8][0])) * (hpre > 0)
    stable = (np.abs(hpre) > 1e-3 * np.abs(hpre).max()).all(axis=0)  # [128]
    af = np.abs(f) + 2.0 ** -7 * np.abs(f).max()
    scales = {8: (adz @ np.abs(h))[None, :], 9: np.array([adz.sum()]), 6: adh.T @ af, 7: adh.sum(axis=0)}
    for ti, m in scales.items():
        a = g_gpu[offs[ti]:offs[ti + 1]].reshape(m.shape)
        b = g_ref[offs[ti]:offs[ti + 1]].reshape(m.shape)
        ok = np.abs(a - b) <= 2.0 ** -6 * m + 1e-7
        if ti in (6, 7):
            ok |= ~(stable[:, None] if ti == 6 else stable)
        ratio = float((np.abs(a - b) / (2.0 ** -6 * m + 1e-7)).max())
        print(f"fc tensor {ti}: largest error / bound = {ratio:.3g}")
        assert ok.all(), (ti, np.argwhere(~ok)[:4], ratio)


def test_inference_sifter_matches_training_path():
    """A sifter built without training state runs the inference variants of the convolution
    kernels (no argmax, no transposed fc1 rows). With the same parameters its logits equal
    those of a training-capable sifter, whose training variants also write the argmax of
    every pooled cell: both take the same roundings in the same order, and only the split-K
    FP32 atomics of fc1 may reorder the last bits."""
    rng = np.random.default_rng(21)
    theta = osf.init_params(9).astype(np.float32)
    x = rng.normal(size=(70, 64, 256)).astype(np.float32)  # not a multiple of 64
    x[:20, 20:40, 60:200] += 2.5
    xd = torch.from_numpy(x).cuda()
    za = g.Sifter(max_batch=128, training=True, seed=1)
    zb = g.Sifter(max_batch=128, training=False, seed=1)
    za.set_params(theta)
    zb.set_params(theta)
    a = za.forward(xd).cpu().numpy()
    b = zb.forward(xd).cpu().numpy()
    assert np.abs(a).max() > 0.1
    assert np.allclose(a, b, rtol=1e-5, atol=1e-5), float(np.abs(a - b).max())


def test_training_learns_a_separable_task():
    """Bright sloped tracks (burst-like) against pure noise: Adam on the GPU drives the loss
    down and classifies held-out snippets."""
    gen = np.random.default_rng(2)

    def batch(n):
        x = gen.normal(size=(n, 64, 256)).astype(np.float32)
        y = (gen.random(n) < 0.5).astype(np.float32)
        for i in np.nonzero(y)[0]:
            t0 = gen.integers(60, 190)
            slope = gen.uniform(-1.0, 1.0)
            for r in range(64):
                c = int(t0 + slope * (r - 32))
                x[i, r, max(0, c - 2):c + 3] += 1.5
        return torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()

    sf = g.Sifter(max_batch=128, training=True, seed=3)
    xt, yt = batch(128)
    l0 = float(sf.gradients(xt, yt)[0].item())
    loss = torch.zeros(1, device="cuda")
    for _ in range(60):
        xb, yb = batch(128)
        sf.train_step(xb, yb, 1e-3, loss)
    sf.status()
    l1 = float(sf.gradients(xt, yt)[0].item())
    xv, yv = batch(128)
    acc = float(((sf.forward(xv) > 0).float() == yv).float().mean().item())
    assert l1 < 0.5 * l0 and acc >= 0.9, (l0, l1, acc)


def test_learned_sifter_beats_plain_sifter_at_equal_false_alarms():
    """Trained on snippets the pipeline itself produced (float mode, S/N > 5) from synthetic
    beams with bursts, zero-DM impulses and narrowband spikes, the network misses fewer
    bursts than the plain S/N >= 7 sifter at the plain sifter's false-alarm rate."""
    from paper_2606_15361_gb300 import sifter_data as sd
    tr = sd.concat([sd.make_run(3000 + s, n_burst=96) for s in range(40)])
    te = sd.concat([sd.make_run(93000 + s, n_burst=96) for s in range(12)])
    assert tr.label.sum() >= 500 and (tr.label == 0).sum() >= 2000
    sf = g.Sifter(max_batch=256, training=True, seed=2)
    sd.train(sf, tr, epochs=6, batch=256, lr=5e-4)
    r = sd.compare(sd.logits(sf, te.x, 256), te)
    print("\nlearned vs plain sifter:", {k: v for k, v in r.items() if k != "by_kind"})
    assert r["far_learned"] <= r["far_plain"]
    assert r["miss_learned"] < 0.75 * r["miss_plain"], r
