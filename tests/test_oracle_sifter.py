"""Pins for oracle.sifter: convolution against scipy's correlate2d, pooling against brute
force, backpropagation against central finite differences, the loss at known points, and
the snippet standardisation on hand-made planes."""
import numpy as np
import pytest

from oracle import sifter as osf

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv3x3_matches_correlate2d():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 9, 11))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = osf.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = sum(scipy_signal.correlate2d(x[n, i], w[o, i], mode="same", boundary="fill") for i in range(3))
            assert np.allclose(y[n, o], ref + b[o], rtol=1e-12, atol=1e-12)


def test_maxpool_brute_force_and_ties():
    rng = np.random.default_rng(2)
    x = rng.integers(0, 3, size=(2, 3, 6, 8)).astype(float)  # many ties
    y, a = osf.maxpool2(x)
    for n in range(2):
        for c in range(3):
            for i in range(3):
                for j in range(4):
                    blk = [x[n, c, 2 * i, 2 * j], x[n, c, 2 * i, 2 * j + 1], x[n, c, 2 * i + 1, 2 * j],
                           x[n, c, 2 * i + 1, 2 * j + 1]]
                    assert y[n, c, i, j] == max(blk)
                    assert a[n, c, i, j] == blk.index(max(blk))  # first maximum
    g = osf.maxpool2_backward(np.ones_like(y), a, x.shape)
    assert g.sum() == y.size and set(np.unique(g)) <= {0.0, 1.0}


def test_loss_known_points():
    assert osf.loss([0.0], [1.0]) == pytest.approx(np.log(2.0))
    assert osf.loss([0.0, 0.0], [0.0, 1.0]) == pytest.approx(np.log(2.0))
    assert osf.loss([50.0], [1.0]) == pytest.approx(np.exp(-50.0), rel=1e-6)
    assert osf.loss([-50.0], [1.0]) == pytest.approx(50.0, rel=1e-12)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(3)
    theta = osf.init_params(7)
    theta[np.concatenate([[16 * 9 + i for i in range(16)]])] = rng.normal(0, 0.1, 16)  # nonzero b1
    x = rng.normal(size=(2, 64, 256))
    y = np.array([1.0, 0.0])
    _, g = osf.gradients(theta, x, y)
    shapes = osf.param_shapes()
    offs = np.concatenate([[0], np.cumsum([int(np.prod(s)) for s in shapes])])
    picks = []
    for t in range(len(shapes)):
        n = offs[t + 1] - offs[t]
        picks += list(offs[t] + rng.choice(n, size=min(3, n), replace=False))
    # the largest-gradient entry of every tensor, so each check is well above the FD noise
    picks += [offs[t] + int(np.argmax(np.abs(g[offs[t]:offs[t + 1]]))) for t in range(len(shapes))]
    def decisions(t):
        # every ReLU sign and pooling choice of the forward pass
        _, (cache, _, hpre, _) = osf.forward(t, x)
        return [np.concatenate([(c[1] > 0).ravel(), c[3].ravel()]) for c in cache] + [hpre > 0]

    eps = 1e-7
    checked = 0
    for i in picks:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        if any((a != b).any() for a, b in zip(decisions(tp), decisions(tm))):
            continue  # the step crosses a ReLU or pooling kink: the loss is not differentiable there
        fd = (osf.loss(osf.forward(tp, x)[0], y) - osf.loss(osf.forward(tm, x)[0], y)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])
        checked += 1
    assert checked >= len(picks) - 3
    assert osf.num_params() == theta.size == 2120705


def test_snippet_standardisation_and_edges():
    plane = np.zeros((100, 1000))
    plane[50, 500] = 10.0
    s = osf.snippet(plane, 50, 500)
    assert s.shape == (64, 256)
    n = 64 * 256
    mu, sd = 10.0 / n, np.sqrt(100.0 / n - (10.0 / n) ** 2)
    assert s[32, 128] == pytest.approx((10.0 - mu) / sd)
    assert s[0, 0] == pytest.approx(-mu / sd)
    assert abs(s.mean()) < 1e-12 and s.std() == pytest.approx(1.0)
    # corner: rows below 0 and columns below 0 are missing and stay 0
    s2 = osf.snippet(plane + np.arange(1000)[None, :], 3, 10)
    assert (s2[:29] == 0).all() and (s2[:, :118] == 0).all()
    present = s2[29:, 118:]
    assert abs(present.mean()) < 1e-12 and present.std() == pytest.approx(1.0)
    # a constant plane standardises to zeros (std 0 -> 1)
    assert not osf.snippet(np.full((70, 300), 3.0), 35, 150).any()
