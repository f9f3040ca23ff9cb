"""Pins of the warm-start network oracle: convolution against scipy's correlation and closed forms,
every gradient against central finite differences (brute force), Adam's first step in closed
form, and the input / target / stitching transforms on inputs with known answers."""
import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import cnn


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("mode", cnn.MODES)
def test_conv_matches_scipy_correlation(mode):
    x = _rand((2, 3, 8, 8), 1)
    w = _rand((4, 3, 3, 3), 2)
    b = _rand(4, 3)
    y = cnn.conv_forward(x, w, b, mode)
    xi = np.repeat(np.repeat(x, 2, 2), 2, 3) if mode == "up" else x
    for bb in range(2):
        for o in range(4):
            full = sum(ndi.correlate(xi[bb, c], w[o, c], mode="constant", cval=0.0) for c in range(3)) + b[o]
            ref = full[::2, ::2] if mode == "s2" else full
            np.testing.assert_allclose(y[bb, o], ref, atol=1e-12)


def test_conv_identity_kernels():
    x = _rand((1, 2, 6, 6), 4)
    w = np.zeros((2, 2, 3, 3))
    w[0, 0, 1, 1] = w[1, 1, 1, 1] = 1.0
    z = np.zeros(2)
    np.testing.assert_allclose(cnn.conv_forward(x, w, z, "s1"), x)
    np.testing.assert_allclose(cnn.conv_forward(x, w, z, "s2"), x[:, :, ::2, ::2])
    np.testing.assert_allclose(cnn.conv_forward(x, w, z, "up"), np.repeat(np.repeat(x, 2, 2), 2, 3))
    assert [cnn.out_side(8, m) for m in cnn.MODES] == [8, 4, 16]


@pytest.mark.parametrize("mode", cnn.MODES)
def test_conv_backward_finite_differences(mode):
    x = _rand((2, 2, 4, 4), 5)
    w = _rand((3, 2, 3, 3), 6)
    b = _rand(3, 7)
    dy = _rand(cnn.conv_forward(x, w, b, mode).shape, 8)
    dx, dw, db = cnn.conv_backward(x, w, dy, mode)
    f = lambda x_, w_, b_: float(np.sum(dy * cnn.conv_forward(x_, w_, b_, mode)))
    h = 1e-6
    rng = np.random.default_rng(9)
    for _ in range(6):
        i = tuple(rng.integers(0, s) for s in x.shape)
        e = np.zeros_like(x); e[i] = h
        assert (f(x + e, w, b) - f(x - e, w, b)) / (2 * h) == pytest.approx(dx[i], rel=1e-6, abs=1e-8)
        k = tuple(rng.integers(0, s) for s in w.shape)
        e = np.zeros_like(w); e[k] = h
        assert (f(x, w + e, b) - f(x, w - e, b)) / (2 * h) == pytest.approx(dw[k], rel=1e-6, abs=1e-8)
    e = np.zeros_like(b); e[1] = h
    assert (f(x, w, b + e) - f(x, w, b - e)) / (2 * h) == pytest.approx(db[1], rel=1e-6)


def test_network_gradient_finite_differences():
    layers = [(1, 3, "s2"), (3, 4, "s1"), (4, 2, "up")]
    rng = np.random.default_rng(10)
    params = [(0.5 * rng.standard_normal((o, c, 3, 3)), 0.1 * rng.standard_normal(o)) for c, o, _ in layers]
    x = rng.standard_normal((2, 1, 8, 8))
    y0, _, _ = cnn.network_forward(layers, params, x)
    t = rng.standard_normal(y0.shape)

    def loss(ps):
        y, _, _ = cnn.network_forward(layers, ps, x)
        return cnn.mse(y, t)[0]

    y, acts, pre = cnn.network_forward(layers, params, x)
    L, dout = cnn.mse(y, t)
    grads, _ = cnn.network_backward(layers, params, acts, pre, dout)
    h = 1e-6
    for li in range(3):
        for _ in range(3):
            k = tuple(rng.integers(0, s) for s in params[li][0].shape)
            ps_p = [(w.copy(), b.copy()) for w, b in params]
            ps_m = [(w.copy(), b.copy()) for w, b in params]
            ps_p[li][0][k] += h
            ps_m[li][0][k] -= h
            fd = (loss(ps_p) - loss(ps_m)) / (2 * h)
            assert fd == pytest.approx(grads[li][0][k], rel=1e-5, abs=1e-9)
        ps_p = [(w.copy(), b.copy()) for w, b in params]
        ps_m = [(w.copy(), b.copy()) for w, b in params]
        ps_p[li][1][0] += h
        ps_m[li][1][0] -= h
        assert (loss(ps_p) - loss(ps_m)) / (2 * h) == pytest.approx(grads[li][1][0], rel=1e-5, abs=1e-9)


def test_mse_gradient_closed_form():
    y = np.array([1.0, 2.0, 4.0])
    t = np.array([0.0, 2.0, 1.0])
    L, g = cnn.mse(y, t)
    assert L == pytest.approx((1 + 0 + 9) / 3)
    np.testing.assert_allclose(g, [2 / 3, 0, 2])


def test_adam_first_step_is_a_signed_step():
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    w1, m, v = cnn.adam_step(w, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    np.testing.assert_allclose(w1, w - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_preprocess_and_targets_closed_forms():
    f = np.full((2, 8, 8), 3.0)
    f[1] = -1.0                                   # negative fused values clip to zero
    x = cnn.preprocess(f)
    assert x.shape == (2, 1, 4, 4)
    np.testing.assert_allclose(x[0], np.log1p(12.0) / 10)
    np.testing.assert_allclose(x[1], 0.0)
    obj = np.add.outer(np.arange(16.0), 1j * np.arange(16.0))   # re = row, im = column
    t = cnn.targets(obj, [(0, 0), (4, 8)], 8)
    assert t.shape == (2, 2, 2, 2)
    np.testing.assert_allclose(t[0, 0], [[1.5, 1.5], [5.5, 5.5]])
    np.testing.assert_allclose(t[1, 1], [[9.5, 13.5], [9.5, 13.5]])


def test_stitch_constant_and_uncovered():
    N, M = 16, 64
    probe = np.ones((N, N), complex)
    pos = [(0, 0), (8, 8), (16, 12)]
    pred = np.zeros((3, 2, 4, 4))
    pred[:, 0], pred[:, 1] = 2.0, -1.0
    o = cnn.stitch(pred, pos, probe, M)
    assert o.shape == (M, M)
    np.testing.assert_allclose(o[0:14, 0:14], 2 - 1j)          # bilinear footprint inside patch 0
    np.testing.assert_allclose(o[48:, 48:], 1.0)                # never covered: the flat object


def test_stitch_bilinear_reproduces_a_coarse_ramp():
    N, M = 16, 64
    probe = np.ones((N, N), complex)
    pos = [(y, x) for y in range(0, M - N + 1, 16) for x in range(0, M - N + 1, 16)]
    pred = np.zeros((len(pos), 2, 4, 4))
    for j, (y, x) in enumerate(pos):
        pred[j, 0] = (y // 4 + np.arange(4))[:, None] * np.ones(4)[None]   # coarse value = coarse row
    o = cnn.stitch(pred, pos, probe, M)
    rows = np.arange(2, M - 2)
    np.testing.assert_allclose(o.real[rows, 20], (rows - 1.5) / 4.0, atol=1e-12)
