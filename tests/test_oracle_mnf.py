"""Pins of the MNF oracle (§3.4) against library routines, hand-worked values, closed forms
and the invariants the paper states (weights sum to one; single exposure is the linear case)."""
import os

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
from oracle.mnf import W_G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def scipy_blur_down(x):
    # scipy "mirror" mode is reflect-101 (d c b | a b c d | c b a)
    return ndi.correlate(x, np.outer(W_G, W_G), mode="mirror")[::2, ::2]


def scipy_upsample(x):
    n = x.shape[0]
    z = np.zeros((2 * n, 2 * n))
    z[::2, ::2] = x
    return ndi.correlate(z, 4.0 * np.outer(W_G, W_G), mode="mirror")


@pytest.mark.parametrize("n", [4, 8, 16, 64])
def test_pyramid_operators_match_scipy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n))
    np.testing.assert_allclose(oracle.blur_down(x), scipy_blur_down(x), atol=1e-13)
    np.testing.assert_allclose(oracle.upsample(x), scipy_upsample(x), atol=1e-13)


def test_pyramid_ramp_golden():
    txt = open(os.path.join(GOLDEN, "pyramid_1d_ramp.txt")).read().split("# fine_index")
    coarse = np.loadtxt(txt[0].splitlines()[-2:])
    fine = np.loadtxt(txt[1].splitlines()[1:])
    x = np.repeat(np.arange(16.0)[:, None], 16, axis=1)    # x[i, j] = i
    d = oracle.blur_down(x)
    for i, v in coarse:
        np.testing.assert_allclose(d[int(i), :], v, atol=1e-13)
    u = oracle.upsample(np.repeat(np.arange(8.0)[:, None], 8, axis=1))
    for m, v in fine:
        np.testing.assert_allclose(u[int(m), :], v, atol=1e-13)


def test_constant_preserved_by_every_operator():
    c = np.full((32, 32), 3.25)
    np.testing.assert_allclose(oracle.blur_down(c), 3.25, rtol=1e-15)
    np.testing.assert_allclose(oracle.upsample(c[:16, :16]), 3.25, rtol=1e-15)
    for g in oracle.gaussian_pyramid(c, 4):
        np.testing.assert_allclose(g, 3.25, rtol=1e-15)


def test_laplacian_perfect_reconstruction():
    rng = np.random.default_rng(11)
    x = rng.uniform(0, 1000, (64, 64))
    g = oracle.gaussian_pyramid(x, 5)
    lap = oracle.laplacian_pyramid(g)
    r = g[-1]
    for l in range(len(lap) - 1, -1, -1):
        r = oracle.upsample(r) + lap[l]
    np.testing.assert_allclose(r, x, rtol=1e-13, atol=1e-10)


def test_weights_closed_form_and_sum_to_one():
    clip, mu, sigma = 1000.0, 0.5, 0.2
    raw = np.array([[[500.0]], [[700.0]], [[5000.0]]])      # Ibar = 0.5, 0.7, 1 (clipped)
    W = oracle.exposure_weights(raw, clip, mu, sigma)
    w = np.array([1.0, np.exp(-0.5), np.exp(-0.25 / 0.08)])
    np.testing.assert_allclose(W[:, 0, 0], w / w.sum(), rtol=1e-14)
    rng = np.random.default_rng(2)
    raw = rng.integers(0, 5000, (5, 16, 16)).astype(float)
    W = oracle.exposure_weights(raw, 4095.0, mu, sigma)
    np.testing.assert_allclose(W.sum(axis=0), 1.0, rtol=1e-14)
    # ... and at every pyramid level (linearity of the Gaussian pyramid)
    g = [oracle.gaussian_pyramid(W[k], 4) for k in range(5)]
    for l in range(4):
        np.testing.assert_allclose(sum(gk[l] for gk in g), 1.0, rtol=1e-13)


def test_radiance_scaling():
    raw = np.ones((3, 2, 2))
    E = oracle.radiance(raw, [1.0, 10.0, 100.0])
    np.testing.assert_allclose(E[:, 0, 0], [100.0, 10.0, 1.0])
    np.testing.assert_allclose(oracle.radiance(raw, [1.0, 10.0, 100.0], "raw"), raw)


def test_quantiser():
    d = 0.5
    x = np.array([0.0, 0.24, 0.26, 1.25, 1.75, -0.75, 3.0])
    q = oracle.quantise(x, d)
    assert np.all(np.abs(q - x) <= d / 2 + 1e-15)
    assert np.allclose(q / d, np.rint(q / d))
    np.testing.assert_array_equal(q, [0.0, 0.0, 0.5, 1.0, 2.0, -1.0, 3.0])  # ties to even
    np.testing.assert_array_equal(oracle.quantise(x, 0.0), x)


@pytest.mark.parametrize("mode", ["mean", "sum", "weighted"])
def test_single_exposure_is_linear_case(mode):
    rng = np.random.default_rng(4)
    raw = rng.integers(0, 4096, (1, 32, 32)).astype(float)
    p = oracle.FuseParams(levels=4, clip=4095.0, delta0=0.0, base_mode=mode)
    np.testing.assert_allclose(oracle.mnf_position(raw, [7.0], p), raw[0], rtol=1e-12)


def test_identical_consistent_exposures():
    rng = np.random.default_rng(6)
    E = rng.uniform(0, 100, (32, 32))
    t = np.array([1.0, 2.0, 4.0])
    raw = E[None] * (t / t.max())[:, None, None]           # radiance-consistent, no clipping
    for mode in ("mean", "weighted"):
        p = oracle.FuseParams(levels=3, clip=1000.0, delta0=0.0, base_mode=mode)
        np.testing.assert_allclose(oracle.mnf_position(raw, t, p), E, rtol=1e-12)
    p = oracle.FuseParams(levels=3, clip=1000.0, delta0=0.0, base_mode="sum")
    top = oracle.gaussian_pyramid(E, 3)[-1]
    expect = E + 2.0 * oracle.upsample(oracle.upsample(top))
    np.testing.assert_allclose(oracle.mnf_position(raw, t, p), expect, rtol=1e-12)


def test_quantisation_error_bound_and_continuity():
    # U2 has non-negative taps summing to one, so it never grows the max-norm: the fused
    # output moves by at most sum_l K Delta_l / 2 when the quantiser is switched on.
    rng = np.random.default_rng(8)
    raw = rng.integers(0, 4096, (3, 32, 32)).astype(float)
    t = [1.0, 10.0, 100.0]
    base = oracle.mnf_position(raw, t, oracle.FuseParams(levels=4, delta0=0.0))
    for d0 in (2.0, 0.5, 1e-3):
        p = oracle.FuseParams(levels=4, delta0=d0)
        bound = sum(3 * p.delta(l) / 2 for l in range(3))
        diff = np.max(np.abs(oracle.mnf_position(raw, t, p) - base))
        assert diff <= bound * (1 + 1e-12)
        assert diff > 0
    small = oracle.mnf_position(raw, t, oracle.FuseParams(levels=4, delta0=1e-9))
    assert np.max(np.abs(small - base)) < 1e-7


def test_coefficient_ratios_returned():
    rng = np.random.default_rng(9)
    raw = rng.integers(0, 4096, (3, 16, 16)).astype(float)
    p = oracle.FuseParams(levels=3, delta0=0.5)
    fused, ratios = oracle.mnf_position(raw, [1.0, 10.0, 100.0], p, return_coeffs=True)
    assert [r.shape for r in ratios] == [(3, 16, 16), (3, 8, 8)]
    assert fused.shape == (16, 16)


def test_rejects_too_many_levels():
    with pytest.raises(ValueError):
        oracle.mnf_position(np.zeros((1, 16, 16)), [1.0], oracle.FuseParams(levels=4))


def test_sli_closed_forms():
    t = [1.0, 4.0, 16.0]
    clip = 1000.0
    # consistent counts (rate 10 per unit time, none saturated): every exposure says 10 * t_max
    raw = np.array([[[10.0]], [[40.0]], [[160.0]]])
    assert oracle.sli_position(raw, t, clip)[0, 0] == pytest.approx(160.0)
    # the long exposure saturates: only the first two count, (10 + 40) / (1 + 4) * 16
    raw = np.array([[[10.0]], [[40.0]], [[1000.0]]])
    assert oracle.sli_position(raw, t, clip)[0, 0] == pytest.approx(160.0)
    # all saturated: the shortest exposure's clipped rate, 1000 * 16 / 1
    raw = np.full((3, 1, 1), 1000.0)
    assert oracle.sli_position(raw, t, clip)[0, 0] == pytest.approx(16000.0)
    # single unsaturated exposure is the identity in its own units
    rng = np.random.default_rng(0)
    r1 = rng.integers(0, 999, (1, 8, 8)).astype(float)
    np.testing.assert_allclose(oracle.sli_position(r1, [2.0], clip), r1[0])
