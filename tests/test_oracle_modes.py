"""Pins of the mixed-state (broadband, Eq. 4 with a discrete spectrum) oracle."""
import numpy as np
import pytest

import oracle
from paper_2608_01746_b300 import synth


def test_single_mode_reduces_to_coherent_iteration():
    sc = synth.make_scan("tiny")
    M = sc["cfg"].M
    p = oracle.FuseParams(levels=3, clip=4095.0)
    A = oracle.amplitudes(oracle.mnf_stack(sc["raw"], sc["times"], p))
    rng = np.random.default_rng(0)
    obj = 1 + 0.1 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)))
    o1, p1, e1 = oracle.iterate_once(obj, sc["probe"], sc["pos"], A, 1e-3, 1e-3, True)
    o2, p2, e2 = oracle.iterate_once_modes(obj, sc["probe"][None], sc["pos"], A, 1e-3, 1e-3, True)
    np.testing.assert_allclose(o2, o1, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(p2[0], p1, rtol=1e-12, atol=1e-14)
    assert e2 == pytest.approx(e1, rel=1e-12)


def test_modes_modulus_projection():
    rng = np.random.default_rng(1)
    Psi = rng.standard_normal((4, 8, 8)) + 1j * rng.standard_normal((4, 8, 8))
    Psi[:, 2, 2] = 0.0
    A = rng.uniform(0.1, 3.0, (8, 8))
    out = oracle.modes_modulus_projection(Psi, A)
    np.testing.assert_allclose(np.sum(np.abs(out) ** 2, axis=0), A ** 2, rtol=1e-13)
    np.testing.assert_allclose(oracle.modes_modulus_projection(out, A), out, rtol=1e-13, atol=1e-15)
    assert out[0, 2, 2] == A[2, 2] and np.all(out[1:, 2, 2] == 0)
    # every mode keeps its phase and the modes keep their relative powers
    nz = np.ones((8, 8), bool)
    nz[2, 2] = False
    ratio = np.abs(out[:, nz]) ** 2 / np.sum(np.abs(out[:, nz]) ** 2, axis=0)
    ratio0 = np.abs(Psi[:, nz]) ** 2 / np.sum(np.abs(Psi[:, nz]) ** 2, axis=0)
    np.testing.assert_allclose(ratio, ratio0, rtol=1e-12)


def test_consistent_state_is_a_fixed_point():
    # Data generated from (O, P_m) exactly: the projection changes nothing, so with alpha = 0 the
    # object and every probe mode come back unchanged.
    rng = np.random.default_rng(2)
    M, N, Q = 24, 8, 3
    obj = np.exp(1j * rng.uniform(-1, 1, (M, M))) * rng.uniform(0.5, 1, (M, M))
    probes = rng.standard_normal((Q, N, N)) + 1j * rng.standard_normal((Q, N, N))
    pos = np.array([[0, 0], [0, 8], [8, 4], [16, 16], [12, 2], [4, 14]])
    A = np.stack([np.sqrt(np.sum(np.abs(oracle.fft2u(probes * obj[y:y + N, x:x + N][None])) ** 2, axis=0))
                  for y, x in pos])
    o, p, e = oracle.iterate_once_modes(obj, probes, pos, A, 0.0, 0.0, True)
    cover = oracle.illumination(probes[0], pos, M) > 0
    np.testing.assert_allclose(o[cover], obj[cover], rtol=1e-10)
    np.testing.assert_allclose(p, probes, rtol=1e-10, atol=1e-12)
    assert e == pytest.approx(0.0, abs=1e-18)


def test_generator_sums_mode_intensities():
    sc = synth.make_scan("mixed_small", noise=False, clip=False)
    probes = sc["probe"]
    assert probes.shape == (8, 64, 64)
    y, x = sc["pos"][5]
    f = np.fft.fftshift(np.fft.fft2(probes * sc["obj"][y:y + 64, x:x + 64][None], norm="ortho"), axes=(-2, -1))
    np.testing.assert_allclose(sc["intensity"][5], np.sum(np.abs(f) ** 2, axis=0), rtol=1e-12)
    # modes are magnified copies: mode radius grows with the wavelength
    w = np.sum(np.abs(probes) ** 2, axis=(1, 2))
    assert np.all(np.diff(w) > 0)


def test_noiseless_known_modes_reach_ground_truth():
    cfg = synth.CONFIGS["tiny"]
    import dataclasses
    cfg = dataclasses.replace(cfg, modes=3, name="tiny3")
    sc = synth.make_scan(cfg, seed=7, noise=False, clip=False, times=(1.0,))
    M = cfg.M
    den = oracle.illumination(sc["probe"][0], sc["pos"], M)
    mask = den >= 0.1 * den.max()
    obj, _, errs = oracle.reconstruct_modes(sc["intensity"], sc["pos"], np.ones((M, M), complex),
                                            sc["probe"], 600, alpha_O=1e-6, alpha_P=1e-6,
                                            probe_update_start=10**9)
    assert oracle.nrmse(obj, sc["obj"], mask) < 2e-2
    assert errs[-1] < 1e-3 * errs[0]
