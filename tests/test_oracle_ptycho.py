"""Pins of the reconstruction oracle: least-squares updates against numpy.linalg.lstsq,
the single-position exact case, noiseless convergence to ground truth, NRMSE invariances."""
import numpy as np
import pytest

import oracle
from paper_2608_01746_b300 import synth


def _shift_ops(M, N, pos, field):
    """Rows of the linear map O -> stack_j(field * O_j), as a dense matrix."""
    rows = []
    for y, x in pos:
        for a in range(N):
            for b in range(N):
                r = np.zeros(M * M, dtype=np.complex128)
                r[(y + a) * M + (x + b)] = field[a, b]
                rows.append(r)
    return np.array(rows)


def test_object_update_is_least_squares():
    rng = np.random.default_rng(1)
    M, N = 10, 4
    pos = np.array([[0, 0], [0, 3], [3, 1], [6, 6], [5, 2]])
    probe = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    psi = rng.standard_normal((5, N, N)) + 1j * rng.standard_normal((5, N, N))
    obj0 = np.full((M, M), 7.0 + 0j)
    got = oracle.object_update(obj0, probe, pos, psi, 0.0)
    Amat = _shift_ops(M, N, pos, probe)
    sol, *_ = np.linalg.lstsq(Amat, psi.reshape(-1), rcond=None)
    cover = np.abs(Amat).sum(axis=0) > 0
    np.testing.assert_allclose(got.reshape(-1)[cover], sol[cover], rtol=1e-10, atol=1e-12)
    assert np.all(got.reshape(-1)[~cover] == 7.0)              # uncovered pixels unchanged


def test_probe_update_is_least_squares():
    rng = np.random.default_rng(2)
    M, N = 12, 4
    pos = np.array([[0, 0], [2, 5], [7, 3], [8, 8]])
    obj = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    psi = rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))
    got = oracle.probe_update(obj, np.zeros((N, N), complex), pos, psi, 0.0)
    # P -> stack_j(O_j * P): a diagonal block per position
    Amat = np.concatenate([np.diag(obj[y:y + N, x:x + N].reshape(-1)) for y, x in pos])
    sol, *_ = np.linalg.lstsq(Amat, psi.reshape(-1), rcond=None)
    np.testing.assert_allclose(got.reshape(-1), sol, rtol=1e-10, atol=1e-12)


def test_regulariser_scales_denominator():
    probe = np.full((2, 2), 2.0 + 0j)
    psi = np.ones((1, 2, 2), complex)
    out = oracle.object_update(np.zeros((4, 4), complex), probe, np.array([[1, 1]]), psi, 0.5)
    # den = |P|^2 = 4 everywhere in the patch, max 4: O = 2 / (4 + 0.5 * 4)
    np.testing.assert_allclose(out[1:3, 1:3], 2.0 / 6.0)


def test_single_position_update_is_exact():
    # One position, alpha = 0, probe nowhere zero: P * O_new = psi' exactly, so the new
    # exit wave satisfies the modulus constraint |F(P O_new)| = A.
    rng = np.random.default_rng(3)
    N = 16
    probe = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    obj = np.exp(1j * rng.uniform(-2, 2, (N, N)))
    A = rng.uniform(0.1, 3.0, (1, N, N))
    new, _, _ = oracle.iterate_once(obj, probe, np.array([[0, 0]]), A, 0.0, 0.0, False)
    np.testing.assert_allclose(np.abs(oracle.fft2u(probe * new)), A[0], rtol=1e-11)


def test_noiseless_known_probe_reaches_ground_truth():
    sc = synth.make_scan("tiny", noise=False, clip=False, times=(1.0,))
    M = sc["cfg"].M
    den = oracle.illumination(sc["probe"], sc["pos"], M)
    mask = den >= 0.1 * den.max()
    obj, _, errs = oracle.reconstruct(sc["intensity"], sc["pos"], np.ones((M, M), complex),
                                      sc["probe"], 800, alpha_O=1e-6, alpha_P=1e-6,
                                      probe_update_start=10**9)
    assert oracle.nrmse(obj, sc["obj"], mask) < 1e-3
    assert np.all(np.diff(errs) <= 1e-15)          # projections: error never increases
    assert errs[-1] < 1e-6


def test_nrmse_invariant_to_global_complex_scale():
    rng = np.random.default_rng(4)
    t = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    mask = np.ones((8, 8), bool)
    assert oracle.nrmse((0.3 - 2.0j) * t, t, mask) < 1e-14
    assert oracle.nrmse(t + 0.1, t, mask) > 0
