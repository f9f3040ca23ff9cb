"""Pins of the oracle's forward model and modulus constraint (§3.3, Eqs. 2-3) against
brute force, hand-worked values and closed forms."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_dft2(x):
    """Direct O(N^4) double sum of the unitary 2-D DFT definition."""
    n1, n2 = x.shape
    out = np.zeros((n1, n2), dtype=np.complex128)
    for k1 in range(n1):
        for k2 in range(n2):
            acc = 0j
            for a in range(n1):
                for b in range(n2):
                    acc += x[a, b] * np.exp(-2j * np.pi * (k1 * a / n1 + k2 * b / n2))
            out[k1, k2] = acc / np.sqrt(n1 * n2)
    return out


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16])
def test_fft_matches_brute_force(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    ref = brute_dft2(x)
    got = oracle.fft2u(x)
    assert np.linalg.norm(got - ref) <= 1e-12 * max(1.0, np.linalg.norm(ref))


def test_fft_golden_2x2():
    rows = np.loadtxt(os.path.join(GOLDEN, "dft_2x2.txt"))
    x = np.array([[1.0, 2.0], [3.0, 4.0]])
    X = oracle.fft2u(x)
    for k1, k2, re, im in rows:
        assert X[int(k1), int(k2)] == pytest.approx(re + 1j * im, abs=1e-14)


def test_fft_impulse_closed_form():
    # an impulse at (1, 0) has transform exp(-2 pi i k1 / 4) / 4 = (-i)^k1 / 4
    x = np.zeros((4, 4))
    x[1, 0] = 1.0
    X = oracle.fft2u(x)
    k1 = np.arange(4)[:, None] * np.ones((1, 4))
    np.testing.assert_allclose(X, ((-1j) ** k1) / 4.0, atol=1e-15)


def test_parseval_and_round_trip():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))
    X = oracle.fft2u(x)
    assert np.linalg.norm(X) == pytest.approx(np.linalg.norm(x), rel=1e-13)
    np.testing.assert_allclose(oracle.ifft2u(X), x, atol=1e-13)


def test_modulus_projection_properties():
    rng = np.random.default_rng(3)
    Psi = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    Psi[2, 3] = 0.0
    A = rng.uniform(0.0, 2.0, (16, 16))
    P1 = oracle.modulus_projection(Psi, A)
    np.testing.assert_allclose(np.abs(P1), A, rtol=1e-14)        # |Psi'| = A exactly
    np.testing.assert_allclose(oracle.modulus_projection(P1, A), P1, rtol=1e-14, atol=1e-15)
    assert P1[2, 3] == A[2, 3] + 0j                                # zero guard
    nz = np.abs(Psi) > 0                                           # phase kept
    np.testing.assert_allclose(np.angle(P1[nz & (A > 0)]), np.angle(Psi[nz & (A > 0)]),
                               atol=1e-13)


def test_amplitudes_move_centred_dc_to_origin():
    fused = np.zeros((8, 8))
    fused[4, 4] = 9.0           # DC of a centred detector pattern
    fused[4, 5] = -1.0          # negative fused values clamp to zero
    A = oracle.amplitudes(fused)
    assert A[0, 0] == 3.0
    assert A[0, 1] == 0.0
    assert np.count_nonzero(A) == 1


def test_fourier_error_scale_case():
    # Exit waves twice the consistent ones give |Psi| = 2A, so the normalised error is 1.
    rng = np.random.default_rng(5)
    M, N = 24, 8
    obj = np.exp(1j * rng.uniform(-1, 1, (M, M)))
    probe = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    pos = np.array([[0, 0], [4, 8], [16, 16]])
    A = np.stack([np.abs(oracle.fft2u(probe * obj[y:y + N, x:x + N])) for y, x in pos])
    _, _, e0 = oracle.iterate_once(obj, probe, pos, A, 0.0, 0.0, False)
    assert e0 == pytest.approx(0.0, abs=1e-20)
    _, _, e1 = oracle.iterate_once(2 * obj, probe, pos, A, 0.0, 0.0, False)
    assert e1 / np.sum(A * A) == pytest.approx(1.0, rel=1e-12)
