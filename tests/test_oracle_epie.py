"""Pins of the ePIE-by-colour oracle: the colouring is a proper colouring built greedily, a
single position per colour is plain sequential ePIE, consistent data is a fixed point, and
noiseless known-probe data converge."""
import numpy as np
import pytest

import oracle
from paper_2608_01746_b300 import synth


def overlaps(a, b, N):
    return abs(int(a[0]) - int(b[0])) < N and abs(int(a[1]) - int(b[1])) < N


def test_colouring_is_proper_and_greedy():
    pos = synth.make_scan("small")["pos"]
    N = 64
    col = oracle.greedy_colouring(pos, N)
    for i in range(len(pos)):
        for j in range(i):
            if overlaps(pos[i], pos[j], N):
                assert col[i] != col[j]
        # greedy: every smaller colour is used by an earlier overlapping position
        used = {int(col[k]) for k in range(i) if overlaps(pos[i], pos[k], N)}
        assert all(c in used for c in range(int(col[i])))
    # a grid whose step equals the patch size needs one colour
    grid = np.array([[y, x] for y in (0, 8, 16) for x in (0, 8, 16)])
    assert np.all(oracle.greedy_colouring(grid, 8) == 0)


def test_single_position_is_one_epie_step():
    rng = np.random.default_rng(1)
    N, M = 16, 24
    probe = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    obj = np.exp(1j * rng.uniform(-1, 1, (M, M)))
    A = rng.uniform(0.5, 2.0, (1, N, N))
    pos = np.array([[3, 5]])
    o, p, e = oracle.epie_by_colour(None, pos, obj, probe, 1, A=A)
    psi = probe * obj[3:19, 5:21]
    d = oracle.ifft2u(oracle.modulus_projection(oracle.fft2u(psi), A[0])) - psi
    expect_o = obj.copy()
    expect_o[3:19, 5:21] += np.conj(probe) * d / np.max(np.abs(probe) ** 2)
    expect_p = probe + np.conj(obj[3:19, 5:21]) * d / np.max(np.abs(obj[3:19, 5:21]) ** 2)
    np.testing.assert_allclose(o, expect_o, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(p, expect_p, rtol=1e-12, atol=1e-14)


def test_consistent_data_is_fixed_point():
    sc = synth.make_scan("tiny", noise=False, clip=False, times=(1.0,))
    A = oracle.amplitudes(sc["intensity"])
    o, p, e = oracle.epie_by_colour(None, sc["pos"], sc["obj"], sc["probe"], 2, A=A)
    np.testing.assert_allclose(o, sc["obj"], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(p, sc["probe"], rtol=1e-10, atol=1e-12)
    assert e[0] < 1e-20


def test_noiseless_known_probe_converges():
    sc = synth.make_scan("tiny", noise=False, clip=False, times=(1.0,))
    M = sc["cfg"].M
    den = oracle.illumination(sc["probe"], sc["pos"], M)
    mask = den >= 0.1 * den.max()
    o, _, errs = oracle.epie_by_colour(sc["intensity"], sc["pos"], np.ones((M, M), complex), sc["probe"],
                                       150, probe_update_start=10**9)
    assert oracle.nrmse(o, sc["obj"], mask) < 1e-2
    assert errs[-1] < 1e-3 * errs[0]
