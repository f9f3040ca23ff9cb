"""Degenerate reconstructions through the C ABI against the FP64 oracle: one position whose
patch is the whole object (every object tile's list has one entry), two positions at opposite
corners of a barely larger object (tiles covered once, twice and never), and fewer positions
than exit-wave CTAs.  Inputs are seeded non-negative intensities (the reconstruction accepts
any), not fusion output, so that the cases stay tiny."""
import numpy as np
import pytest

import oracle
from tests.parity_helpers import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_01746_b300 import api as a
    a.lib()
    return a


def case(N, M, pos, seed):
    rng = np.random.default_rng(seed)
    J = len(pos)
    fused = (rng.gamma(2.0, 50.0, size=(J, N, N))).astype(np.float32)
    yy, xx = np.mgrid[:N, :N] - (N - 1) / 2.0
    probe = np.exp(-(yy ** 2 + xx ** 2) / (2 * (N / 5.0) ** 2)) * np.exp(1j * 0.3 * rng.standard_normal((N, N)))
    obj0 = 1.0 + 0.1 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)))
    return fused, np.asarray(pos, np.int32), obj0.astype(np.complex64), probe.astype(np.complex64)


def run(api, fused, pos, obj0, probe0, n_iter):
    h = api.ptycho_init(torch.from_numpy(fused).cuda(), pos, obj0, probe0, probe_update_start=0)
    errs = api.ptycho_iterate(h, n_iter)
    o, p = api.ptycho_get_object(h), api.ptycho_get_probe(h)
    api.ptycho_destroy(h)
    ro, rp, re = oracle.reconstruct(fused.astype(np.float64), pos, obj0.astype(np.complex128),
                                    probe0.astype(np.complex128), n_iter, 1e-3, 1e-3, 0)
    return (o, p, errs), (ro, rp, re)


@pytest.mark.parametrize("N", [64, 128, 256])
def test_single_position_covering_the_object(api, N):
    fused, pos, obj0, probe0 = case(N, N, [(0, 0)], seed=N)
    (o, p, e), (ro, rp, re) = run(api, fused, pos, obj0, probe0, 3)
    assert rel_l2(o, ro) <= 1e-5 and rel_l2(p, rp) <= 1e-5
    np.testing.assert_allclose(e, re, rtol=1e-5)


@pytest.mark.parametrize("N,M", [(64, 100), (256, 300)])
def test_two_positions_at_opposite_corners(api, N, M):
    # the corners leave object pixels covered by no patch (they keep their initial value)
    fused, pos, obj0, probe0 = case(N, M, [(0, 0), (M - N, M - N)], seed=M)
    (o, p, e), (ro, rp, re) = run(api, fused, pos, obj0, probe0, 3)
    assert rel_l2(o, ro) <= 1e-5 and rel_l2(p, rp) <= 1e-5
    np.testing.assert_allclose(e, re, rtol=1e-5)
    assert np.array_equal(o[0, M - 1], obj0[0, M - 1])        # covered by neither patch


def test_fewer_positions_than_ctas(api):
    # 7 positions of N = 256 on a 400^2 object: the persistent grid shrinks to the positions
    rng = np.random.default_rng(3)
    pos = [(int(y), int(x)) for y, x in rng.integers(0, 400 - 256 + 1, size=(7, 2))]
    fused, pos, obj0, probe0 = case(256, 400, pos, seed=7)
    (o, p, e), (ro, rp, re) = run(api, fused, pos, obj0, probe0, 3)
    assert rel_l2(o, ro) <= 1e-5 and rel_l2(p, rp) <= 1e-5
    np.testing.assert_allclose(e, re, rtol=1e-5)
