"""ePIE by colour on the GPU against the FP64 oracle, through the C ABI."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2608_01746_b300 import synth
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


def noisy_start(M, seed=0):
    rng = np.random.default_rng(seed)
    return (1.0 + 0.1 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)))).astype(np.complex64)


def sensitivity(fused, pos, obj0, probe0, n_iter, pus):
    a = oracle.epie_by_colour(fused, pos, obj0, probe0, n_iter, probe_update_start=pus)
    pert = obj0 * (1.0 + 2.0 ** -24 * np.random.default_rng(99).standard_normal(obj0.shape))
    b = oracle.epie_by_colour(fused, pos, pert, probe0, n_iter, probe_update_start=pus)
    return max(rel_l2(b[0], a[0]), rel_l2(b[1], a[1])), a


def check(api, sc, fused32, n_iter, pus):
    M = sc["cfg"].M
    obj0 = noisy_start(M)
    probe0 = sc["probe"].astype(np.complex64)
    f64 = fused32.astype(np.float64)
    sens, (ro, rp, re) = sensitivity(f64, sc["pos"], obj0.astype(np.complex128), probe0.astype(np.complex128),
                                     n_iter, pus)
    assert sens <= 2e-6                      # well conditioned at FP32 resolution
    h = api.ptycho_init(torch.from_numpy(fused32).cuda(), sc["pos"], obj0, probe0, probe_update_start=pus,
                        algorithm="epie_colour")
    col, ncol = api.ptycho_get_colouring(h)
    ref_col = oracle.greedy_colouring(sc["pos"], sc["cfg"].N)
    assert np.array_equal(col, ref_col) and ncol == ref_col.max() + 1
    e = api.ptycho_iterate(h, n_iter)
    o = api.ptycho_get_object(h)
    p = api.ptycho_get_probe(h)
    api.ptycho_destroy(h)
    assert rel_l2(o, ro) <= 1e-5
    assert rel_l2(p, rp) <= 1e-5
    np.testing.assert_allclose(e, re, rtol=1e-5)


def fused_for(name):
    sc = synth.make_scan(name)
    cfg = sc["cfg"]
    p = oracle.FuseParams(levels=cfg.levels, clip=float(cfg.clip))
    return sc, oracle.mnf_stack(sc["raw"], sc["times"], p).astype(np.float32)


@pytest.mark.parametrize("pus", [0, 10**6])
def test_epie_tiny_matches_oracle(api, pus):
    sc, fused = fused_for("tiny")
    check(api, sc, fused, 10, pus)


def test_epie_mid_fixed_probe_matches_oracle(api):
    sc, fused = fused_for("mid")
    check(api, sc, fused, 1, 10**6)


def test_epie_128_matches_oracle(api):
    """N = 128 (8 x 16 group FFTs), list form of the exit-wave kernel: four disjoint patches (one
    colour; on the overlapped 5 x 5 scan every position is its own colour and 25 sequential unit
    steps amplify a 2^-24 perturbation of the start beyond FP32 reach), two iterations."""
    sc, fused = fused_for("mid128")
    sc = dict(sc)
    sc["pos"] = np.array([[0, 0], [0, 128], [128, 0], [128, 128]], np.int32)
    check(api, sc, fused[:4].copy(), 2, 0)


def test_epie_256_matches_oracle(api):
    """Colour lists through the N = 256 TMA exit-wave kernel: lab geometry, 60 positions."""
    cfg = dataclasses.replace(synth.CONFIGS["lab"], J=60, name="lab60")
    sc = synth.make_scan_torch(cfg, seed=61, device="cuda")
    params = api.fuse_params(levels=cfg.levels, clip=float(cfg.clip))
    fused = api.fuse_stack(sc["raw"], cfg.times, params)
    torch.cuda.synchronize()
    fused = fused.cpu().numpy()
    del sc["raw"]
    check(api, sc, fused, 1, 10**6)


def test_colouring_of_the_lab_scan(api):
    cfg = synth.CONFIGS["lab"]
    pos = synth.spiral_positions(cfg.M, cfg.N, cfg.J)
    fused = torch.zeros((cfg.J, cfg.N, cfg.N), dtype=torch.float32, device="cuda")
    h = api.ptycho_init(fused, pos, np.ones((cfg.M, cfg.M), np.complex64),
                        np.ones((cfg.N, cfg.N), np.complex64), algorithm="epie_colour")
    col, ncol = api.ptycho_get_colouring(h)
    api.ptycho_destroy(h)
    assert np.array_equal(col, oracle.greedy_colouring(pos, cfg.N))
