"""Mixed-state reconstruction (Eq. 4 with a discrete spectrum, 8 probe modes): CUDA FP32 vs the
FP64 oracle through the C ABI, fed the same fused intensities (the oracle's fusion, in FP32)."""
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


def run(api, sc, fused32, n_iter, pus):
    M = sc["cfg"].M
    obj0 = noisy_start(M)
    probes0 = sc["probe"].astype(np.complex64)
    h = api.ptycho_init(torch.from_numpy(fused32).cuda(), sc["pos"], obj0, probes0, probe_update_start=pus)
    e = api.ptycho_iterate(h, n_iter)
    o = api.ptycho_get_object(h)
    p = api.ptycho_get_probe(h)
    api.ptycho_destroy(h)
    ro, rp, re = oracle.reconstruct_modes(fused32.astype(np.float64), sc["pos"], obj0.astype(np.complex128),
                                          probes0.astype(np.complex128), n_iter, 1e-3, 1e-3, pus)
    return (o, p, e), (ro, rp, re)


@pytest.mark.parametrize("n_iter,pus", [(10, 0), (10, 10**6)])
def test_mixed_state_small_matches_oracle(api, n_iter, pus):
    sc = synth.make_scan("mixed_small")
    cfg = sc["cfg"]
    p = oracle.FuseParams(levels=cfg.levels, clip=float(cfg.clip))
    fused = oracle.mnf_stack(sc["raw"], sc["times"], p).astype(np.float32)
    (o, pr, e), (ro, rp, re) = run(api, sc, fused, n_iter, pus)
    assert pr.shape == (8, 64, 64)
    assert rel_l2(o, ro) <= 1e-5
    assert rel_l2(pr, rp) <= 1e-5
    np.testing.assert_allclose(e, re, rtol=1e-5)


def test_mixed_state_workload_each_iteration_matches_oracle(api):
    """The mixed-state workload as specified (the small scan with 8 probe modes, 100 iterations
    from a flat object, probe updates on), followed step by step: after every GPU iteration the
    FP64 oracle takes one iteration from the GPU's own object and probe modes, and the GPU's next
    state must agree with it (bound 1e-5 on the first step from the flat object, 1e-6 after)."""
    sc = synth.make_scan("mixed_small")
    cfg = sc["cfg"]
    p = oracle.FuseParams(levels=cfg.levels, clip=float(cfg.clip))
    fused = oracle.mnf_stack(sc["raw"], sc["times"], p).astype(np.float32)
    f64 = fused.astype(np.float64)
    A = oracle.amplitudes(f64)
    M = cfg.M
    o0 = np.ones((M, M), np.complex64)
    p0 = sc["probe"].astype(np.complex64)
    h = api.ptycho_init(torch.from_numpy(fused).cuda(), sc["pos"], o0, p0, probe_update_start=0)
    obj, probes = o0.astype(np.complex128), p0.astype(np.complex128)
    worst = [0.0, 0.0]
    n_iter = 100                                   # the mixed-state workload's iteration count
    for k in range(n_iter):
        e = api.ptycho_iterate(h, 1)
        go, gp = api.ptycho_get_object(h), api.ptycho_get_probe(h)
        ro, rp, re = oracle.reconstruct_modes(f64, sc["pos"], obj, probes, 1, 1e-3, 1e-3, 0, A=A)
        d = max(rel_l2(go, ro), rel_l2(gp, rp))
        assert d <= (1e-5 if k == 0 else 1e-6), (k, d)
        assert abs(e[0] - re[0]) <= 1e-6 * re[0], k
        worst[min(k, 1)] = max(worst[min(k, 1)], d)
        obj, probes = go.astype(np.complex128), gp.astype(np.complex128)
    api.ptycho_destroy(h)
    print(f"first step {worst[0]:.2e}, worst later step {worst[1]:.2e} over {n_iter} iterations")


@pytest.mark.parametrize("modes", [2, 4, 8])
def test_mixed_state_256_matches_oracle(api, modes):
    """The N = 256 forward / mode-scale / inverse kernels: lab geometry, 120 positions, two
    iterations, for several mode counts (the scale kernel and the inverse pass's scaling are
    compiled per mode count)."""
    cfg = dataclasses.replace(synth.CONFIGS["mixed"], J=120, modes=modes, name="mixed120")
    sc = synth.make_scan_torch(cfg, seed=77, device="cuda")
    params = api.fuse_params(levels=cfg.levels, clip=float(cfg.clip))
    fused = api.fuse_stack(sc["raw"], cfg.times, params)
    torch.cuda.synchronize()
    fused = fused.cpu().numpy()
    del sc["raw"]
    (o, pr, e), (ro, rp, re) = run(api, sc, fused, 2, 0)
    assert pr.shape == (modes, 256, 256)
    assert rel_l2(o, ro) <= 1e-5
    assert rel_l2(pr, rp) <= 1e-5
    np.testing.assert_allclose(e, re, rtol=1e-5)


def test_mixed_state_stage_launches(api):
    sc = synth.make_scan("mixed_small")
    cfg = sc["cfg"]
    p = oracle.FuseParams(levels=cfg.levels, clip=float(cfg.clip))
    fused = oracle.mnf_stack(sc["raw"][:10], sc["times"], p).astype(np.float32)
    h = api.ptycho_init(torch.from_numpy(fused).cuda(), sc["pos"][:10], noisy_start(cfg.M),
                        sc["probe"].astype(np.complex64))
    api.ptycho_set_timing(h, True)
    api.ptycho_iterate(h, 2)
    _, launches = api.ptycho_stage_times(h)
    assert launches == [6, 4, 6, 0]          # forward, modulus, inverse per iteration; the error
                                             # is formed inside the object step's k_apply
    api.ptycho_destroy(h)


@pytest.mark.parametrize("q", [2, 3, 5, 6, 7])
def test_mode_counts_match_oracle(api, q):
    """Every compile-time mode count of the modulus kernel: the first q probe modes of the
    small mixed-state scan, 5 iterations with probe updates, against the FP64 oracle."""
    sc = synth.make_scan("mixed_small")
    cfg = sc["cfg"]
    p = oracle.FuseParams(levels=cfg.levels, clip=float(cfg.clip))
    fused = oracle.mnf_stack(sc["raw"], sc["times"], p).astype(np.float32)
    sc = dict(sc, probe=sc["probe"][:q])
    (o, pr, e), (ro, rp, re) = run(api, sc, fused, 5, 0)
    assert pr.shape == (q, 64, 64)
    assert rel_l2(o, ro) <= 1e-5
    assert rel_l2(pr, rp) <= 1e-5
    np.testing.assert_allclose(e, re, rtol=1e-5)
