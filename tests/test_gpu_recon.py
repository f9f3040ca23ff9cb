"""ptycho_init / ptycho_iterate (CUDA, FP32) against the FP64 reconstruction oracle, through
the C ABI.  Both sides are fed the same fused intensities (the oracle's fusion, rounded to FP32),
so the comparison isolates the reconstruction."""
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


def fused_for(name):
    sc = synth.make_scan(name)
    cfg = sc["cfg"]
    p = oracle.FuseParams(levels=cfg.levels, clip=float(cfg.clip))
    fused = oracle.mnf_stack(sc["raw"], sc["times"], p).astype(np.float32)
    return sc, fused


def run_both(api, sc, fused32, n_iter, obj0, probe0, alpha=1e-3, pus=0, device_init=False):
    f_t = torch.from_numpy(fused32).cuda()
    if device_init:
        o0 = torch.from_numpy(obj0.astype(np.complex64)).cuda()
        p0 = torch.from_numpy(probe0.astype(np.complex64)).cuda()
    else:
        o0, p0 = obj0.astype(np.complex64), probe0.astype(np.complex64)
    h = api.ptycho_init(f_t, sc["pos"], o0, p0, alpha_O=alpha, alpha_P=alpha, probe_update_start=pus)
    errs = api.ptycho_iterate(h, n_iter)
    obj = api.ptycho_get_object(h)
    probe = api.ptycho_get_probe(h)
    api.ptycho_destroy(h)
    # the oracle starts from the same FP32-rounded inputs
    ro, rp, rerr = oracle.reconstruct(fused32.astype(np.float64), sc["pos"],
                                      obj0.astype(np.complex64).astype(np.complex128),
                                      probe0.astype(np.complex64).astype(np.complex128),
                                      n_iter, alpha, alpha, pus)
    return (obj, probe, errs), (ro, rp, rerr)


def noisy_start(M, seed=0):
    """A well-conditioned initial object: 1 + 0.1 complex Gaussian noise (seeded)."""
    rng = np.random.default_rng(seed)
    return 1.0 + 0.1 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)))


def oracle_sensitivity(sc, fused32, obj0, probe0, n_iter, pus):
    """How far the FP64 oracle itself moves when its initial object is perturbed by one FP32
    unit roundoff (2^-24 relative): the floor below which no FP32 path can be asked to agree."""
    rng = np.random.default_rng(99)
    pert = obj0 * (1.0 + 2.0 ** -24 * rng.standard_normal(obj0.shape))
    f = fused32.astype(np.float64)
    a = oracle.reconstruct(f, sc["pos"], obj0, probe0, n_iter, 1e-3, 1e-3, pus)
    b = oracle.reconstruct(f, sc["pos"], pert, probe0, n_iter, 1e-3, 1e-3, pus)
    return max(rel_l2(b[0], a[0]), rel_l2(b[1], a[1]))


@pytest.mark.parametrize("name,n_iter,pus", [("tiny", 30, 0), ("tiny", 30, 5), ("mid", 10, 0),
                                              ("small", 10, 0), ("small", 10, 10**6), ("mid128", 3, 0),
                                              ("mid128", 10, 10**6)])
def test_reconstruction_matches_oracle(api, name, n_iter, pus):
    """Fixed iteration count, FP32 GPU vs FP64 oracle within 1e-5 relative L2 on object and
    probe, from a start where the method is well conditioned at FP32 resolution."""
    sc, fused = fused_for(name)
    M = sc["cfg"].M
    obj0 = noisy_start(M).astype(np.complex64).astype(np.complex128)
    probe0 = sc["probe"].astype(np.complex64).astype(np.complex128)
    assert oracle_sensitivity(sc, fused, obj0, probe0, n_iter, pus) <= 2e-6
    (o, p, e), (ro, rp, re) = run_both(api, sc, fused, n_iter, obj0, probe0, pus=pus)
    assert rel_l2(o, ro) <= 1e-5
    assert rel_l2(p, rp) <= 1e-5
    np.testing.assert_allclose(e, re, rtol=1e-5)


def test_flat_start_workload_properties(api):
    """The 256 x 256 / 64 x 64 / 100-position workload as specified: 50 iterations from a flat
    object with probe updates.  A flat start is a degenerate point of phase retrieval: the FP64
    oracle itself moves by several percent when its start is perturbed by 1e-7, so the check is
    on what is stable -- the Fourier-error trajectory and the NRMSE to the ground truth."""
    sc, fused = fused_for("small")
    cfg = sc["cfg"]
    M = cfg.M
    (o, p, e), (ro, rp, re) = run_both(api, sc, fused, cfg.n_iter, np.ones((M, M), complex),
                                       sc["probe"])
    np.testing.assert_allclose(e, re, rtol=5e-2)
    assert e[-1] < 0.5 * e[0]
    den = oracle.illumination(sc["probe"], sc["pos"], M)
    mask = den >= 0.1 * den.max()
    n_gpu = oracle.nrmse(o.astype(np.complex128), sc["obj"], mask)
    n_ref = oracle.nrmse(ro, sc["obj"], mask)
    assert abs(n_gpu - n_ref) <= 0.1 * n_ref


def test_flat_start_workload_each_iteration_matches_oracle(api):
    """The same workload followed step by step: after every GPU iteration k (k = 0 .. 49, flat
    start, probe updates on) the FP64 oracle takes one iteration from the GPU's own state at k
    (object and probe as the GPU holds them), and the GPU's state at k + 1 must agree with it.
    Each of the 50 steps is then checked at single-iteration precision, which the trajectory's
    sensitivity to rounding does not blur.  Measured: 1.7e-6 (object) / 6.5e-6 (probe) on the
    first step from the flat object, <= 1.1e-7 on every later step (the FP32 storage rounding of
    the state), Fourier errors within 1e-8."""
    sc, fused = fused_for("small")
    cfg = sc["cfg"]
    M = cfg.M
    f64 = fused.astype(np.float64)
    A = oracle.amplitudes(f64)
    o0 = np.ones((M, M), np.complex64)
    p0 = sc["probe"].astype(np.complex64)
    h = api.ptycho_init(torch.from_numpy(fused).cuda(), sc["pos"], o0, p0, alpha_O=1e-3, alpha_P=1e-3,
                        probe_update_start=0)
    obj, probe = o0.astype(np.complex128), p0.astype(np.complex128)
    worst_later = 0.0
    for k in range(cfg.n_iter):
        e = api.ptycho_iterate(h, 1)
        go, gp = api.ptycho_get_object(h), api.ptycho_get_probe(h)
        ro, rp, re = oracle.reconstruct(f64, sc["pos"], obj, probe, 1, 1e-3, 1e-3, 0, A=A)
        d = max(rel_l2(go, ro), rel_l2(gp, rp))
        assert d <= (1e-5 if k == 0 else 1e-6), (k, d)
        assert abs(e[0] - re[0]) <= 1e-6 * re[0], k
        if k > 0:
            worst_later = max(worst_later, d)
        obj, probe = go.astype(np.complex128), gp.astype(np.complex128)
    api.ptycho_destroy(h)
    print(f"worst single-step deviation after the first step: {worst_later:.2e}")


def test_single_position_and_ragged_object(api):
    # one position, an object side that is not a multiple of the 32-pixel tile
    sc, fused = fused_for("tiny")
    sc = dict(sc)
    sel = [0, 7, 24]
    sc["pos"] = sc["pos"][sel] + np.array([0, 3])
    fused = fused[sel]
    obj0 = noisy_start(70)
    for subset in ([0], [0, 1, 2]):
        s2 = dict(sc)
        s2["pos"] = sc["pos"][subset]
        (o, p, e), (ro, rp, re) = run_both(api, s2, fused[subset], 10, obj0, sc["probe"])
        assert rel_l2(o, ro) <= 1e-5
        assert rel_l2(p, rp) <= 1e-5


def test_device_initial_guesses_and_resume(api):
    """Initial guesses from device memory; 6 iterations equal 4 + re-init + 2 (checkpoint and
    resume through get_object / get_probe), bit for bit."""
    sc, fused = fused_for("tiny")
    M = sc["cfg"].M
    f_t = torch.from_numpy(fused).cuda()
    o0 = torch.ones((M, M), dtype=torch.complex64, device="cuda")
    p0 = torch.from_numpy(sc["probe"].astype(np.complex64)).cuda()
    h = api.ptycho_init(f_t, sc["pos"], o0, p0, probe_update_start=10**6)
    api.ptycho_iterate(h, 6)
    full = api.ptycho_get_object(h)
    api.ptycho_destroy(h)
    h = api.ptycho_init(f_t, sc["pos"], o0, p0, probe_update_start=10**6)
    api.ptycho_iterate(h, 4, errors=False)
    mid_o = torch.empty((M, M), dtype=torch.complex64, device="cuda")
    mid_p = torch.empty_like(p0)
    api.ptycho_get_object(h, mid_o)
    api.ptycho_get_probe(h, mid_p)
    api.ptycho_destroy(h)
    h = api.ptycho_init(f_t, sc["pos"], mid_o, mid_p, probe_update_start=10**6)
    api.ptycho_iterate(h, 2)
    resumed = api.ptycho_get_object(h)
    api.ptycho_destroy(h)
    assert np.array_equal(full, resumed)


def test_deterministic(api):
    sc, fused = fused_for("tiny")
    M = sc["cfg"].M
    outs = []
    for _ in range(2):
        f_t = torch.from_numpy(fused).cuda()
        h = api.ptycho_init(f_t, sc["pos"], np.ones((M, M), np.complex64), sc["probe"])
        api.ptycho_iterate(h, 5)
        outs.append((api.ptycho_get_object(h), api.ptycho_get_probe(h)))
        api.ptycho_destroy(h)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_nonfinite_input_reports_error(api):
    sc, fused = fused_for("tiny")
    M = sc["cfg"].M
    bad = fused.copy()
    bad[3, 5, 5] = np.inf
    h = api.ptycho_init(torch.from_numpy(bad).cuda(), sc["pos"], np.ones((M, M), np.complex64), sc["probe"])
    with pytest.raises(api.PtychoError) as ei:
        api.ptycho_iterate(h, 2)
    assert ei.value.code == api.PTYCHO_ENONFINITE
    api.ptycho_destroy(h)


def test_stage_timing(api):
    sc, fused = fused_for("tiny")
    M = sc["cfg"].M
    h = api.ptycho_init(torch.from_numpy(fused).cuda(), sc["pos"], np.ones((M, M), np.complex64), sc["probe"])
    api.ptycho_set_timing(h, True)
    api.ptycho_iterate(h, 3)
    ms, launches = api.ptycho_stage_times(h)
    # the error is formed inside the object step's k_apply: the error stage launches nothing
    assert launches == [3, 6, 9, 0]
    assert all(m > 0 for m in ms[:3]) and ms[3] >= 0
    api.ptycho_destroy(h)


def test_lab_scale_flat_start_steps(api):
    """The benchmarked configuration as the bench runs it (flat object, true probe, probe updates
    on, 1600 positions of 256 x 256 on a 1024 x 1024 object), followed for four iterations: each
    GPU step against one FP64 oracle iteration from the GPU's own previous state.

    The first step from the flat object is ill-conditioned: every exit wave is P, and |F P| has
    exact zeros and ~22,000 of its 65,536 pixels below 1e-6 of its maximum, where the modulus
    projection takes a phase that rounding decides, so FP32 and FP64 part there (measured
    1.6e-4 object / 5.7e-4 probe; bound 2e-3).  From the second step on each step agrees at the
    FP32 storage rounding of the state (measured 1.1e-7; bound 1e-6), and the Fourier error
    agrees on every step (measured <= 1.9e-7; bound 1e-6)."""
    sc = synth.make_scan_torch("lab", device="cuda")
    cfg = sc["cfg"]
    fused_t = api.fuse_stack(sc["raw"], cfg.times, api.fuse_params(levels=cfg.levels, clip=float(cfg.clip)))
    torch.cuda.synchronize()
    fused = fused_t.cpu().numpy()
    del sc["raw"]
    M = cfg.M
    A = oracle.amplitudes(fused.astype(np.float64))
    norm = np.sum(A * A)
    o0 = np.ones((M, M), np.complex64)
    p0 = sc["probe"].astype(np.complex64)
    h = api.ptycho_init(torch.from_numpy(fused).cuda(), sc["pos"], o0, p0)
    obj, probe = o0.astype(np.complex128), p0.astype(np.complex128)
    for k in range(4):
        e = api.ptycho_iterate(h, 1)
        go, gp = api.ptycho_get_object(h), api.ptycho_get_probe(h)
        ro, rp, re = oracle.iterate_once(obj, probe, sc["pos"], A, 1e-3, 1e-3, True)
        print(f"lab step {k}: object {rel_l2(go, ro):.2e} probe {rel_l2(gp, rp):.2e}")
        bound = 2e-3 if k == 0 else 1e-6
        assert rel_l2(go, ro) <= bound, k
        assert rel_l2(gp, rp) <= bound, k
        assert e[0] == pytest.approx(re / norm, rel=1e-6), k
        obj, probe = go.astype(np.complex128), gp.astype(np.complex128)
    api.ptycho_destroy(h)


def test_lab_scale_one_iteration(api):
    """1600 positions, 256 x 256 probe, 1024 x 1024 object: one iteration against the oracle."""
    sc = synth.make_scan_torch("lab", device="cuda")
    cfg = sc["cfg"]
    params = api.fuse_params(levels=cfg.levels, clip=float(cfg.clip))
    fused_t = api.fuse_stack(sc["raw"], cfg.times, params)
    torch.cuda.synchronize()
    fused = fused_t.cpu().numpy()          # FP32 input fed to both sides
    del sc["raw"]
    M = cfg.M
    obj0 = noisy_start(M).astype(np.complex64)
    h = api.ptycho_init(torch.from_numpy(fused).cuda(), sc["pos"], obj0, sc["probe"])
    e = api.ptycho_iterate(h, 1)
    o = api.ptycho_get_object(h)
    p = api.ptycho_get_probe(h)
    api.ptycho_destroy(h)
    A = oracle.amplitudes(fused.astype(np.float64))
    ro, rp, re = oracle.iterate_once(obj0.astype(np.complex128), sc["probe"].astype(np.complex64).astype(np.complex128),
                                     sc["pos"], A, 1e-3, 1e-3, True)
    assert rel_l2(o, ro) <= 1e-5
    assert rel_l2(p, rp) <= 1e-5
    assert e[0] == pytest.approx(re / np.sum(A * A), rel=1e-4)
