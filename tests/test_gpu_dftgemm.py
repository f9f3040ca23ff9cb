"""Split-BF16 (3-term) DFT-as-GEMM on the tensor cores against the FP64 oracle, through the C ABI.

Error bound of the form (per 1-D pass, relative to the operand scale): each operand x is
represented by hi + lo with |x - hi - lo| <= 2^-16 |x| (two BF16 roundings, unit roundoff
2^-8 each), and the dropped lo x lo product is <= 2^-16 |G| |x|; with the FP32 accumulation
(2^-24 per add) that is at most 3 x 2^-16 per pass.  A 2-D transform is two passes, so the
per-transform bound asserted below is 6 x 2^-16 (relative L2); the exit wave psi' (four
passes plus the modulus step) is bounded by 12 x 2^-16 relative, and so is one reconstruction
iteration built on it.  The measured values are printed (-s) and are several times smaller.
"""
import numpy as np
import pytest

import oracle
from paper_2608_01746_b300 import synth
from tests.parity_helpers import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PASS_BOUND = 3 * 2.0 ** -16
DFT_BOUND = 2 * PASS_BOUND
EXIT_BOUND = 4 * PASS_BOUND


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_01746_b300 import api as a
    a.lib()
    return a


def _inputs(B, seed, N=64):
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal((B, N, N)) + 1j * rng.standard_normal((B, N, N))).astype(np.complex64)
    x[0] = 0
    x[0, 3, 5] = 1.0                     # impulse: a pure twiddle pattern
    if B > 1:
        x[1] = 2.5 - 1.0j                # constant: all energy in the DC bin
    return x


def _per_transform_rel(a, b):
    return np.array([rel_l2(a[i], b[i]) for i in range(a.shape[0])])


@pytest.mark.parametrize("B,N", [(1, 64), (3, 64), (4, 64), (13, 64), (600, 64), (1, 128), (5, 128),
                                 (150, 128)])
def test_forward_and_inverse_match_fp64(api, B, N):
    x = _inputs(B, B, N)
    xt = torch.from_numpy(x).cuda()
    y, st = api.dft2_split_bf16(xt)
    z, st2 = api.dft2_split_bf16(xt, inverse=True)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and int(st2.item()) == 0
    ref_f = np.stack([oracle.fft2u(x[i].astype(np.complex128)) for i in range(B)])
    ref_i = np.stack([oracle.ifft2u(x[i].astype(np.complex128)) for i in range(B)])
    ef = _per_transform_rel(y.cpu().numpy(), ref_f)
    ei = _per_transform_rel(z.cpu().numpy(), ref_i)
    print(f"B={B} N={N}: forward rel L2 max {ef.max():.3e} mean {ef.mean():.3e}; "
          f"inverse max {ei.max():.3e} (bound {DFT_BOUND:.3e})")
    assert ef.max() <= DFT_BOUND
    assert ei.max() <= DFT_BOUND


def test_in_place_round_trip(api):
    x = _inputs(9, 5)
    xt = torch.from_numpy(x).cuda()
    buf = xt.clone()
    api.dft2_split_bf16(buf, out=buf)
    api.dft2_split_bf16(buf, inverse=True, out=buf)
    e = _per_transform_rel(buf.cpu().numpy(), x.astype(np.complex128))
    print(f"round trip rel L2 max {e.max():.3e}")
    assert e.max() <= 2 * DFT_BOUND


def _fused(name):
    sc = synth.make_scan(name)
    cfg = sc["cfg"]
    p = oracle.FuseParams(levels=cfg.levels, clip=float(cfg.clip))
    return sc, oracle.mnf_stack(sc["raw"], sc["times"], p).astype(np.float32)


def _run(api, sc, fused32, pos, obj0, probe0, n_iter, fft_path, pus=0):
    h = api.ptycho_init(torch.from_numpy(fused32).cuda(), pos, obj0.astype(np.complex64),
                        probe0.astype(np.complex64), probe_update_start=pus, fft_path=fft_path)
    e = api.ptycho_iterate(h, n_iter)
    o, p = api.ptycho_get_object(h), api.ptycho_get_probe(h)
    api.ptycho_destroy(h)
    return o, p, e


@pytest.mark.parametrize("subset", [None, [0], [0, 1, 2, 3, 4], [5, 9, 11, 20, 33, 47, 60]])
def test_one_iteration_matches_oracle(api, subset):
    """One full-batch iteration (exit waves by tensor-core DFTs, object and probe updates) from a
    noisy start; whole 100-position scan and ragged position counts (groups of 4 patches)."""
    sc, fused = _fused("small")
    pos = sc["pos"] if subset is None else sc["pos"][subset]
    fused = fused if subset is None else fused[subset]
    M = sc["cfg"].M
    rng = np.random.default_rng(0)
    obj0 = (1.0 + 0.1 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)))).astype(np.complex64)
    probe0 = sc["probe"].astype(np.complex64)
    o, p, e = _run(api, sc, fused, pos, obj0, probe0, 1, "dftgemm_bf16x3")
    ro, rp, re = oracle.reconstruct(fused.astype(np.float64), pos, obj0.astype(np.complex128),
                                    probe0.astype(np.complex128), 1, 1e-3, 1e-3, 0)
    eo, ep = rel_l2(o, ro), rel_l2(p, rp)
    print(f"J={len(pos)}: object {eo:.3e} probe {ep:.3e} error {abs(e[0] - re[0]) / re[0]:.3e} "
          f"(bound {EXIT_BOUND:.3e})")
    assert eo <= EXIT_BOUND
    assert ep <= EXIT_BOUND
    assert abs(e[0] - re[0]) <= EXIT_BOUND * re[0]


def test_ten_iterations_track_oracle_and_radix_path(api):
    """Ten iterations, probe update on: the tensor-core form stays within the per-iteration bound
    times the iteration count of the FP64 oracle, and the FP32 radix path within 1e-5."""
    sc, fused = _fused("small")
    M = sc["cfg"].M
    rng = np.random.default_rng(0)
    obj0 = (1.0 + 0.1 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)))).astype(np.complex64)
    probe0 = sc["probe"].astype(np.complex64)
    og, pg, eg = _run(api, sc, fused, sc["pos"], obj0, probe0, 10, "dftgemm_bf16x3")
    orx, prx, erx = _run(api, sc, fused, sc["pos"], obj0, probe0, 10, "radix_fp32")
    ro, rp, re = oracle.reconstruct(fused.astype(np.float64), sc["pos"], obj0.astype(np.complex128),
                                    probe0.astype(np.complex128), 10, 1e-3, 1e-3, 0)
    print(f"10 it: gemm object {rel_l2(og, ro):.3e} probe {rel_l2(pg, rp):.3e}; "
          f"radix object {rel_l2(orx, ro):.3e} probe {rel_l2(prx, rp):.3e}")
    assert rel_l2(og, ro) <= 10 * EXIT_BOUND
    assert rel_l2(pg, rp) <= 10 * EXIT_BOUND
    np.testing.assert_allclose(eg, re, rtol=10 * EXIT_BOUND)
    assert rel_l2(orx, ro) <= 1e-5


def test_gemm_path_is_deterministic_and_timed(api):
    sc, fused = _fused("small")
    M = sc["cfg"].M
    obj0 = np.ones((M, M), np.complex64)
    outs = []
    for _ in range(2):
        h = api.ptycho_init(torch.from_numpy(fused).cuda(), sc["pos"], obj0, sc["probe"].astype(np.complex64),
                            fft_path="dftgemm_bf16x3")
        api.ptycho_set_timing(h, True)
        api.ptycho_iterate(h, 3)
        ms, launches = api.ptycho_stage_times(h)
        outs.append(api.ptycho_get_object(h))
        api.ptycho_destroy(h)
        assert list(launches)[0] == 3               # one exit-wave launch per iteration
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("subset", [None, [0, 6, 12]])
def test_n128_iteration_matches_oracle(api, subset):
    """N = 128 (two 64-point GEMM halves + radix-2 butterfly per pass): one iteration on the
    5 x 5 / 128^2-probe scan and on a 3-position subset, within the exit-wave bound."""
    sc, fused = _fused("mid128")
    pos = sc["pos"] if subset is None else sc["pos"][subset]
    fused = fused if subset is None else fused[subset]
    M = sc["cfg"].M
    rng = np.random.default_rng(1)
    obj0 = (1.0 + 0.1 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)))).astype(np.complex64)
    probe0 = sc["probe"].astype(np.complex64)
    o, p, e = _run(api, sc, fused, pos, obj0, probe0, 1, "dftgemm_bf16x3")
    ro, rp, re = oracle.reconstruct(fused.astype(np.float64), pos, obj0.astype(np.complex128),
                                    probe0.astype(np.complex128), 1, 1e-3, 1e-3, 0)
    print(f"N=128 J={len(pos)}: object {rel_l2(o, ro):.3e} probe {rel_l2(p, rp):.3e}")
    assert rel_l2(o, ro) <= EXIT_BOUND
    assert rel_l2(p, rp) <= EXIT_BOUND
    assert abs(e[0] - re[0]) <= EXIT_BOUND * re[0]


@pytest.fixture(scope="module")
def lab24():
    """24 positions of the lab scan (N = 256), fused by the oracle."""
    import dataclasses
    cfg = dataclasses.replace(synth.CONFIGS["lab"], J=24)
    sc = synth.make_scan_torch(cfg, seed=2024, device="cpu")
    raw = sc["raw"].numpy()
    p = oracle.FuseParams(levels=cfg.levels, clip=float(cfg.clip))
    sc["cfg"] = cfg
    return sc, oracle.mnf_stack(raw, cfg.times, p).astype(np.float32)


@pytest.mark.parametrize("n_iter,subset", [(1, None), (1, [0, 7, 23]), (3, None)])
def test_n256_iterations_match_oracle(api, lab24, n_iter, subset):
    """N = 256 on the tensor cores (each 256-point transform = four 64-point split-BF16 GEMMs
    and a radix-4 epilogue, inside the TMA slot pipeline of the radix kernel): 1 and 3
    iterations against the oracle, within the exit-wave bound per iteration."""
    sc, fused = lab24
    pos = sc["pos"] if subset is None else sc["pos"][subset]
    fused = fused if subset is None else fused[subset]
    M = sc["cfg"].M
    rng = np.random.default_rng(3)
    obj0 = (1.0 + 0.1 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)))).astype(np.complex64)
    probe0 = sc["probe"].astype(np.complex64)
    o, p, e = _run(api, sc, fused, pos, obj0, probe0, n_iter, "dftgemm_bf16x3")
    ro, rp, re = oracle.reconstruct(fused.astype(np.float64), pos, obj0.astype(np.complex128),
                                    probe0.astype(np.complex128), n_iter, 1e-3, 1e-3, 0)
    print(f"N=256 J={len(pos)} {n_iter} it: object {rel_l2(o, ro):.3e} probe {rel_l2(p, rp):.3e} "
          f"error {abs(e[-1] - re[-1]) / re[-1]:.3e}")
    assert rel_l2(o, ro) <= n_iter * EXIT_BOUND
    assert rel_l2(p, rp) <= n_iter * EXIT_BOUND
    np.testing.assert_allclose(e, re, rtol=n_iter * EXIT_BOUND)
