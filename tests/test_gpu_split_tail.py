"""The split last round of the N = 256 exit-wave launch.  With J positions on G persistent CTAs
(two per SM), the J mod G leftover positions run in a second, cooperative launch in which S CTAs
share each position (a batch range of every phase, two hand-offs through global counters).  The
position counts below leave 18, 37 and 120 positions over, which the launcher splits 8, 4 and 2
ways on a 148-SM part.  Each case is checked against the FP64 oracle, and against the same
dataset advanced in a captured batch graph (where the launch is never split): object, probe and
Fourier error must agree bit for bit, since a part computes exactly what the whole unit would and
the error is summed per batch in a fixed order."""
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


@pytest.mark.parametrize("leftover", [18, 37, 120])
def test_split_tail_matches_oracle_and_unsplit(api, leftover):
    G = 2 * torch.cuda.get_device_properties(0).multi_processor_count
    cfg = dataclasses.replace(synth.CONFIGS["lab"], J=G + leftover)
    sc = synth.make_scan_torch(cfg, seed=77)
    fused_t = api.fuse_stack(sc["raw"], cfg.times, api.fuse_params(levels=cfg.levels, clip=float(cfg.clip)))
    torch.cuda.synchronize()
    fused = fused_t.cpu().numpy()
    del sc["raw"]
    M = cfg.M
    rng = np.random.default_rng(leftover)
    obj0 = (1 + 0.1 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)))).astype(np.complex64)
    probe0 = sc["probe"].astype(np.complex64)
    # split: a single handle (the launcher splits the tail when not capturing)
    h = api.ptycho_init(torch.from_numpy(fused).cuda(), sc["pos"], obj0, probe0)
    e_split = api.ptycho_iterate(h, 2)
    o_split, p_split = api.ptycho_get_object(h), api.ptycho_get_probe(h)
    api.ptycho_destroy(h)
    # unsplit: the same dataset in a captured batch graph
    h = api.ptycho_init(torch.from_numpy(fused).cuda(), sc["pos"], obj0, probe0)
    b = api.ptycho_batch_create([h], graph=True)
    e_graph = [api.ptycho_batch_iterate(b, 1)[0] for _ in range(2)]
    o_graph, p_graph = api.ptycho_get_object(h), api.ptycho_get_probe(h)
    api.ptycho_batch_destroy(b)
    api.ptycho_destroy(h)
    assert np.array_equal(o_split, o_graph)
    assert np.array_equal(p_split, p_graph)
    assert np.array_equal(np.asarray(e_split, np.float64).ravel(), np.asarray(e_graph, np.float64).ravel())
    # and the FP64 oracle, one iteration from the same start
    A = oracle.amplitudes(fused.astype(np.float64))
    ro, rp, re = oracle.reconstruct(fused.astype(np.float64), sc["pos"], obj0.astype(np.complex128),
                                    probe0.astype(np.complex128), 2, 1e-3, 1e-3, 0, A=A)
    assert rel_l2(o_split, ro) <= 1e-5
    assert rel_l2(p_split, rp) <= 1e-5
    np.testing.assert_allclose(e_split, re, rtol=1e-5)
