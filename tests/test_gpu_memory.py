"""The library's per-device memory pool (stream-ordered allocations kept for reuse): a
reconstruction created after others were destroyed runs in pooled memory that still holds their
contents and must give the same result bit for bit; ptycho_release_memory hands the pooled
memory back to the device and leaves live handles working."""
import dataclasses

import numpy as np
import pytest

from paper_2608_01746_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_01746_b300 import api as a
    a.lib()
    return a


def lab_scan(api, J, seed):
    """Lab geometry (N = 256, 1024^2 object) with J positions, fused on the GPU."""
    cfg = dataclasses.replace(synth.CONFIGS["lab"], J=J)
    sc = synth.make_scan_torch(cfg, seed=seed, device="cuda")
    fused = api.fuse_stack(sc["raw"], cfg.times, api.fuse_params(levels=cfg.levels, clip=float(cfg.clip)))
    obj0 = torch.ones((cfg.M, cfg.M), dtype=torch.complex64, device="cuda")
    probe0 = torch.from_numpy(sc["probe"].astype(np.complex64)).cuda()
    return sc["pos"], fused, obj0, probe0


def reconstruct(api, scan, n_iter, destroy=True):
    pos, fused, obj0, probe0 = scan
    h = api.ptycho_init(fused, pos, obj0, probe0)
    errs = api.ptycho_iterate(h, n_iter)
    out = (errs, api.ptycho_get_object(h), api.ptycho_get_probe(h))
    if destroy:
        api.ptycho_destroy(h)
        return out
    return out, h


def test_pooled_memory_reuse_is_bit_identical(api):
    # 337 positions on the 296-CTA grid: the split last round runs too
    scan = lab_scan(api, 337, seed=11)
    first = reconstruct(api, scan, 5)
    # other reconstructions in between leave their contents in the pooled memory
    other = lab_scan(api, 150, seed=12)
    reconstruct(api, other, 3)
    reconstruct(api, lab_scan(api, 500, seed=13), 2)
    again = reconstruct(api, scan, 5)
    for a, b in zip(first, again):
        assert np.array_equal(a, b)


def test_release_memory_returns_pool_and_keeps_live_handles(api):
    scan = lab_scan(api, 337, seed=21)
    whole = reconstruct(api, scan, 7)
    torch.cuda.synchronize()
    kept = torch.cuda.mem_get_info()[0]          # the destroyed handle's buffers stay pooled
    api.ptycho_release_memory()
    torch.cuda.synchronize()
    freed = torch.cuda.mem_get_info()[0] - kept
    # psi' (337 x 256^2 complex64 = 177 MB), amplitudes (88 MB) and the 296 column slots (155 MB)
    assert freed > 300e6, freed
    # a release while a handle lives leaves its buffers valid
    (e4, _, _), h = reconstruct(api, scan, 4, destroy=False)
    api.ptycho_release_memory()
    e3 = api.ptycho_iterate(h, 3)
    obj, probe = api.ptycho_get_object(h), api.ptycho_get_probe(h)
    api.ptycho_destroy(h)
    assert np.array_equal(np.concatenate([e4, e3]), whole[0])
    assert np.array_equal(obj, whole[1]) and np.array_equal(probe, whole[2])
