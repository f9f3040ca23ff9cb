"""fuse_stack_noalloc: the allocation-free fusion entry point (for callers that cannot call a
device allocator) must give the results of fuse_stack, call after call.  Collected last on
purpose, so a run that stops at the first failure has already run every other test."""
import ctypes

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


@pytest.mark.parametrize("case", ["small", "lab200"])
def test_matches_fuse_stack_two_calls_in_a_row(api, case):
    if case == "small":
        sc = synth.make_scan("small")
        cfg = sc["cfg"]
        raw = torch.from_numpy(sc["raw"]).cuda()
    else:
        # 200 lab positions need ~190 MB of scratch: the call runs in 17-position chunks
        import dataclasses
        cfg = dataclasses.replace(synth.CONFIGS["lab"], J=200)
        raw = synth.make_scan_torch(cfg, device="cuda")["raw"]
    params = api.fuse_params(levels=cfg.levels, clip=float(cfg.clip))
    ref = api.fuse_stack(raw, cfg.times, params)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    for _ in range(2):
        out = torch.full(ref.shape, float("nan"), dtype=torch.float32, device="cuda")
        api.fuse_stack_noalloc(raw, cfg.times, params, out)
        torch.cuda.synchronize()
        # the same kernels on the same positions (only the chunking differs): bit-identical
        assert np.array_equal(out.cpu().numpy(), ref)


def test_rejects_scratch_beyond_the_static_buffer(api):
    # N = 1024, K = 8, 2 levels: one position needs ~17 MiB of scratch > 16 MiB
    p = api.fuse_params(levels=2, clip=4095.0)
    t = (ctypes.c_float * 8)(*range(1, 9))
    raw = torch.zeros((1, 8, 1024, 1024), dtype=torch.uint16, device="cuda")
    out = torch.zeros((1, 1024, 1024), dtype=torch.float32, device="cuda")
    rc = api.lib().fuse_stack_noalloc(ctypes.c_void_p(raw.data_ptr()), 1, 8, 1024, t, ctypes.byref(p),
                                      ctypes.c_void_p(out.data_ptr()), None)
    assert rc == api.PTYCHO_EINVAL
    assert "static buffer" in api.last_error()
