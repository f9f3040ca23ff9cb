"""Failure paths of the C ABI on the GPU, made without faulting the device: a bounded wait that
runs out (a barrier nothing arrives on, limited to ~2^20 cycles; a hand-off counter a partner
never completes, limited to ~2^31 cycles) must come back as PTYCHO_ETIMEDOUT with the context
still usable, and a device allocation that fails (host-side
hook) must come back as PTYCHO_ENOMEM with everything the call had allocated released."""
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


@pytest.fixture(scope="module")
def lab8(api):
    """Eight positions of the lab scan (N = 256: the TMA exit-wave kernel with bounded waits)."""
    cfg = dataclasses.replace(synth.CONFIGS["lab"], J=8)
    sc = synth.make_scan_torch(cfg, seed=4242)
    fused = api.fuse_stack(sc["raw"], cfg.times, api.fuse_params(levels=cfg.levels, clip=float(cfg.clip)))
    torch.cuda.synchronize()
    obj0 = np.ones((cfg.M, cfg.M), np.complex64)
    return dict(fused=fused, pos=sc["pos"], obj0=obj0, probe0=sc["probe"].astype(np.complex64), cfg=cfg)


def _init(api, d, **kw):
    return api.ptycho_init(d["fused"], d["pos"], d["obj0"], d["probe0"], **kw)


def test_wait_timeout_reports_etimedout_and_context_survives(api, lab8):
    ref = _init(api, lab8)
    e_ref = api.ptycho_iterate(ref, 2)
    o_ref = api.ptycho_get_object(ref)
    api.ptycho_destroy(ref)

    h = _init(api, lab8)
    api.ptycho_debug_wait_timeout(h, True)
    with pytest.raises(api.PtychoError) as ei:
        api.ptycho_iterate(h, 1)
    assert ei.value.code == api.PTYCHO_ETIMEDOUT
    assert "gave up" in api.last_error()
    # the status is sticky for this handle, even with the hook off
    api.ptycho_debug_wait_timeout(h, False)
    with pytest.raises(api.PtychoError) as ei:
        api.ptycho_iterate(h, 1)
    assert ei.value.code == api.PTYCHO_ETIMEDOUT
    api.ptycho_destroy(h)

    # the context is intact: a fresh handle gives exactly the reference result
    h = _init(api, lab8)
    e = api.ptycho_iterate(h, 2)
    o = api.ptycho_get_object(h)
    api.ptycho_destroy(h)
    assert np.array_equal(e, e_ref)
    assert np.array_equal(o, o_ref)


def test_split_tail_handoff_timeout(api):
    """The hand-off of the split last round (CTAs sharing a leftover position meet on a global
    counter) gives up after its bounded wait when a partner never arrives (hook 2: the first CTA
    of each leftover position skips its first arrival): PTYCHO_ETIMEDOUT, and a fresh handle on
    the same data then reproduces the reference bit for bit."""
    G = 2 * torch.cuda.get_device_properties(0).multi_processor_count
    cfg = dataclasses.replace(synth.CONFIGS["lab"], J=G + 40)        # 40 leftover positions: split
    sc = synth.make_scan_torch(cfg, seed=99)
    fused = api.fuse_stack(sc["raw"], cfg.times, api.fuse_params(levels=cfg.levels, clip=float(cfg.clip)))
    del sc["raw"]
    torch.cuda.synchronize()
    d = dict(fused=fused, pos=sc["pos"], obj0=np.ones((cfg.M, cfg.M), np.complex64),
             probe0=sc["probe"].astype(np.complex64))
    ref = _init(api, d)
    e_ref = api.ptycho_iterate(ref, 1)
    o_ref = api.ptycho_get_object(ref)
    api.ptycho_destroy(ref)

    h = _init(api, d)
    api.ptycho_debug_wait_timeout(h, 2)
    with pytest.raises(api.PtychoError) as ei:
        api.ptycho_iterate(h, 1)
    assert ei.value.code == api.PTYCHO_ETIMEDOUT
    api.ptycho_destroy(h)

    h = _init(api, d)
    e = api.ptycho_iterate(h, 1)
    o = api.ptycho_get_object(h)
    api.ptycho_destroy(h)
    assert np.array_equal(e, e_ref)
    assert np.array_equal(o, o_ref)


def test_wait_timeout_hook_needs_a_kernel_with_waits(api):
    sc = synth.make_scan("tiny")
    cfg = sc["cfg"]
    fused = api.fuse_stack(torch.from_numpy(sc["raw"]).cuda(), cfg.times,
                           api.fuse_params(levels=cfg.levels, clip=float(cfg.clip)))
    h = api.ptycho_init(fused, sc["pos"], np.ones((cfg.M, cfg.M), np.complex64), sc["probe"].astype(np.complex64))
    with pytest.raises(api.PtychoError) as ei:
        api.ptycho_debug_wait_timeout(h, True)
    assert ei.value.code == api.PTYCHO_EINVAL
    api.ptycho_destroy(h)


def test_batch_reports_a_member_timeout(api, lab8):
    sc = synth.make_scan("small")
    cfg = sc["cfg"]
    fused = api.fuse_stack(torch.from_numpy(sc["raw"]).cuda(), cfg.times,
                           api.fuse_params(levels=cfg.levels, clip=float(cfg.clip)))
    small = api.ptycho_init(fused, sc["pos"], np.ones((cfg.M, cfg.M), np.complex64), sc["probe"].astype(np.complex64))
    big = _init(api, lab8)
    api.ptycho_debug_wait_timeout(big, True)
    b = api.ptycho_batch_create([small, big], graph=True)
    with pytest.raises(api.PtychoError) as ei:
        api.ptycho_batch_iterate(b, 1)
    assert ei.value.code == api.PTYCHO_ETIMEDOUT
    api.ptycho_batch_destroy(b)
    api.ptycho_destroy(big)
    api.ptycho_destroy(small)


def _free_bytes(api):
    """Device free bytes with the library's memory pool trimmed first: memory a call returned
    to the pool is handed back, memory still allocated (a leak) is not."""
    torch.cuda.synchronize()
    api.ptycho_release_memory()
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_allocation_failure_reports_enomem_without_leaks(api, lab8):
    free0 = _free_bytes(api)
    n_allocs = None
    try:
        for nth in range(1, 200):
            api.ptycho_debug_fail_alloc(nth)
            try:
                h = _init(api, lab8)
            except api.PtychoError as e:
                assert e.code == api.PTYCHO_ENOMEM, (nth, str(e))
                # nothing the failed call allocated is still held
                assert abs(_free_bytes(api) - free0) <= 4 << 20, nth
                continue
            n_allocs = nth - 1
            api.ptycho_destroy(h)
            break
    finally:
        api.ptycho_debug_fail_alloc(0)
    assert n_allocs is not None and n_allocs >= 20     # every allocation of ptycho_init was failed once
    assert abs(_free_bytes(api) - free0) <= 4 << 20


def test_fusion_allocation_failure(api, lab8):
    cfg = lab8["cfg"]
    raw = torch.zeros((2, cfg.K, cfg.N, cfg.N), dtype=torch.uint16, device="cuda")
    api.ptycho_debug_fail_alloc(1)
    try:
        with pytest.raises(api.PtychoError) as ei:
            api.fuse_stack(raw, cfg.times, api.fuse_params(levels=cfg.levels, clip=float(cfg.clip)))
        assert ei.value.code == api.PTYCHO_ENOMEM
    finally:
        api.ptycho_debug_fail_alloc(0)
    out = api.fuse_stack(raw, cfg.times, api.fuse_params(levels=cfg.levels, clip=float(cfg.clip)))
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
