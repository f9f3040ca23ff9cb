"""The C-ABI library without a GPU: it loads, exports every symbol the header declares, and
rejects invalid arguments before touching the device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2608_01746_b300 import api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(\w+)\s*\(", text, re.M):
            names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def L():
    return api.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("fuse_stack", "ptycho_init", "ptycho_iterate", "ptycho_get_object",
              "ptycho_get_probe", "ptycho_destroy", "ptycho_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    for n in declared_functions():
        assert hasattr(L, n), n


def _params(**kw):
    base = dict(levels=4, clip=4095.0)
    base.update(kw)
    return api.fuse_params(**base)


@pytest.mark.parametrize("J,K,N,kw", [
    (1, 0, 64, {}), (1, 9, 64, {}), (1, 3, 48, {}), (1, 3, 4, {}), (-1, 3, 64, {}),
    (1, 3, 16, {"levels": 4}), (1, 3, 64, {"sigma": 0.0}), (1, 3, 64, {"clip": 0.0}),
    (1, 3, 64, {"delta0": -1.0}), (1, 3, 64, {"delta_ratio": 0.0}),
])
def test_fuse_stack_rejects_bad_arguments(L, J, K, N, kw):
    p = _params(**kw)
    t = (ctypes.c_float * 8)(1, 10, 100, 1, 1, 1, 1, 1)
    rc = L.fuse_stack(ctypes.c_void_p(16), J, K, N, t, ctypes.byref(p), ctypes.c_void_p(16), None)
    assert rc == api.PTYCHO_EINVAL
    assert api.last_error().startswith("fuse_stack")


def test_fuse_stack_rejects_bad_times_and_modes(L):
    t = (ctypes.c_float * 3)(1, 0, 100)
    rc = L.fuse_stack(ctypes.c_void_p(16), 1, 3, 64, t, ctypes.byref(_params()), ctypes.c_void_p(16), None)
    assert rc == api.PTYCHO_EINVAL and "t[1]" in api.last_error()
    t = (ctypes.c_float * 3)(1, 10, 100)
    p = _params()
    p.base_mode = 7
    assert L.fuse_stack(ctypes.c_void_p(16), 1, 3, 64, t, ctypes.byref(p), ctypes.c_void_p(16), None) == api.PTYCHO_EINVAL
    assert L.fuse_stack(ctypes.c_void_p(16), 1, 3, 64, t, None, ctypes.c_void_p(16), None) == api.PTYCHO_EINVAL


def test_fuse_stack_host_rejects_bad_arguments(L):
    t = (ctypes.c_float * 3)(1, 10, 100)
    p = ctypes.byref(_params())
    # no host stack, negative chunk, and the fuse_stack checks (NULL device buffers)
    assert L.fuse_stack_host(None, ctypes.c_void_p(16), 1, 3, 64, t, p, ctypes.c_void_p(16), 0, None) == api.PTYCHO_EINVAL
    assert "host raw" in api.last_error()
    assert L.fuse_stack_host(ctypes.c_void_p(16), ctypes.c_void_p(16), 1, 3, 64, t, p, ctypes.c_void_p(16), -1,
                             None) == api.PTYCHO_EINVAL
    assert L.fuse_stack_host(ctypes.c_void_p(16), None, 1, 3, 64, t, p, ctypes.c_void_p(16), 0, None) == api.PTYCHO_EINVAL
    assert L.fuse_stack_host(None, None, 0, 3, 64, t, p, None, 0, None) == api.PTYCHO_OK      # J = 0: no-op


def test_fuse_stack_zero_positions_is_noop(L):
    t = (ctypes.c_float * 3)(1, 10, 100)
    assert L.fuse_stack(None, 0, 3, 64, t, ctypes.byref(_params()), None, None) == api.PTYCHO_OK


def _desc(**kw):
    pos = np.zeros((4, 2), np.int32)
    d = dict(M=128, N=64, J=4, modes=1, h_pos=pos.ctypes.data, d_fused=16, obj0=16, probe0=16,
             init_on_device=1, alpha_O=1e-3, alpha_P=1e-3, probe_update_start=0, algorithm=0,
             epie_alpha=1.0, epie_beta=1.0, fft_path=0, cuda_stream=None)
    d.update(kw)
    return api.PtychoDescC(**d), pos


@pytest.mark.parametrize("kw", [{"N": 32}, {"N": 512, "M": 512}, {"N": 128, "modes": 2}, {"J": 0}, {"M": 32}, {"alpha_O": -1.0},
                                {"modes": 0}, {"modes": 9}, {"algorithm": 2},
                                {"algorithm": 1, "modes": 2}, {"algorithm": 1, "epie_alpha": 0.0},
                                {"probe_update_start": -1}, {"d_fused": None}, {"obj0": None},
                                {"fft_path": 2}, {"fft_path": 1, "N": 16, "M": 64}, {"fft_path": 1, "N": 256, "M": 256, "modes": 2},
                                {"fft_path": 1, "modes": 2}, {"fft_path": 1, "algorithm": 1}])
def test_ptycho_init_rejects_bad_arguments(L, kw):
    d, _pos = _desc(**kw)
    h = ctypes.c_void_p(1234)
    assert L.ptycho_init(ctypes.byref(h), ctypes.byref(d)) == api.PTYCHO_EINVAL
    assert h.value is None
    assert api.last_error().startswith("ptycho_init")


def test_ptycho_init_rejects_positions_out_of_range(L):
    pos = np.array([[0, 0], [0, 65], [3, 3], [64, 64]], np.int32)
    d, _ = _desc(h_pos=pos.ctypes.data)
    h = ctypes.c_void_p()
    assert L.ptycho_init(ctypes.byref(h), ctypes.byref(d)) == api.PTYCHO_EINVAL
    assert "position 1" in api.last_error()


def test_null_handles(L):
    assert L.ptycho_iterate(None, 1, None) == api.PTYCHO_EINVAL
    assert L.ptycho_get_object(None, ctypes.c_void_p(16), 0) == api.PTYCHO_EINVAL
    assert L.ptycho_get_probe(None, ctypes.c_void_p(16), 0) == api.PTYCHO_EINVAL
    assert L.ptycho_set_timing(None, 1) == api.PTYCHO_EINVAL
    L.ptycho_destroy(None)


@pytest.mark.parametrize("B,N,inv", [(1, 32, 0), (1, 256, 0), (-1, 64, 0), (1, 64, 2), (-1, 128, 0)])
def test_dft2_split_bf16_rejects_bad_arguments(L, B, N, inv):
    rc = L.dft2_split_bf16(ctypes.c_void_p(16), ctypes.c_void_p(16), B, N, inv, ctypes.c_void_p(16), None)
    assert rc == api.PTYCHO_EINVAL
    assert api.last_error().startswith("dft2_split_bf16")


def test_dft2_split_bf16_empty_batch_is_noop(L):
    assert L.dft2_split_bf16(None, None, 0, 64, 0, None, None) == api.PTYCHO_OK


@pytest.mark.parametrize("n,flags", [(0, 0), (-1, 0), (1, 4)])
def test_batch_create_rejects_bad_arguments(L, n, flags):
    arr = (ctypes.c_void_p * 1)(None)
    b = ctypes.c_void_p(1234)
    assert L.ptycho_batch_create(ctypes.byref(b), arr, n, flags, None) == api.PTYCHO_EINVAL
    assert b.value is None
    assert api.last_error().startswith("ptycho_batch_create")


def test_batch_create_rejects_null_handle(L):
    arr = (ctypes.c_void_p * 2)(None, None)
    b = ctypes.c_void_p()
    assert L.ptycho_batch_create(ctypes.byref(b), arr, 2, 0, None) == api.PTYCHO_EINVAL
    assert "handle 0 is NULL" in api.last_error()
    assert L.ptycho_batch_iterate(None, 1, None) == api.PTYCHO_EINVAL
    L.ptycho_batch_destroy(None)


def test_release_memory_without_pools(L):
    """Nothing has allocated (no device here): ptycho_release_memory has no pool to trim and
    succeeds; the destroy of a NULL handle is a no-op."""
    assert L.ptycho_release_memory() == api.PTYCHO_OK
    L.ptycho_destroy(None)
