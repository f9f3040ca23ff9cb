"""Thin ctypes binding of the C ABI in ``include/ptycho_mnf.h`` (argument marshalling only).

Every function keeps the C name and forwards to ``libptycho_mnf.so``; all arithmetic runs in the
library's CUDA kernels.  Device buffers are torch CUDA tensors (PyTorch provides device memory
and streams), host buffers are numpy arrays.  Loading fails loudly if the library is missing:
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

PTYCHO_OK = 0
PTYCHO_EINVAL = -1
PTYCHO_ENOMEM = -2
PTYCHO_ECUDA = -3
PTYCHO_ENONFINITE = -4
PTYCHO_ETIMEDOUT = -5

BASE_MODES = {"mean": 0, "sum": 1, "weighted": 2}
ALGORITHMS = {"ap": 0, "epie_colour": 1}
DOMAINS = {"radiance": 0, "raw": 1}

EXPORTS = ("fuse_stack", "fuse_stack_noalloc", "fuse_stack_host", "fuse_sli", "ptycho_init", "ptycho_iterate",
           "ptycho_get_object", "ptycho_get_probe", "ptycho_get_colouring", "ptycho_destroy", "ptycho_set_timing", "ptycho_stage_times", "ptycho_release_memory", "ptycho_last_error")


class FuseParamsC(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_float), ("sigma", ctypes.c_float), ("levels", ctypes.c_int),
                ("delta0", ctypes.c_float), ("delta_ratio", ctypes.c_float),
                ("clip", ctypes.c_float), ("base_mode", ctypes.c_int), ("domain", ctypes.c_int)]


class PtychoDescC(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("N", ctypes.c_int), ("J", ctypes.c_int),
                ("modes", ctypes.c_int), ("h_pos", ctypes.c_void_p), ("d_fused", ctypes.c_void_p),
                ("obj0", ctypes.c_void_p), ("probe0", ctypes.c_void_p),
                ("init_on_device", ctypes.c_int), ("alpha_O", ctypes.c_float),
                ("alpha_P", ctypes.c_float), ("probe_update_start", ctypes.c_int),
                ("algorithm", ctypes.c_int), ("epie_alpha", ctypes.c_float),
                ("epie_beta", ctypes.c_float), ("fft_path", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p)]


class PtychoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_LIB = None


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load ``libptycho_mnf.so`` (built in-tree by ``__graft_entry__.build()``)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.fuse_stack.argtypes = [vp, ci, ci, ci, ctypes.POINTER(ctypes.c_float),
                             ctypes.POINTER(FuseParamsC), vp, vp]
    L.fuse_stack.restype = ci
    L.fuse_stack_noalloc.argtypes = L.fuse_stack.argtypes
    L.fuse_stack_noalloc.restype = ci
    L.fuse_stack_host.argtypes = [vp, vp, ci, ci, ci, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(FuseParamsC),
                                  vp, ci, vp]
    L.fuse_stack_host.restype = ci
    L.fuse_sli.argtypes = [vp, ci, ci, ci, ctypes.POINTER(ctypes.c_float), ctypes.c_float, vp, vp]
    L.ptycho_batch_create.restype = ci
    L.ptycho_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ci, ci, vp]
    L.ptycho_batch_iterate.restype = ci
    L.ptycho_batch_iterate.argtypes = [vp, ci, ctypes.POINTER(cd)]
    L.ptycho_batch_describe.restype = ci
    L.ptycho_batch_describe.argtypes = [vp, ctypes.c_char_p, ci]
    L.ptycho_batch_destroy.restype = None
    L.ptycho_batch_destroy.argtypes = [vp]
    L.gemm_bf16.restype = ci
    L.gemm_bf16.argtypes = [vp, vp, vp, ci, ci, ci, vp, vp]
    ip = ctypes.POINTER(ci)
    fp = ctypes.POINTER(ctypes.c_float)
    L.wsnet_create.restype = ci
    L.wsnet_create.argtypes = [ctypes.POINTER(vp), ip, ip, ip, ci, ci, ci, ctypes.c_ulonglong, vp]
    for name in ("wsnet_set_params", "wsnet_get_params", "wsnet_get_grads"):
        getattr(L, name).restype = ci
        getattr(L, name).argtypes = [vp, ci, fp, fp]
    L.wsnet_forward.restype = ci
    L.wsnet_forward.argtypes = [vp, vp, ci, vp]
    L.wsnet_backward.restype = ci
    L.wsnet_backward.argtypes = [vp, vp, vp, ci, ctypes.POINTER(cd)]
    L.wsnet_adam.restype = ci
    L.wsnet_adam.argtypes = [vp, ctypes.c_float]
    L.wsnet_train_step.restype = ci
    L.wsnet_train_step.argtypes = [vp, vp, vp, ci, ctypes.c_float, ctypes.POINTER(cd)]
    L.wsnet_destroy.restype = None
    L.wsnet_destroy.argtypes = [vp]
    L.ws_preprocess.restype = ci
    L.ws_preprocess.argtypes = [vp, ci, ci, vp, vp]
    L.ws_targets.restype = ci
    L.ws_targets.argtypes = [vp, ci, vp, ci, ci, vp, vp]
    L.ws_stitch.restype = ci
    L.ws_stitch.argtypes = [vp, vp, ci, vp, ci, ci, vp, vp]
    L.dft2_split_bf16.restype = ci
    L.dft2_split_bf16.argtypes = [vp, vp, ci, ci, ci, vp, vp]
    L.fuse_sli.restype = ci
    L.ptycho_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(PtychoDescC)]
    L.ptycho_init.restype = ci
    L.ptycho_iterate.argtypes = [vp, ci, ctypes.POINTER(cd)]
    L.ptycho_iterate.restype = ci
    L.ptycho_get_object.argtypes = [vp, vp, ci]
    L.ptycho_get_object.restype = ci
    L.ptycho_get_probe.argtypes = [vp, vp, ci]
    L.ptycho_get_probe.restype = ci
    L.ptycho_get_colouring.argtypes = [vp, vp, ctypes.POINTER(ci)]
    L.ptycho_get_colouring.restype = ci
    L.ptycho_destroy.argtypes = [vp]
    L.ptycho_destroy.restype = None
    L.ptycho_set_timing.argtypes = [vp, ci]
    L.ptycho_set_timing.restype = ci
    L.ptycho_stage_times.argtypes = [vp, ctypes.POINTER(cd), ctypes.POINTER(ctypes.c_longlong)]
    L.ptycho_stage_times.restype = ci
    L.ptycho_last_error.argtypes = []
    L.ptycho_last_error.restype = ctypes.c_char_p
    L.ptycho_debug_wait_timeout.argtypes = [vp, ci]
    L.ptycho_debug_wait_timeout.restype = ci
    L.ptycho_debug_fail_alloc.argtypes = [ci]
    L.ptycho_debug_fail_alloc.restype = ci
    L.ptycho_release_memory.argtypes = []
    L.ptycho_release_memory.restype = ci
    L.measure_fp32_fma.argtypes = [ci, ci, vp, ctypes.POINTER(cd), vp]
    L.measure_fp32_fma.restype = ci
    L.measure_fma_threads_per_block.argtypes = []
    L.measure_fma_threads_per_block.restype = ci
    _LIB = L
    return L


def last_error() -> str:
    return lib().ptycho_last_error().decode()


def _check(rc: int) -> None:
    if rc != PTYCHO_OK:
        raise PtychoError(rc, last_error())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def fuse_params(levels: int, clip: float, mu: float = 0.5, sigma: float = 0.2,
                delta0: float = 0.5, delta_ratio: float = 2.0, base_mode: str = "mean",
                domain: str = "radiance") -> FuseParamsC:
    return FuseParamsC(mu, sigma, levels, delta0, delta_ratio, clip, BASE_MODES[base_mode],
                       DOMAINS[domain])


def fuse_stack(raw, times, params: FuseParamsC, out=None, stream=None):
    """MNF of raw[J][K][N][N] (torch.uint16 CUDA tensor) into out[J][N][N] (float32 CUDA)."""
    import torch
    if raw.dtype != torch.uint16 or not raw.is_cuda or not raw.is_contiguous():
        raise ValueError("raw must be a contiguous torch.uint16 CUDA tensor [J][K][N][N]")
    J, K, N, N2 = raw.shape
    if N != N2:
        raise ValueError("frames must be square")
    if out is None:
        out = torch.empty((J, N, N), dtype=torch.float32, device=raw.device)
    if out.dtype != torch.float32 or not out.is_contiguous() or tuple(out.shape) != (J, N, N):
        raise ValueError("out must be a contiguous float32 tensor [J][N][N]")
    t = (ctypes.c_float * K)(*[float(x) for x in times])
    _check(lib().fuse_stack(ctypes.c_void_p(raw.data_ptr()), J, K, N, t, ctypes.byref(params),
                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
    return out


def fuse_stack_host(raw_host, raw_dev, times, params: FuseParamsC, out=None, stream=None, chunk_positions=0):
    """MNF of a host-resident stack: raw_host (torch.uint16 CPU tensor [J][K][N][N], pinned for
    overlap) is copied into raw_dev (torch.uint16 CUDA tensor of the same shape) chunk by chunk
    while the chunks already copied are fused into out[J][N][N] (float32 CUDA)."""
    import torch
    if raw_host.dtype != torch.uint16 or raw_host.is_cuda or not raw_host.is_contiguous():
        raise ValueError("raw_host must be a contiguous torch.uint16 CPU tensor [J][K][N][N]")
    if raw_dev.dtype != torch.uint16 or not raw_dev.is_cuda or not raw_dev.is_contiguous() or \
            tuple(raw_dev.shape) != tuple(raw_host.shape):
        raise ValueError("raw_dev must be a contiguous torch.uint16 CUDA tensor shaped like raw_host")
    J, K, N, N2 = raw_host.shape
    if N != N2:
        raise ValueError("frames must be square")
    if out is None:
        out = torch.empty((J, N, N), dtype=torch.float32, device=raw_dev.device)
    if out.dtype != torch.float32 or not out.is_contiguous() or tuple(out.shape) != (J, N, N):
        raise ValueError("out must be a contiguous float32 tensor [J][N][N]")
    t = (ctypes.c_float * K)(*[float(x) for x in times])
    _check(lib().fuse_stack_host(ctypes.c_void_p(raw_host.data_ptr()), ctypes.c_void_p(raw_dev.data_ptr()), J, K, N,
                                 t, ctypes.byref(params), ctypes.c_void_p(out.data_ptr()), int(chunk_positions),
                                 ctypes.c_void_p(_stream_ptr(stream))))
    return out


def fuse_stack_noalloc(raw, times, params: FuseParamsC, out, stream=None):
    """Allocation-free fusion (scratch in the library's static 16 MiB device array).  ``out``
    must be preallocated: a contiguous float32 CUDA tensor [J][N][N]."""
    import torch
    if raw.dtype != torch.uint16 or not raw.is_cuda or not raw.is_contiguous():
        raise ValueError("raw must be a contiguous torch.uint16 CUDA tensor [J][K][N][N]")
    J, K, N, _ = raw.shape
    if out.dtype != torch.float32 or not out.is_contiguous() or tuple(out.shape) != (J, N, N):
        raise ValueError("out must be a contiguous float32 tensor [J][N][N]")
    t = (ctypes.c_float * K)(*[float(x) for x in times])
    _check(lib().fuse_stack_noalloc(ctypes.c_void_p(raw.data_ptr()), J, K, N, t, ctypes.byref(params),
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
    return out


def fuse_sli(raw, times, clip: float, out=None, stream=None):
    """Standard Linear Integration of raw[J][K][N][N] (torch.uint16 CUDA) into out[J][N][N]."""
    import torch
    if raw.dtype != torch.uint16 or not raw.is_cuda or not raw.is_contiguous():
        raise ValueError("raw must be a contiguous torch.uint16 CUDA tensor [J][K][N][N]")
    J, K, N, _ = raw.shape
    if out is None:
        out = torch.empty((J, N, N), dtype=torch.float32, device=raw.device)
    t = (ctypes.c_float * K)(*[float(x) for x in times])
    _check(lib().fuse_sli(ctypes.c_void_p(raw.data_ptr()), J, K, N, t, float(clip),
                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
    return out


def dft2_split_bf16(x, inverse: bool = False, out=None, status=None, stream=None):
    """Unitary 2-D DFT (or inverse) of x[B][N][N] (complex64 CUDA) on the tensor cores, split-BF16
    3-term GEMM form.  ``status`` (int32 CUDA tensor [1]) receives 1 if a device wait gave up;
    a fresh zeroed one is used when omitted.  Returns (out, status)."""
    import torch
    if x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous() or x.dim() != 3:
        raise ValueError("x must be a contiguous complex64 CUDA tensor [B][N][N]")
    B, N, _ = x.shape
    if out is None:
        out = torch.empty_like(x)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=x.device)
    _check(lib().dft2_split_bf16(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), B, N,
                                 1 if inverse else 0, ctypes.c_void_p(status.data_ptr()),
                                 ctypes.c_void_p(_stream_ptr(stream))))
    return out, status


FFT_PATHS = {"radix_fp32": 0, "dftgemm_bf16x3": 1}


class PtychoHandle:
    """Owner of a ``ptycho_handle``; ``close()`` (or garbage collection) destroys it."""

    def __init__(self, ptr: int, M: int, N: int, J: int, Q: int = 1):
        self.ptr = ctypes.c_void_p(ptr)
        self.M, self.N, self.J, self.Q = M, N, J, Q

    def close(self) -> None:
        if self.ptr:
            lib().ptycho_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ptycho_init(fused, pos, obj0, probe0, alpha_O: float = 1e-3, alpha_P: float = 1e-3,
                probe_update_start: int = 0, stream=None, algorithm: str = "ap",
                epie_alpha: float = 1.0, epie_beta: float = 1.0,
                fft_path: str = "radix_fp32") -> PtychoHandle:
    """fused: float32 CUDA tensor [J][N][N]; pos: int [J][2] (y, x); obj0 / probe0: complex64,
    both numpy (host) or both torch CUDA tensors (device); probe0 is [N][N] (one mode) or
    [Q][N][N] (Q incoherent modes)."""
    import torch
    if fused.dtype != torch.float32 or not fused.is_cuda or not fused.is_contiguous():
        raise ValueError("fused must be a contiguous float32 CUDA tensor [J][N][N]")
    J, N, _ = fused.shape
    pos = np.ascontiguousarray(pos, dtype=np.int32)
    if pos.shape != (J, 2):
        raise ValueError("pos must be [J][2]")
    on_dev = isinstance(obj0, torch.Tensor)
    if on_dev:
        if not (isinstance(probe0, torch.Tensor) and obj0.is_cuda and probe0.is_cuda):
            raise ValueError("obj0 and probe0 must both be CUDA tensors or both numpy arrays")
        obj0 = obj0.to(torch.complex64).contiguous()
        probe0 = probe0.to(torch.complex64).contiguous()
        op, pp = obj0.data_ptr(), probe0.data_ptr()
    else:
        obj0 = np.ascontiguousarray(obj0, dtype=np.complex64)
        probe0 = np.ascontiguousarray(probe0, dtype=np.complex64)
        op, pp = obj0.ctypes.data, probe0.ctypes.data
    M = obj0.shape[0]
    Q = probe0.shape[0] if len(probe0.shape) == 3 else 1
    desc = PtychoDescC(M, N, J, Q, pos.ctypes.data, fused.data_ptr(), op, pp, 1 if on_dev else 0,
                       alpha_O, alpha_P, probe_update_start, ALGORITHMS[algorithm], epie_alpha,
                       epie_beta, FFT_PATHS[fft_path], _stream_ptr(stream))
    h = ctypes.c_void_p()
    _check(lib().ptycho_init(ctypes.byref(h), ctypes.byref(desc)))
    return PtychoHandle(h.value, M, N, J, Q)


def ptycho_iterate(h: PtychoHandle, n_iter: int, errors: bool = True):
    """Run n_iter iterations; returns the per-iteration errors (numpy) or None."""
    if errors:
        err = np.zeros(max(n_iter, 1), dtype=np.float64)
        _check(lib().ptycho_iterate(h.ptr, n_iter, err.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return err[:n_iter]
    _check(lib().ptycho_iterate(h.ptr, n_iter, None))
    return None


def _get(fn, h: PtychoHandle, shape, out):
    if out is None:
        out = np.empty(shape, dtype=np.complex64)
    import torch
    if isinstance(out, torch.Tensor):
        if out.dtype != torch.complex64 or not out.is_cuda or not out.is_contiguous() or tuple(out.shape) != shape:
            raise ValueError(f"out must be a contiguous complex64 CUDA tensor {shape}")
        _check(fn(h.ptr, ctypes.c_void_p(out.data_ptr()), 1))
    else:
        if out.dtype != np.complex64 or not out.flags.c_contiguous or out.shape != shape:
            raise ValueError(f"out must be a contiguous complex64 array {shape}")
        _check(fn(h.ptr, ctypes.c_void_p(out.ctypes.data), 0))
    return out


def ptycho_get_object(h: PtychoHandle, out=None):
    return _get(lib().ptycho_get_object, h, (h.M, h.M), out)


def ptycho_get_probe(h: PtychoHandle, out=None):
    shape = (h.N, h.N) if h.Q == 1 else (h.Q, h.N, h.N)
    return _get(lib().ptycho_get_probe, h, shape, out)


def ptycho_get_colouring(h: PtychoHandle):
    """(colour per position, number of colours) of an ePIE-by-colour handle."""
    col = np.empty(h.J, dtype=np.int32)
    n = ctypes.c_int()
    _check(lib().ptycho_get_colouring(h.ptr, ctypes.c_void_p(col.ctypes.data), ctypes.byref(n)))
    return col, n.value


def ptycho_destroy(h: PtychoHandle) -> None:
    h.close()


def ptycho_debug_wait_timeout(h: PtychoHandle, enable) -> None:
    """Test hook: 1 (or True) = the handle's exit-wave launches first wait on a barrier nothing
    arrives on; 2 = in the split last round, the first CTA of each leftover position skips its
    first hand-off arrival, so its partners' bounded waits run out; 0 = off."""
    _check(lib().ptycho_debug_wait_timeout(h.ptr, int(enable)))


def ptycho_release_memory() -> None:
    """Hand the memory kept by the library's per-device pools back to the device."""
    _check(lib().ptycho_release_memory())


def ptycho_debug_fail_alloc(nth: int) -> None:
    """Test hook: the nth device allocation of the library from now on fails (0 = off)."""
    _check(lib().ptycho_debug_fail_alloc(int(nth)))


def measure_fp32_fma_tflops(blocks_per_sm: int = 8, iters: int = 4096, reps: int = 5, device=None) -> dict:
    """The device's FP32 FMA rate: the best of ``reps`` timed launches of the library's FMA
    kernel (CUDA events on the current stream, after one warm-up launch)."""
    import torch
    dev = torch.device("cuda") if device is None else torch.device(device)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = blocks_per_sm * sms
    sink = torch.empty(blocks * lib().measure_fma_threads_per_block(), dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream(dev)
    flops = ctypes.c_double()
    best = None
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _check(lib().measure_fp32_fma(blocks, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(flops),
                                      ctypes.c_void_p(st.cuda_stream)))
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        if r > 0 and (best is None or ms < best):
            best = ms
    return {"tflops": flops.value / (best / 1e3) / 1e12, "ms": best, "blocks": blocks, "iters": iters}


def ptycho_set_timing(h: PtychoHandle, enable: bool) -> None:
    _check(lib().ptycho_set_timing(h.ptr, 1 if enable else 0))


def ptycho_stage_times(h: PtychoHandle):
    """(ms[4], launches[4]) for stages exit-wave, object, probe, error."""
    ms = (ctypes.c_double * 4)()
    n = (ctypes.c_longlong * 4)()
    _check(lib().ptycho_stage_times(h.ptr, ms, n))
    return list(ms), list(n)


BATCH_GRAPH = 1
BATCH_AUTOTUNE = 2
BATCH_ONE_LAUNCH = 4


class PtychoBatch:
    """Owner of a ``ptycho_batch`` over existing handles (which it does not own)."""

    def __init__(self, ptr: int, handles):
        self.ptr = ctypes.c_void_p(ptr)
        self.handles = list(handles)

    def close(self) -> None:
        if self.ptr:
            lib().ptycho_batch_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ptycho_batch_create(handles, graph: bool = False, autotune: bool = False, one_launch: bool = False,
                        stream=None) -> PtychoBatch:
    n = len(handles)
    arr = (ctypes.c_void_p * n)(*[h.ptr.value for h in handles])
    b = ctypes.c_void_p()
    flags = (BATCH_GRAPH if graph else 0) | (BATCH_AUTOTUNE if autotune else 0) | (BATCH_ONE_LAUNCH if one_launch else 0)
    _check(lib().ptycho_batch_create(ctypes.byref(b), arr, n, flags, ctypes.c_void_p(_stream_ptr(stream))))
    return PtychoBatch(b.value, handles)


def ptycho_batch_iterate(b: PtychoBatch, n_iter: int, errors: bool = True):
    """Run n_iter iterations of every dataset; returns each dataset's last-iteration error."""
    if errors:
        err = np.zeros(len(b.handles), dtype=np.float64)
        _check(lib().ptycho_batch_iterate(b.ptr, n_iter, err.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return err
    _check(lib().ptycho_batch_iterate(b.ptr, n_iter, None))
    return None


def ptycho_batch_describe(b: PtychoBatch) -> str:
    buf = ctypes.create_string_buffer(4096)
    _check(lib().ptycho_batch_describe(b.ptr, buf, len(buf)))
    return buf.value.decode()


def ptycho_batch_destroy(b: PtychoBatch) -> None:
    b.close()


# ----------------------------------------------------------------------------- warm start
WS_MODES = {"s1": 0, "s2": 1, "up": 2}


def gemm_bf16(A, B, status=None, stream=None):
    """C = A B^T on the tensor cores; A [M][K], B [N][K] bfloat16 CUDA tensors -> float32 [M][N]."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib().gemm_bf16(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(C.data_ptr()),
                           M, N, K, ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
    return C


class WsNet:
    """Owner of a ``wsnet`` (the warm-start network)."""

    def __init__(self, ptr, layers, in_side, max_batch):
        self.ptr = ctypes.c_void_p(ptr)
        self.layers = [tuple(l) for l in layers]
        self.in_side = in_side
        self.max_batch = max_batch
        side = in_side
        for _, _, m in self.layers:
            side = side // 2 if m == "s2" else (side * 2 if m == "up" else side)
        self.out_side = side
        self.out_channels = self.layers[-1][1]

    def close(self):
        if self.ptr:
            lib().wsnet_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wsnet_create(layers, in_side: int, max_batch: int, seed: int = 0, stream=None) -> WsNet:
    n = len(layers)
    ci = ctypes.c_int * n
    cin = ci(*[l[0] for l in layers])
    cout = ci(*[l[1] for l in layers])
    mode = ci(*[WS_MODES[l[2]] for l in layers])
    p = ctypes.c_void_p()
    _check(lib().wsnet_create(ctypes.byref(p), cin, cout, mode, n, in_side, max_batch, seed,
                              ctypes.c_void_p(_stream_ptr(stream))))
    return WsNet(p.value, layers, in_side, max_batch)


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def wsnet_set_params(net: WsNet, layer: int, w, b):
    w = np.ascontiguousarray(w, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    _check(lib().wsnet_set_params(net.ptr, layer, _fptr(w), _fptr(b)))


def _get2(fn, net: WsNet, layer: int):
    cin, cout, _ = net.layers[layer]
    w = np.empty((cout, cin, 3, 3), np.float32)
    b = np.empty(cout, np.float32)
    _check(fn(net.ptr, layer, _fptr(w), _fptr(b)))
    return w, b


def wsnet_get_params(net: WsNet, layer: int):
    return _get2(lib().wsnet_get_params, net, layer)


def wsnet_get_grads(net: WsNet, layer: int):
    return _get2(lib().wsnet_get_grads, net, layer)


def wsnet_forward(net: WsNet, x, out=None):
    """x: bfloat16 CUDA tensor [B][cin][s][s] -> float32 [B][cout][s'][s']."""
    import torch
    B = x.shape[0]
    if out is None:
        out = torch.empty((B, net.out_channels, net.out_side, net.out_side), dtype=torch.float32, device=x.device)
    _check(lib().wsnet_forward(net.ptr, ctypes.c_void_p(x.data_ptr()), B, ctypes.c_void_p(out.data_ptr())))
    return out


def wsnet_backward(net: WsNet, x, t, loss: bool = True):
    v = ctypes.c_double()
    _check(lib().wsnet_backward(net.ptr, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()), x.shape[0],
                                ctypes.byref(v) if loss else None))
    return v.value if loss else None


def wsnet_adam(net: WsNet, lr: float):
    _check(lib().wsnet_adam(net.ptr, lr))


def wsnet_train_step(net: WsNet, x, t, lr: float, loss: bool = False):
    v = ctypes.c_double()
    _check(lib().wsnet_train_step(net.ptr, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()), x.shape[0],
                                  lr, ctypes.byref(v) if loss else None))
    return v.value if loss else None


def wsnet_destroy(net: WsNet):
    net.close()


def ws_preprocess(fused, out=None, stream=None):
    """float32 CUDA [J][N][N] fused patterns -> bfloat16 [J][1][N/2][N/2] network input."""
    import torch
    J, N, _ = fused.shape
    if out is None:
        out = torch.empty((J, 1, N // 2, N // 2), dtype=torch.bfloat16, device=fused.device)
    _check(lib().ws_preprocess(ctypes.c_void_p(fused.data_ptr()), J, N, ctypes.c_void_p(out.data_ptr()),
                               ctypes.c_void_p(_stream_ptr(stream))))
    return out


def ws_targets(obj, pos, N: int, out=None, stream=None):
    """obj complex64 CUDA [M][M], pos int32 CUDA [J][2] -> float32 [J][2][N/4][N/4]."""
    import torch
    J = pos.shape[0]
    if out is None:
        out = torch.empty((J, 2, N // 4, N // 4), dtype=torch.float32, device=obj.device)
    _check(lib().ws_targets(ctypes.c_void_p(obj.data_ptr()), obj.shape[0], ctypes.c_void_p(pos.data_ptr()), J, N,
                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
    return out


def ws_stitch(pred, pos, probe, M: int, out=None, stream=None):
    """pred float32 CUDA [J][2][N/4][N/4], pos int32 CUDA [J][2], probe complex64 CUDA [N][N]
    -> complex64 [M][M] initial object."""
    import torch
    J = pred.shape[0]
    N = probe.shape[0]
    if out is None:
        out = torch.empty((M, M), dtype=torch.complex64, device=pred.device)
    _check(lib().ws_stitch(ctypes.c_void_p(pred.data_ptr()), ctypes.c_void_p(pos.data_ptr()), J,
                           ctypes.c_void_p(probe.data_ptr()), N, M, ctypes.c_void_p(out.data_ptr()),
                           ctypes.c_void_p(_stream_ptr(stream))))
    return out
