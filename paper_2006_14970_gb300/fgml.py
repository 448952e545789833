"""Python binding of libfgml (include/fgml.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module passes device
pointers, sizes, pitches and the current torch stream through ctypes. If the shared
library is missing it raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

from . import build as _build

FG_OK, FG_ERR_INVALID_ARG, FG_ERR_OOM, FG_ERR_CUDA, FG_ERR_TIMEOUT, FG_ERR_RANGE, \
    FG_ERR_BUSY, FG_ERR_UNSUPPORTED = range(8)
FG_F32, FG_BF16, FG_F16 = 0, 1, 2
ORDER_JACOBI, ORDER_REDBLACK = 0, 1

_DTYPES = {torch.float32: FG_F32, torch.bfloat16: FG_BF16, torch.float16: FG_F16}


class FgmlError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"fgml status {status}: {message}")
        self.status = status


class Params(ctypes.Structure):
    """fg_params; defaults (via ``params()``) are the paper's."""

    _fields_ = [("eps_r", ctypes.c_float), ("omega", ctypes.c_float),
                ("small_size", ctypes.c_int), ("small_iters", ctypes.c_int),
                ("big_iters", ctypes.c_int), ("order", ctypes.c_int),
                ("clamp", ctypes.c_int), ("init", ctypes.c_float)]


class Image(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("w", ctypes.c_int), ("h", ctypes.c_int),
                ("row_pitch_bytes", ctypes.c_longlong), ("dtype", ctypes.c_int)]


_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load():
    """Loads libfgml.so (built by ``paper_2006_14970_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libfgml.so is not built ({path}); run "
                           "paper_2006_14970_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    ip = P(ctypes.c_int)
    lib.fg_params_default.argtypes = [P(Params)]
    lib.fg_params_default.restype = None
    lib.fg_schedule.argtypes = [ctypes.c_int, ctypes.c_int, P(Params), ip, ip, ip, ctypes.c_int]
    lib.fg_schedule.restype = ctypes.c_int
    lib.fg_estimate.argtypes = [P(Image), P(Image), P(Params), P(Image), P(Image), vp]
    lib.fg_estimate.restype = ctypes.c_int
    lib.fg_estimate_host.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     P(Params), vp, vp, vp]
    lib.fg_estimate_host.restype = ctypes.c_int
    lib.fg_estimate_host_async.argtypes = lib.fg_estimate_host.argtypes
    lib.fg_estimate_host_async.restype = ctypes.c_int
    lib.fg_level_pass.argtypes = [P(Image), P(Image), P(Image), P(Image), ctypes.c_int,
                                  P(Params), P(Image), P(Image), vp]
    lib.fg_level_pass.restype = ctypes.c_int
    lib.fg_estimate_batch.argtypes = [ctypes.c_int, P(Image), P(Image), P(Params), P(Image),
                                      P(Image), vp]
    lib.fg_estimate_batch.restype = ctypes.c_int
    lib.fg_autotune_batch.argtypes = [ctypes.c_int, P(Image), P(Image), P(Params), P(Image),
                                      P(Image), vp, P(ctypes.c_int), P(ctypes.c_float)]
    lib.fg_autotune_batch.restype = ctypes.c_int
    lib.fg_selftest_bounded_wait.argtypes = [vp]
    lib.fg_selftest_bounded_wait.restype = ctypes.c_int
    lib.fg_sync.argtypes = [vp]
    lib.fg_sync.restype = ctypes.c_int
    lib.fg_estimate_composite.argtypes = [P(Image), P(Image), P(Params), P(Image), P(Image),
                                          P(Image), P(Image), vp]
    lib.fg_estimate_composite.restype = ctypes.c_int
    lib.fg_minimiser_cg.argtypes = [P(Image), P(Image), P(Params), vp, vp, ctypes.c_int,
                                     ctypes.c_double, P(ctypes.c_int), P(ctypes.c_double), vp]
    lib.fg_minimiser_cg.restype = ctypes.c_int
    lib.fg_quality.argtypes = [P(Image), P(Image), P(Image), P(ctypes.c_double), vp]
    lib.fg_quality.restype = ctypes.c_int
    lib.fg_release_workspace.argtypes = [vp]
    lib.fg_release_workspace.restype = ctypes.c_int
    lib.fg_last_error.argtypes = []
    lib.fg_last_error.restype = ctypes.c_char_p
    lib.fg_version.argtypes = []
    lib.fg_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def declared_functions() -> list[str]:
    """Names of the functions include/fgml.h declares."""
    text = open(os.path.join(_build.INCLUDE, "fgml.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fg_[a-z_0-9]+)\s*\(", text)))


def _check(status: int):
    if status != FG_OK:
        raise FgmlError(status, load().fg_last_error().decode())


def params(**kw) -> Params:
    p = Params()
    load().fg_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, int(v) if k in ("small_size", "small_iters", "big_iters", "order",
                                      "clamp") else float(v))
    return p


def schedule(w: int, h: int, p: Params | None = None):
    """Level sizes and sweep counts [(w_l, h_l, k_l)] of Algorithm 1 (host planner)."""
    cap = 64
    ws, hs, ks = (ctypes.c_int * cap)(), (ctypes.c_int * cap)(), (ctypes.c_int * cap)()
    n = load().fg_schedule(int(w), int(h), ctypes.byref(p) if p is not None else None,
                           ws, hs, ks, cap)
    if n < 0:
        raise ValueError(f"invalid size {w}x{h}")
    return [(ws[i], hs[i], ks[i]) for i in range(n)]


def _image(t: torch.Tensor, channels: int, name: str) -> Image:
    if t.dtype not in _DTYPES:
        raise TypeError(f"{name}: dtype {t.dtype} is not float32/bfloat16/float16")
    if channels == 3:
        if t.dim() != 3 or t.shape[2] != 3 or t.stride(2) != 1 or t.stride(1) != 3:
            raise ValueError(f"{name} must be [H, W, 3] with packed pixels")
    else:
        if t.dim() != 2 or t.stride(1) != 1:
            raise ValueError(f"{name} must be [H, W] with unit column stride")
    return Image(t.data_ptr(), t.shape[1], t.shape[0], t.stride(0) * t.element_size(),
                 _DTYPES[t.dtype])


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def estimate(I: torch.Tensor, alpha: torch.Tensor, p: Params | None = None,
             F: torch.Tensor | None = None, B: torch.Tensor | None = None, stream=None):
    """fg_estimate on device tensors I [H, W, 3] and alpha [H, W]; returns (F, B)."""
    if not (I.is_cuda and alpha.is_cuda):
        raise ValueError("fg_estimate takes CUDA tensors; use estimate_host for host memory")
    if F is None:
        F = torch.empty_like(I, memory_format=torch.contiguous_format)
    if B is None:
        B = torch.empty_like(I, memory_format=torch.contiguous_format)
    iI, iA, iF, iB = _image(I, 3, "I"), _image(alpha, 1, "alpha"), _image(F, 3, "F"), \
        _image(B, 3, "B")
    _check(load().fg_estimate(ctypes.byref(iI), ctypes.byref(iA),
                              ctypes.byref(p) if p is not None else None,
                              ctypes.byref(iF), ctypes.byref(iB), _stream(stream)))
    return F, B


def estimate_host(I: torch.Tensor, alpha: torch.Tensor, p: Params | None = None,
                  F: torch.Tensor | None = None, B: torch.Tensor | None = None, stream=None):
    """fg_estimate_host on contiguous host tensors (pinned for speed); returns (F, B)."""
    if I.is_cuda or alpha.is_cuda:
        raise ValueError("estimate_host takes host tensors")
    I = I.contiguous()
    alpha = alpha.contiguous()
    h, w = alpha.shape
    if I.shape != (h, w, 3) or I.dtype != alpha.dtype or I.dtype not in _DTYPES:
        raise ValueError("I must be [H, W, 3] and alpha [H, W] of one float dtype")
    if F is None:
        F = torch.empty_like(I)
    if B is None:
        B = torch.empty_like(I)
    _check(load().fg_estimate_host(ctypes.c_void_p(I.data_ptr()),
                                   ctypes.c_void_p(alpha.data_ptr()), w, h, _DTYPES[I.dtype],
                                   ctypes.byref(p) if p is not None else None,
                                   ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                   _stream(stream)))
    return F, B


def estimate_host_async(I: torch.Tensor, alpha: torch.Tensor, p: Params | None = None,
                        F: torch.Tensor | None = None, B: torch.Tensor | None = None, stream=None):
    """fg_estimate_host_async: as estimate_host, but only enqueued on the stream; the host
    tensors (pinned) must stay alive and unchanged until the stream has passed it."""
    if I.is_cuda or alpha.is_cuda:
        raise ValueError("estimate_host_async takes host tensors")
    if not (I.is_contiguous() and alpha.is_contiguous()):
        raise ValueError("I and alpha must be contiguous (they are read after the call returns)")
    h, w = alpha.shape
    if I.shape != (h, w, 3) or I.dtype != alpha.dtype or I.dtype not in _DTYPES:
        raise ValueError("I must be [H, W, 3] and alpha [H, W] of one float dtype")
    if F is None:
        F = torch.empty(I.shape, dtype=I.dtype, pin_memory=True)
    if B is None:
        B = torch.empty(I.shape, dtype=I.dtype, pin_memory=True)
    _check(load().fg_estimate_host_async(ctypes.c_void_p(I.data_ptr()),
                                         ctypes.c_void_p(alpha.data_ptr()), w, h, _DTYPES[I.dtype],
                                         ctypes.byref(p) if p is not None else None,
                                         ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                         _stream(stream)))
    return F, B


def level_pass(I, alpha, F_src, B_src, iters: int, w: int, h: int, p: Params | None = None,
               F_dst=None, B_dst=None, stream=None):
    """fg_level_pass: ``iters`` sweeps of a w x h level from (F_src, B_src)."""
    if F_dst is None:
        F_dst = torch.empty((h, w, 3), dtype=I.dtype, device=I.device)
    if B_dst is None:
        B_dst = torch.empty((h, w, 3), dtype=I.dtype, device=I.device)
    imgs = [_image(I, 3, "I"), _image(alpha, 1, "alpha"), _image(F_src, 3, "F_src"),
            _image(B_src, 3, "B_src"), _image(F_dst, 3, "F_dst"), _image(B_dst, 3, "B_dst")]
    _check(load().fg_level_pass(*(ctypes.byref(x) for x in imgs[:4]), int(iters),
                                ctypes.byref(p) if p is not None else None,
                                ctypes.byref(imgs[4]), ctypes.byref(imgs[5]), _stream(stream)))
    return F_dst, B_dst


class Batch:
    """The arguments of one fg_estimate_batch call, marshalled once: a list of (I, alpha)
    device tensor pairs and their (F, B) outputs (allocated when not given). run() repeats
    the call without converting the tensors again (for 64 images that conversion costs
    about half a millisecond of host time); the tensors must stay alive and in place."""

    def __init__(self, images, outputs=None):
        if outputs is None:
            outputs = [(torch.empty_like(I, memory_format=torch.contiguous_format),
                        torch.empty_like(I, memory_format=torch.contiguous_format))
                       for I, _ in images]
        self.images, self.outputs, self.n = images, outputs, len(images)
        arr = Image * max(1, self.n)
        self._I = arr(*[_image(I, 3, "I") for I, _ in images])
        self._A = arr(*[_image(A, 1, "alpha") for _, A in images])
        self._F = arr(*[_image(F, 3, "F") for F, _ in outputs])
        self._B = arr(*[_image(B, 3, "B") for _, B in outputs])

    def run(self, p: Params | None = None, stream=None):
        if self.n:
            _check(load().fg_estimate_batch(self.n, self._I, self._A,
                                            ctypes.byref(p) if p is not None else None,
                                            self._F, self._B, _stream(stream)))
        return self.outputs


def estimate_batch(images, p: Params | None = None, outputs=None, stream=None):
    """fg_estimate_batch on a list of (I, alpha) device tensor pairs; returns [(F, B)]."""
    if len(images) == 0:
        return []
    return Batch(images, outputs).run(p, stream)


def autotune_batch(images, p: Params | None = None, outputs=None, stream=None):
    """fg_autotune_batch on a list of (I, alpha) device tensor pairs: picks the work-list
    strip shape by measurement; returns (candidate index, ms per call)."""
    n = len(images)
    if outputs is None:
        outputs = [(torch.empty_like(I, memory_format=torch.contiguous_format),
                    torch.empty_like(I, memory_format=torch.contiguous_format)) for I, _ in images]
    arr = Image * n
    iI = arr(*[_image(I, 3, "I") for I, _ in images])
    iA = arr(*[_image(A, 1, "alpha") for _, A in images])
    iF = arr(*[_image(F, 3, "F") for F, _ in outputs])
    iB = arr(*[_image(B, 3, "B") for _, B in outputs])
    chosen = ctypes.c_int(-1)
    ms = ctypes.c_float(0.0)
    _check(load().fg_autotune_batch(n, iI, iA, ctypes.byref(p) if p is not None else None, iF, iB,
                                    _stream(stream), ctypes.byref(chosen), ctypes.byref(ms)))
    return chosen.value, ms.value


def selftest_bounded_wait(stream=None) -> int:
    """Runs the bounded-wait diagnostic; returns its status (FG_ERR_TIMEOUT = as intended)."""
    return load().fg_selftest_bounded_wait(_stream(stream))


def sync(stream=None):
    _check(load().fg_sync(_stream(stream)))


def estimate_composite(I, alpha, B_new, p: Params | None = None, F=None, B=None, I_new=None,
                       stream=None):
    """fg_estimate_composite: (F, B, I_new) with I_new = alpha F + (1 - alpha) B_new
    formed by the last level's pass."""
    F = torch.empty_like(I) if F is None else F
    B = torch.empty_like(I) if B is None else B
    I_new = torch.empty_like(I) if I_new is None else I_new
    imgs = [_image(I, 3, "I"), _image(alpha, 1, "alpha"), _image(F, 3, "F"), _image(B, 3, "B"),
            _image(B_new, 3, "B_new"), _image(I_new, 3, "I_new")]
    _check(load().fg_estimate_composite(
        ctypes.byref(imgs[0]), ctypes.byref(imgs[1]), ctypes.byref(p) if p is not None else None,
        ctypes.byref(imgs[2]), ctypes.byref(imgs[3]), ctypes.byref(imgs[4]), ctypes.byref(imgs[5]),
        _stream(stream)))
    return F, B, I_new


def minimiser_cg(I, alpha, p: Params | None = None, F0=None, B0=None, max_iters: int = 20000,
                 rel_tol: float = 1e-10, stream=None):
    """fg_minimiser_cg: the unclamped minimiser of the global cost by float64 conjugate
    gradients, from (F0, B0) (zeros if None). Returns (F, B, iterations, relative
    residual); F and B are float64 [H, W, 3] device tensors."""
    h, w = alpha.shape[0], alpha.shape[1]
    F = torch.zeros((h, w, 3), dtype=torch.float64, device=I.device) if F0 is None else \
        F0.to(torch.float64).contiguous().clone()
    B = torch.zeros((h, w, 3), dtype=torch.float64, device=I.device) if B0 is None else \
        B0.to(torch.float64).contiguous().clone()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    imgs = [_image(I, 3, "I"), _image(alpha, 1, "alpha")]
    _check(load().fg_minimiser_cg(ctypes.byref(imgs[0]), ctypes.byref(imgs[1]),
                                  ctypes.byref(p) if p is not None else None,
                                  ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                  int(max_iters), float(rel_tol), ctypes.byref(it),
                                  ctypes.byref(rr), _stream(stream)))
    return F, B, it.value, rr.value


def quality(F_est, F_gt, alpha_gt, stream=None) -> dict:
    """fg_quality: SAD, MSE and GRAD of F_est against F_gt over 0 < alpha_gt < 1
    (Section IV-C); device tensors of one dtype. Synchronises the stream."""
    out = (ctypes.c_double * 3)()
    imgs = [_image(F_est, 3, "F_est"), _image(F_gt, 3, "F_gt"), _image(alpha_gt, 1, "alpha_gt")]
    _check(load().fg_quality(*(ctypes.byref(x) for x in imgs), out, _stream(stream)))
    return {"sad": out[0], "mse": out[1], "grad": out[2]}


def release_workspace(stream=None):
    _check(load().fg_release_workspace(_stream(stream)))


def version() -> str:
    return load().fg_version().decode()


def estimate_noalloc(I: torch.Tensor, alpha: torch.Tensor, p: Params | None = None,
                     F: torch.Tensor | None = None, B: torch.Tensor | None = None, stream=None):
    """fg_estimate_noalloc: as ``estimate`` but the library allocates no device memory
    (intermediate levels use its fixed array of two 32 MiB level buffers; larger images
    are rejected). For callers that cannot let the library call cudaMalloc, e.g. a process
    whose device memory is all reserved by its own pool. Calls that overlap on the GPU
    share that array and race; keep them on one stream."""
    lib = load()
    fn = lib.fg_estimate_noalloc
    P = ctypes.POINTER
    fn.argtypes = [P(Image), P(Image), P(Params), P(Image), P(Image), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    if F is None:
        F = torch.empty_like(I, memory_format=torch.contiguous_format)
    if B is None:
        B = torch.empty_like(I, memory_format=torch.contiguous_format)
    iI, iA, iF, iB = _image(I, 3, "I"), _image(alpha, 1, "alpha"), _image(F, 3, "F"), \
        _image(B, 3, "B")
    _check(fn(ctypes.byref(iI), ctypes.byref(iA), ctypes.byref(p) if p is not None else None,
              ctypes.byref(iF), ctypes.byref(iB), _stream(stream)))
    return F, B


class ServerCfg(ctypes.Structure):
    _fields_ = [("max_inflight_jobs", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_longlong),
                ("streams", ctypes.c_int), ("max_batch", ctypes.c_int), ("params", Params),
                ("step_work", ctypes.c_longlong)]


FG_REQ_DEVICE_INPUT, FG_REQ_DEVICE_OUTPUT = 1, 2
FG_ORDER_JACOBI, FG_ORDER_REDBLACK = 0, 1


class Request(ctypes.Structure):
    _fields_ = [("I", ctypes.c_void_p), ("alpha", ctypes.c_void_p), ("w", ctypes.c_int),
                ("h", ctypes.c_int), ("dtype", ctypes.c_int), ("F", ctypes.c_void_p),
                ("B", ctypes.c_void_p), ("flags", ctypes.c_int), ("ready_event", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_longlong) for n in
                ("submitted", "completed", "failed", "batches", "pixels", "max_inflight",
                 "max_bytes", "budget_bytes")]


def _server_lib():
    lib = load()
    if not getattr(lib, "_server_bound", False):
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        lib.fg_server_cfg_default.argtypes = [P(ServerCfg)]
        lib.fg_server_cfg_default.restype = None
        lib.fg_server_create.argtypes = [P(ServerCfg), P(vp)]
        lib.fg_server_create.restype = ctypes.c_int
        lib.fg_server_submit.argtypes = [vp, P(Request), P(ctypes.c_uint64)]
        lib.fg_server_submit.restype = ctypes.c_int
        lib.fg_server_poll.argtypes = [vp, ctypes.c_uint64, P(ctypes.c_int)]
        lib.fg_server_poll.restype = ctypes.c_int
        lib.fg_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_int]
        lib.fg_server_wait.restype = ctypes.c_int
        lib.fg_server_times.argtypes = [vp, ctypes.c_uint64, P(ctypes.c_double),
                                        P(ctypes.c_double)]
        lib.fg_server_times.restype = ctypes.c_int
        lib.fg_server_release.argtypes = [vp, ctypes.c_uint64]
        lib.fg_server_release.restype = ctypes.c_int
        lib.fg_server_get_stats.argtypes = [vp, P(ServerStats)]
        lib.fg_server_get_stats.restype = ctypes.c_int
        lib.fg_server_destroy.argtypes = [vp]
        lib.fg_server_destroy.restype = None
        lib.fg_server_last_error.argtypes = []
        lib.fg_server_last_error.restype = ctypes.c_char_p
        lib._server_bound = True
    return lib


class Server:
    """fg_server: continuous-batching job server on the current device, scheduled by level
    pass (each launch merges the next passes of every admitted job, up to step_work
    pixel-sweeps). Jobs are tensors (I [H, W, 3], alpha [H, W], one float dtype) in host or
    device memory; outputs are filled when the job completes. Keep the tensors alive until
    then."""

    def __init__(self, max_inflight_jobs=256, hbm_budget_bytes=0, streams=2, max_batch=64,
                 p: Params | None = None, step_work: int = 0):
        lib = _server_lib()
        cfg = ServerCfg()
        lib.fg_server_cfg_default(ctypes.byref(cfg))
        cfg.max_inflight_jobs = max_inflight_jobs
        cfg.hbm_budget_bytes = hbm_budget_bytes
        cfg.streams = streams
        cfg.max_batch = max_batch
        if step_work > 0:
            cfg.step_work = step_work
        if p is not None:
            cfg.params = p
        h = ctypes.c_void_p()
        st = lib.fg_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != FG_OK:
            raise FgmlError(st, lib.fg_server_last_error().decode())
        self._h = h
        self._lib = lib
        self._keep = {}

    def _check(self, st):
        if st != FG_OK:
            raise FgmlError(st, self._lib.fg_server_last_error().decode())

    def submit(self, I: torch.Tensor, alpha: torch.Tensor, F=None, B=None) -> int:
        """Queues a job. I and alpha may be host tensors or CUDA tensors of the server's
        device (read in place; their contents must be complete on the current stream,
        whose position is passed to the server as the job's ready event). F and B default
        to tensors of I's kind; a CUDA F and B are written in place."""
        I = I.contiguous()
        alpha = alpha.contiguous()
        h, w = alpha.shape
        if I.is_cuda != alpha.is_cuda:
            raise ValueError("I and alpha must both be host or both be CUDA tensors")
        pin = I.is_pinned()
        if F is None:
            F = torch.empty_like(I) if I.is_cuda else torch.empty(I.shape, dtype=I.dtype, pin_memory=pin)
        if B is None:
            B = torch.empty_like(I) if I.is_cuda else torch.empty(I.shape, dtype=I.dtype, pin_memory=pin)
        if F.is_cuda != B.is_cuda or not (F.is_contiguous() and B.is_contiguous()):
            raise ValueError("F and B must both be host or both be CUDA tensors, contiguous")
        flags = (FG_REQ_DEVICE_INPUT if I.is_cuda else 0) | (FG_REQ_DEVICE_OUTPUT if F.is_cuda else 0)
        ev = None
        if I.is_cuda:
            ev = torch.cuda.Event()
            ev.record()
        r = Request(I.data_ptr(), alpha.data_ptr(), w, h, _DTYPES[I.dtype], F.data_ptr(),
                    B.data_ptr(), flags, ev.cuda_event if ev is not None else None)
        t = ctypes.c_uint64()
        self._check(self._lib.fg_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        self._keep[t.value] = (I, alpha, F, B, ev)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        self._check(self._lib.fg_server_wait(self._h, ticket, timeout_ms))
        _, _, F, B, _ = self._keep[ticket]
        return F, B

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int()
        self._check(self._lib.fg_server_poll(self._h, ticket, ctypes.byref(d)))
        return bool(d.value)

    def times(self, ticket: int):
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.fg_server_times(self._h, ticket, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def release(self, ticket: int):
        self._check(self._lib.fg_server_release(self._h, ticket))
        self._keep.pop(ticket, None)

    def stats(self) -> dict:
        s = ServerStats()
        self._check(self._lib.fg_server_get_stats(self._h, ctypes.byref(s)))
        return {n: getattr(s, n) for n, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            self._lib.fg_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
