"""Thin ctypes binding of libspk.so (include/spk.h): argument marshalling only.

Every entry point keeps its C name.  Device buffers may be given as torch tensors or
raw integer addresses; every step of the reconstruction runs in the CUDA kernels of
libspk.so.  There is no CPU fallback: if the library is missing, calls raise.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB

SPK_OK, SPK_ERR_ARG, SPK_ERR_CUDA, SPK_ERR_OOM, SPK_ERR_TIMEOUT, SPK_ERR_INTERNAL = 0, -1, -2, -3, -4, -5
SPK_F32, SPK_F16, SPK_U8 = 0, 1, 2
SPK_ZERO_HEAD, SPK_ZERO_TAIL = 1, 2  # frame edge policy bits
SPK_FSR, SPK_SSR, SPK_TFI, SPK_TFP, SPK_NORDER = 1, 2, 3, 4, 5

_c = ctypes
EXPORTS = ("spk_create", "spk_destroy", "spk_pitch", "spk_num_frames", "spk_reconstruct",
           "spk_reconstruct_host", "spk_segments", "spk_synchronize", "spk_last_error",
           "spk_launch_count", "spk_reconstruct_host_noalloc", "spk_selftest_wait", "spk_stream_open",
           "spk_stream_close", "spk_stream_steps", "spk_stream_ready", "spk_run", "spk_set_tile",
           "spk_get_tile", "spk_autotune", "spk_features", "spk_refiner_num_params",
           "spk_refiner_create", "spk_refiner_destroy", "spk_refiner_last_error",
           "spk_refiner_set_params", "spk_refiner_get_params", "spk_refiner_forward",
           "spk_refiner_train_step", "spk_refiner_synchronize", "spk_reconstruct_host_async",
           "spk_debug_fail_allocations", "spk_debug_norder_capacity")
SPK_NOALLOC_SCRATCH_BYTES = 16 << 20


class SpkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class spk_config(ctypes.Structure):
    _fields_ = [("method", _c.c_int), ("frame_stride", _c.c_int), ("out_dtype", _c.c_int),
                ("device", _c.c_int), ("stream", _c.c_void_p), ("tfp_window", _c.c_int),
                ("stability_order", _c.c_int), ("edges", _c.c_int)]


class spk_job(ctypes.Structure):
    _fields_ = [("stream", _c.c_void_p), ("H", _c.c_int), ("W", _c.c_int), ("n", _c.c_int),
                ("threshold", _c.c_float), ("out_frames", _c.c_void_p), ("state", _c.c_void_p)]


_lib = None


def load(path: str | None = None):
    """Load libspk.so (built by build.build()); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libspk.so not found at {path}: run paper_2412_11639_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, f32 = _c.c_void_p, _c.c_int, _c.c_int64, _c.c_float
    lib.spk_create.argtypes = [_c.POINTER(vp), _c.POINTER(spk_config)]
    lib.spk_create.restype = i32
    lib.spk_destroy.argtypes = [vp]
    lib.spk_destroy.restype = i32
    lib.spk_pitch.argtypes = [i32, i32]
    lib.spk_pitch.restype = i64
    lib.spk_num_frames.argtypes = [i32, i32]
    lib.spk_num_frames.restype = i64
    lib.spk_reconstruct.argtypes = [vp, vp, i32, i32, i32, f32, vp]
    lib.spk_reconstruct.restype = i32
    lib.spk_reconstruct_host.argtypes = [vp, vp, i32, i32, i32, f32, vp]
    lib.spk_reconstruct_host.restype = i32
    lib.spk_reconstruct_host_async.argtypes = [vp, vp, i32, i32, i32, f32, vp]
    lib.spk_reconstruct_host_async.restype = i32
    lib.spk_segments.argtypes = [vp, vp, i32, i32, i32, f32, vp, vp, vp, vp, vp, vp, i32]
    lib.spk_segments.restype = i32
    lib.spk_synchronize.argtypes = [vp]
    lib.spk_synchronize.restype = i32
    lib.spk_last_error.argtypes = [vp]
    lib.spk_last_error.restype = _c.c_char_p
    lib.spk_launch_count.argtypes = [vp]
    lib.spk_launch_count.restype = i64
    lib.spk_stream_open.argtypes = [vp, i32, i32, i32, _c.POINTER(vp)]
    lib.spk_stream_open.restype = i32
    lib.spk_stream_close.argtypes = [vp, vp]
    lib.spk_stream_close.restype = i32
    lib.spk_stream_steps.argtypes = [vp]
    lib.spk_stream_steps.restype = i64
    lib.spk_stream_ready.argtypes = [vp, vp, _c.POINTER(i64)]
    lib.spk_stream_ready.restype = i32
    lib.spk_run.argtypes = [vp, _c.POINTER(spk_job), i32]
    lib.spk_run.restype = i32
    lib.spk_set_tile.argtypes = [vp, i32]
    lib.spk_set_tile.restype = i32
    lib.spk_get_tile.argtypes = [vp]
    lib.spk_get_tile.restype = i32
    lib.spk_autotune.argtypes = [vp, _c.POINTER(spk_job), i32, _c.POINTER(i32)]
    lib.spk_autotune.restype = i32
    lib.spk_features.argtypes = [vp, vp, i32, i32, i32, f32, vp, vp]
    lib.spk_features.restype = i32
    lib.spk_refiner_num_params.argtypes = []
    lib.spk_refiner_num_params.restype = i64
    lib.spk_refiner_create.argtypes = [i32, _c.c_uint64, _c.POINTER(vp)]
    lib.spk_refiner_create.restype = i32
    lib.spk_refiner_destroy.argtypes = [vp]
    lib.spk_refiner_destroy.restype = i32
    lib.spk_refiner_last_error.argtypes = [vp]
    lib.spk_refiner_last_error.restype = _c.c_char_p
    lib.spk_refiner_set_params.argtypes = [vp, vp, i64]
    lib.spk_refiner_set_params.restype = i32
    lib.spk_refiner_get_params.argtypes = [vp, vp, i64, i32]
    lib.spk_refiner_get_params.restype = i32
    lib.spk_refiner_forward.argtypes = [vp, vp, vp, vp, i32, i32, i32, vp]
    lib.spk_refiner_forward.restype = i32
    lib.spk_refiner_train_step.argtypes = [vp, vp, vp, vp, vp, i32, i32, i32, f32, _c.POINTER(f32)]
    lib.spk_refiner_train_step.restype = i32
    lib.spk_refiner_synchronize.argtypes = [vp, vp]
    lib.spk_refiner_synchronize.restype = i32
    lib.spk_debug_fail_allocations.argtypes = [i32]
    lib.spk_debug_fail_allocations.restype = i32
    lib.spk_debug_norder_capacity.argtypes = [i32]
    lib.spk_debug_norder_capacity.restype = i32
    lib.spk_selftest_wait.argtypes = [vp, i64]
    lib.spk_selftest_wait.restype = i32
    lib.spk_reconstruct_host_noalloc.argtypes = [_c.POINTER(spk_config), vp, i32, i32, i32, f32, vp]
    lib.spk_reconstruct_host_noalloc.restype = i32
    _lib = lib
    return lib


def _addr(x):
    """Device/host address of a tensor, a numpy array, or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _check(ctx, rc):
    if rc != SPK_OK:
        msg = load().spk_last_error(ctx)
        raise SpkError(rc, msg.decode() if msg else "")
    return rc


_CTX_FRAMES = {}  # context handle -> (frame_stride, bytes per output value), for host-buffer checks


def _esz(out_dtype: int) -> int:
    """Bytes per frame value of an output type."""
    return 2 if out_dtype == SPK_F16 else 1 if out_dtype == SPK_U8 else 4


def spk_create(method: int = SPK_SSR, frame_stride: int = 1, out_dtype: int = SPK_F32, device: int = 0,
               stream: int | None = None, tfp_window: int = 32, stability_order: int = 3, edges: int = 0):
    lib = load()
    cfg = spk_config(method, frame_stride, out_dtype, device, stream, tfp_window, stability_order, edges)
    ctx = _c.c_void_p()
    rc = lib.spk_create(_c.byref(ctx), _c.byref(cfg))
    _check(None, rc)
    _CTX_FRAMES[ctx.value] = (frame_stride, _esz(out_dtype))
    return ctx


def spk_destroy(ctx):
    _CTX_FRAMES.pop(getattr(ctx, "value", ctx), None)
    return load().spk_destroy(ctx)


def _nbytes_contiguous(x, name):
    """Size in bytes of a C-contiguous host buffer (numpy array or CPU tensor)."""
    if hasattr(x, "is_contiguous"):          # torch tensor
        if x.is_cuda or not x.is_contiguous():
            raise ValueError(f"{name} must be a C-contiguous host tensor")
        return x.numel() * x.element_size()
    flags = getattr(x, "flags", None)
    if flags is None or not flags["C_CONTIGUOUS"]:
        raise ValueError(f"{name} must be a C-contiguous array")
    return x.nbytes


def _check_host_buffers(host_stream, host_frames, H, W, T, stride, esz, frames_dtype=None):
    """The C side reads T * pitch bytes and writes T_out * H * W * esz bytes: refuse buffers
    that are smaller, strided, or (when known) of the wrong element size."""
    if H <= 0 or W <= 0 or T <= 0 or stride <= 0:
        return  # the library rejects these itself
    need_in = T * ((((H * W + 7) // 8) + 15) // 16 * 16)
    need_out = -(-T // stride) * H * W * esz
    if _nbytes_contiguous(host_stream, "host_stream") < need_in:
        raise ValueError(f"host_stream holds fewer than T * pitch = {need_in} bytes")
    if _nbytes_contiguous(host_frames, "host_frames") < need_out:
        raise ValueError(f"host_frames holds fewer than T_out * H * W * {esz} = {need_out} bytes")
    item = getattr(getattr(host_frames, "dtype", None), "itemsize", None)
    if item is None and hasattr(host_frames, "element_size"):
        item = host_frames.element_size()
    if item is not None and item != esz:
        raise ValueError(f"host_frames has {item}-byte elements, the output type has {esz}")


def spk_pitch(H: int, W: int) -> int:
    return load().spk_pitch(H, W)


def spk_num_frames(T: int, stride: int) -> int:
    return load().spk_num_frames(T, stride)


def spk_reconstruct(ctx, stream, H, W, T, threshold, out_frames):
    return _check(ctx, load().spk_reconstruct(ctx, _addr(stream), H, W, T, threshold, _addr(out_frames)))


def spk_reconstruct_host(ctx, host_stream, H, W, T, threshold, host_frames):
    if getattr(ctx, "value", None) in _CTX_FRAMES:
        _check_host_buffers(host_stream, host_frames, H, W, T, *_CTX_FRAMES[ctx.value])
    return _check(ctx, load().spk_reconstruct_host(ctx, _addr(host_stream), H, W, T, threshold,
                                                   _addr(host_frames)))


def spk_segments(ctx, stream, H, W, T, threshold, spike_counts, counts, t_start, t_end, n_int, value, cap):
    return _check(ctx, load().spk_segments(ctx, _addr(stream), H, W, T, threshold, _addr(spike_counts),
                                           _addr(counts), _addr(t_start), _addr(t_end), _addr(n_int),
                                           _addr(value), cap))


def spk_synchronize(ctx):
    return _check(ctx, load().spk_synchronize(ctx))


def spk_last_error(ctx) -> str:
    m = load().spk_last_error(ctx)
    return m.decode() if m else ""


def spk_launch_count(ctx) -> int:
    return load().spk_launch_count(ctx)


def spk_selftest_wait(ctx, limit_cycles: int):
    return _check(ctx, load().spk_selftest_wait(ctx, limit_cycles))


def spk_reconstruct_host_noalloc(host_stream, H, W, T, threshold, host_frames, method: int = SPK_SSR,
                                 frame_stride: int = 1, out_dtype: int = SPK_F32, device: int = 0,
                                 stream: int | None = None, tfp_window: int = 32,
                                 stability_order: int = 3, edges: int = 0):
    """Host-buffer reconstruction staged in the library's fixed device array (no allocation).
    method: 1 FSR, 2 SSR, 3 TFI, 4 TFP (window tfp_window), 5 the n-order tree
    (stability_order levels, 3..5).  Raises ValueError, before any device work, if a buffer is
    strided or smaller than the call reads or writes."""
    _check_host_buffers(host_stream, host_frames, H, W, T, frame_stride, _esz(out_dtype))
    cfg = spk_config(method, frame_stride, out_dtype, device, stream, tfp_window, stability_order, edges)
    rc = load().spk_reconstruct_host_noalloc(_c.byref(cfg), _addr(host_stream), H, W, T, threshold,
                                             _addr(host_frames))
    return _check(None, rc)


def spk_stream_open(ctx, H: int, W: int, T: int):
    out = _c.c_void_p()
    _check(ctx, load().spk_stream_open(ctx, H, W, T, _c.byref(out)))
    return out


def spk_stream_close(ctx, state):
    return load().spk_stream_close(ctx, state)


def spk_stream_steps(state) -> int:
    return load().spk_stream_steps(state)


def spk_stream_ready(ctx, state) -> int:
    r = _c.c_int64()
    _check(ctx, load().spk_stream_ready(ctx, state, _c.byref(r)))
    return r.value


def _jobs(jobs):
    arr = (spk_job * max(len(jobs), 1))()
    for k, (st, H, W, n, th, out, state) in enumerate(jobs):
        arr[k] = spk_job(_addr(st), H, W, n, th, _addr(out), state)
    return arr


def spk_run(ctx, jobs):
    """jobs: sequence of (stream, H, W, n, threshold, out_frames, state_or_None)."""
    return _check(ctx, load().spk_run(ctx, _jobs(jobs), len(jobs)))


def spk_set_tile(ctx, tile: int):
    return _check(ctx, load().spk_set_tile(ctx, tile))


def spk_get_tile(ctx) -> int:
    return load().spk_get_tile(ctx)


def spk_autotune(ctx, jobs) -> int:
    best = _c.c_int()
    _check(ctx, load().spk_autotune(ctx, _jobs(jobs), len(jobs), _c.byref(best)))
    return best.value


def spk_features(ctx, stream, H, W, T, threshold, plain, x0):
    return _check(ctx, load().spk_features(ctx, _addr(stream), H, W, T, threshold, _addr(plain), _addr(x0)))


def _rcheck(r, rc):
    if rc != SPK_OK:
        msg = load().spk_refiner_last_error(r)
        raise SpkError(rc, msg.decode() if msg else "")
    return rc


def spk_refiner_num_params() -> int:
    return load().spk_refiner_num_params()


def spk_refiner_create(device: int = 0, seed: int = 0):
    out = _c.c_void_p()
    _rcheck(None, load().spk_refiner_create(device, seed, _c.byref(out)))
    return out


def spk_refiner_destroy(r):
    return load().spk_refiner_destroy(r)


def spk_refiner_set_params(r, host):
    return _rcheck(r, load().spk_refiner_set_params(r, _addr(host), len(host)))


def spk_refiner_get_params(r, host, which: int = 0):
    return _rcheck(r, load().spk_refiner_get_params(r, _addr(host), len(host), which))


def spk_refiner_forward(r, stream, x0, plain, N, H, W, out):
    return _rcheck(r, load().spk_refiner_forward(r, stream, _addr(x0), _addr(plain), N, H, W, _addr(out)))


def spk_refiner_train_step(r, stream, x0, plain, gt, N, H, W, lr, want_loss=True):
    loss = _c.c_float(float("nan"))
    _rcheck(r, load().spk_refiner_train_step(r, stream, _addr(x0), _addr(plain), _addr(gt), N, H, W, lr,
                                             _c.byref(loss) if want_loss else None))
    return loss.value


def spk_refiner_synchronize(r, stream=None):
    return _rcheck(r, load().spk_refiner_synchronize(r, stream))


def spk_reconstruct_host_async(ctx, host_stream, H, W, T, threshold, host_frames):
    """Enqueue a host-buffer reconstruction (copies included); spk_synchronize(ctx) waits."""
    if getattr(ctx, "value", None) in _CTX_FRAMES:
        _check_host_buffers(host_stream, host_frames, H, W, T, *_CTX_FRAMES[ctx.value])
    return _check(ctx, load().spk_reconstruct_host_async(ctx, _addr(host_stream), H, W, T, threshold,
                                                         _addr(host_frames)))


def spk_debug_fail_allocations(n: int):
    """Make the library's next n device allocations fail (test hook of the SPK_ERR_OOM paths)."""
    return _check(None, load().spk_debug_fail_allocations(n))


def spk_debug_norder_capacity(cap: int):
    """First pending-cut ring size (cuts per pixel) of later n-order calls; 0 restores 64."""
    return _check(None, load().spk_debug_norder_capacity(cap))
