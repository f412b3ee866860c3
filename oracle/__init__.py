"""ORACLE -- test infrastructure only.

A plain fp64 CPU restatement of the paper's FSR and SSR reconstructions and of the general
n-order tree (Sec. III-B, Def. 2, Fig. 1, Eq. 4), written in C (``oracle.c``) and driven through ctypes, plus a pure-Python
literal reading of Def. 2 for tiny inputs (``bruteforce.py``).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it; the
library in ``paper_2412_11639_gb300`` never does, and the two share no code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into an in-tree shared library (plain C, OpenMP over pixels)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        c = ctypes
        lib.oracle_reconstruct.argtypes = [c.c_void_p, c.c_int64, c.c_int64, c.c_int, c.c_double,
                                           c.c_int, c.c_int, c.c_void_p, c.c_int64, c.c_void_p,
                                           c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p,
                                           c.c_void_p, c.c_void_p, c.c_void_p]
        lib.oracle_reconstruct.restype = c.c_int
        lib.oracle_reconstruct2.argtypes = lib.oracle_reconstruct.argtypes + [c.c_int, c.c_int]
        lib.oracle_reconstruct2.restype = c.c_int
        lib.oracle_u8.argtypes = [c.c_int64, c.c_int64, c.c_int64]
        lib.oracle_u8.restype = c.c_int
        lib.oracle_spike_times.argtypes = [c.c_void_p, c.c_int64, c.c_int, c.c_int64, c.c_void_p]
        lib.oracle_spike_times.restype = c.c_int
        lib.oracle_set_threads.argtypes = [c.c_int]
        lib.oracle_set_threads.restype = None
        lib.oracle_segments_n.argtypes = [c.c_void_p, c.c_int, c.c_int, c.c_double, c.c_void_p,
                                          c.c_void_p, c.c_void_p, c.c_void_p]
        lib.oracle_segments_n.restype = c.c_int
        lib.oracle_tfi.argtypes = [c.c_void_p, c.c_int64, c.c_int64, c.c_int, c.c_double, c.c_int,
                                   c.c_void_p, c.c_int64, c.c_void_p]
        lib.oracle_tfi.restype = c.c_int
        lib.oracle_tfi2.argtypes = lib.oracle_tfi.argtypes + [c.c_int, c.c_int]
        lib.oracle_tfi2.restype = c.c_int
        lib.oracle_tfp.argtypes = [c.c_void_p, c.c_int64, c.c_int64, c.c_int, c.c_double, c.c_int,
                                   c.c_int, c.c_void_p, c.c_int64, c.c_void_p]
        lib.oracle_tfp.restype = c.c_int
        lib.oracle_tfp2.argtypes = lib.oracle_tfp.argtypes + [c.c_int]
        lib.oracle_tfp2.restype = c.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def spike_times(stream: np.ndarray, T: int, p: int) -> np.ndarray:
    """Spike times of pixel p (step 1)."""
    stream = np.ascontiguousarray(stream)
    out = np.empty(T, dtype=np.int32)
    K = _load().oracle_spike_times(stream.ctypes.data, stream.shape[1], T, p, out.ctypes.data)
    return out[:K].copy()


def set_threads(n: int = 0):
    """Threads of the pixel loops (0: every core)."""
    _load().oracle_set_threads(n)


def segments_n(times, n: int, theta: float = 1.0):
    """Stable sequences of one pixel's spike times under the general n-order tree:
    [(t_start, t_end, N, value)] (orders 1 and 2 are FSR and SSR)."""
    s = np.ascontiguousarray(times, dtype=np.int32)
    K = s.shape[0]
    cap = max(K, 1)
    ts, te, nn = (np.empty(cap, dtype=np.int32) for _ in range(3))
    vv = np.empty(cap, dtype=np.float64)
    ns = _load().oracle_segments_n(s.ctypes.data, K, n, theta, ts.ctypes.data, te.ctypes.data,
                                   nn.ctypes.data, vv.ctypes.data)
    return [(int(ts[j]), int(te[j]), int(nn[j]), float(vv[j])) for j in range(ns)]


class Result:
    """Oracle output for a set of pixels.

    frames:   fp64 [T_out][npix] (or None)
    K:        int32 [npix] spike counts
    nseg:     int32 [npix] stable-sequence counts
    seg_off:  int64 [npix+1] offsets into the seg_* arrays (when segments were asked for)
    seg_ts, seg_te, seg_n: int32 start spike time, end spike time, interval count
    seg_val:  fp64 theta * N / (t_end - t_start)
    """

    def __init__(self):
        self.frames = self.K = self.nseg = self.seg_off = None
        self.seg_ts = self.seg_te = self.seg_n = self.seg_val = None

    def segments(self, i: int):
        a, b = self.seg_off[i], self.seg_off[i + 1]
        return (self.seg_ts[a:b], self.seg_te[a:b], self.seg_n[a:b], self.seg_val[a:b])


ZERO_HEAD, ZERO_TAIL = 1, 2   # frame edge policy bits


def u8(theta: int, N: int, D: int) -> int:
    """8-bit value of a sequence of N intervals over D steps: theta * N / D rounded half up,
    clamped to 255 (theta integral)."""
    return _load().oracle_u8(theta, N, D)


def reconstruct(stream: np.ndarray, H: int, W: int, T: int, theta: float = 1.0, order: int = 1,
                stride: int = 1, pixels=None, frames: bool = True,
                segments: bool = False, edges: int = 0, u8: bool = False) -> Result:
    """Run the oracle on packed stream [T][pitch] for the given pixels (default: all).
    order 1 = FSR, 2 = SSR, n > 2 = the general n-order tree (up to 32).  edges: ZERO_HEAD
    and/or ZERO_TAIL (frames up to the first / after the last spike read 0 instead of the
    edge sequence's value); u8: frames hold the 8-bit values (theta integral)."""
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    if stream.ndim != 2 or stream.shape[0] < T:
        raise ValueError("stream must be [T][pitch]")
    P = H * W
    pitch = stream.shape[1]
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int64)
    npix = P if pix is None else pix.shape[0]
    T_out = (T + stride - 1) // stride
    r = Result()
    r.K = np.empty(npix, dtype=np.int32)
    r.nseg = np.empty(npix, dtype=np.int32)
    lib = _load()
    fr = np.empty((T_out, npix), dtype=np.float64) if frames else None
    rc = lib.oracle_reconstruct2(stream.ctypes.data, pitch, P, T, theta, order, stride, _ptr(pix),
                                 npix, _ptr(fr), r.K.ctypes.data, r.nseg.ctypes.data,
                                 None, None, None, None, None, edges, int(bool(u8)))
    if rc != 0:
        raise ValueError(f"oracle_reconstruct failed ({rc})")
    r.frames = fr
    if segments:
        off = np.zeros(npix + 1, dtype=np.int64)
        np.cumsum(r.nseg, out=off[1:])
        tot = int(off[-1])
        r.seg_off = off
        r.seg_ts = np.empty(tot, dtype=np.int32)
        r.seg_te = np.empty(tot, dtype=np.int32)
        r.seg_n = np.empty(tot, dtype=np.int32)
        r.seg_val = np.empty(tot, dtype=np.float64)
        rc = lib.oracle_reconstruct(stream.ctypes.data, pitch, P, T, theta, order, stride,
                                    _ptr(pix), npix, None, None, None, off.ctypes.data,
                                    r.seg_ts.ctypes.data, r.seg_te.ctypes.data,
                                    r.seg_n.ctypes.data, r.seg_val.ctypes.data)
        if rc != 0:
            raise ValueError(f"oracle_reconstruct (segments) failed ({rc})")
    return r


def tfi(stream: np.ndarray, H: int, W: int, T: int, theta: float = 1.0, stride: int = 1,
        pixels=None, edges: int = 0, u8: bool = False) -> np.ndarray:
    """TFI baseline (Sec. II): frames fp64 [T_out][npix] (8-bit values with u8)."""
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int64)
    npix = H * W if pix is None else pix.shape[0]
    out = np.empty(((T + stride - 1) // stride, npix), dtype=np.float64)
    rc = _load().oracle_tfi2(stream.ctypes.data, stream.shape[1], H * W, T, theta, stride, _ptr(pix),
                             npix, out.ctypes.data, edges, int(bool(u8)))
    if rc != 0:
        raise ValueError(f"oracle_tfi failed ({rc})")
    return out


def tfp(stream: np.ndarray, H: int, W: int, T: int, window: int, theta: float = 1.0,
        stride: int = 1, pixels=None, u8: bool = False) -> np.ndarray:
    """TFP baseline (Sec. II) with a window of `window` steps: frames fp64 [T_out][npix]
    (8-bit values with u8)."""
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int64)
    npix = H * W if pix is None else pix.shape[0]
    out = np.empty(((T + stride - 1) // stride, npix), dtype=np.float64)
    rc = _load().oracle_tfp2(stream.ctypes.data, stream.shape[1], H * W, T, theta, stride, window,
                             _ptr(pix), npix, out.ctypes.data, int(bool(u8)))
    if rc != 0:
        raise ValueError(f"oracle_tfp failed ({rc})")
    return out
