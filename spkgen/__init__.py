"""Seeded synthetic spike streams (the input recipe shared by the oracle and the CUDA path).

The sensor is the discrete integrate-and-fire model of Eq. 2 (Sec. II): subtract-on-fire,
threshold theta, one decision per step.  Scenes are a periodic texture (a base level,
32 Gaussian blobs and 2 sinusoidal gratings) that may translate, be multiplied by abrupt
step events and carry Bernoulli dark noise.  The sizes follow the paper's sensor
(400 x 250 pixels at 20 kHz, Sec. IV-A) and a large 1000 x 1000 sensor.

This package holds none of the reconstruction arithmetic: it only writes spike streams.
Random parameters come from NumPy's PCG64 seeded per workload; per-pixel initial
accumulators and dark noise come from a counter-based SplitMix64 hash of (seed, pixel, step).

Stream layout: ``uint8 [T][pitch]`` with ``pitch = round_up(ceil(H*W/8), 16)``; pixel
``p = y*W + x`` is bit ``p % 8`` (LSB first) of byte ``p // 8`` of its frame.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_SO = os.path.join(_HERE, "_spkgen.so")
_lib = None


_CU_SRC = os.path.join(_HERE, "gen.cu")
_CU_SO = os.path.join(_HERE, "_spkgen_cuda.so")
_culib = None


def build(force: bool = False) -> str:
    """Compile gen.c (plain C, OpenMP, no FMA contraction) and gen.cu (the GPU twin, sm_103a,
    -fmad=false) into in-tree shared libraries."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    if force or not os.path.exists(_CU_SO) or os.path.getmtime(_CU_SO) < os.path.getmtime(_CU_SRC):
        tmp = _CU_SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                               "-fmad=false", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                               _CU_SRC, "-o", tmp])
        os.replace(tmp, _CU_SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        c = ctypes
        lib.spkgen_render_texture.argtypes = [c.c_void_p, c.c_int, c.c_double, c.c_int,
                                              c.c_void_p, c.c_int, c.c_void_p]
        lib.spkgen_render_texture.restype = None
        lib.spkgen_simulate.argtypes = [c.c_void_p, c.c_int64, c.c_int, c.c_int, c.c_int,
                                        c.c_void_p, c.c_int, c.c_double, c.c_double, c.c_double,
                                        c.c_double, c.c_int, c.c_void_p, c.c_double, c.c_double,
                                        c.c_double, c.c_uint64, c.c_double, c.c_void_p, c.c_int]
        lib.spkgen_simulate.restype = c.c_int
        lib.spkgen_simulate_table.argtypes = [c.c_void_p, c.c_int64, c.c_int64, c.c_int,
                                              c.c_void_p, c.c_void_p, c.c_double]
        lib.spkgen_simulate_table.restype = c.c_int
        lib.spkgen_uniform.argtypes = [c.c_uint64] * 4
        lib.spkgen_uniform.restype = c.c_double
        _lib = lib
    return _lib


def pitch(H: int, W: int) -> int:
    """Bytes per frame: ceil(H*W/8) rounded up to a multiple of 16."""
    nbytes = (H * W + 7) // 8
    return (nbytes + 15) // 16 * 16


def num_frames(T: int, stride: int) -> int:
    return (T + stride - 1) // stride


@dataclass(frozen=True)
class Workload:
    """One synthetic workload: sensor size, length, frame stride, scene recipe."""
    name: str
    H: int
    W: int
    T: int
    stride: int
    out_dtype: str            # "f32" | "f16"
    seed: int
    ilo: float                # intensity clip range (theta = 1)
    ihi: float = 1.0
    moving: bool = False      # translate at U[0.01, 2] px/step in a random direction
    n_events: int = 0         # abrupt step events (factor U[2, 10] or its inverse)
    noise_p: float = 0.0      # Bernoulli dark-noise rate per pixel-step
    theta: float = 1.0
    L: int = 1024             # torus side of the texture table

    @property
    def P(self) -> int:
        return self.H * self.W

    @property
    def pitch(self) -> int:
        return pitch(self.H, self.W)

    @property
    def T_out(self) -> int:
        return num_frames(self.T, self.stride)

    def resized(self, **kw) -> "Workload":
        """Same scene recipe and seed at other sizes (smaller parity cases)."""
        return replace(self, **kw)


WORKLOADS = {
    # static scene: each pixel sees a constant intensity (Theorem 1 regime)
    "static_250x400x2000": Workload("static_250x400x2000", 250, 400, 2000, 1, "f32", seed=1,
                                    ilo=0.02),
    # moving texture, step events, dark noise; a frame every 10 steps
    "dynamic_250x400x20000": Workload("dynamic_250x400x20000", 250, 400, 20000, 10, "f32",
                                      seed=2, ilo=0.02, moving=True, n_events=8, noise_p=1e-4),
    # large sensor, moving texture, fp16 frame every step
    "large_1000x1000x20000": Workload("large_1000x1000x20000", 1000, 1000, 20000, 1, "f16",
                                      seed=3, ilo=0.005, moving=True),
}


@dataclass
class Scene:
    tex: np.ndarray
    x0: float
    y0: float
    vx: float
    vy: float
    events: np.ndarray = field(default_factory=lambda: np.zeros((0, 6)))


def scene(w: Workload) -> Scene:
    """Draw the texture, motion and events of a workload from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(w.seed))
    L = w.L
    blobs = np.stack([rng.uniform(0, L, 32), rng.uniform(0, L, 32),
                      rng.uniform(4, 64, 32), rng.uniform(-0.4, 0.4, 32)], axis=1)
    grats = np.stack([rng.uniform(0.05, 0.2, 2), rng.uniform(6, 64, 2),
                      rng.uniform(0, math.pi, 2), rng.uniform(0, 2 * math.pi, 2)], axis=1)
    tex = np.empty((L, L), dtype=np.float64)
    lib = _load()
    blobs = np.ascontiguousarray(blobs)
    grats = np.ascontiguousarray(grats)
    lib.spkgen_render_texture(tex.ctypes.data, L, 0.5, 32, blobs.ctypes.data, 2, grats.ctypes.data)
    x0, y0 = rng.uniform(0, L, 2)
    vx = vy = 0.0
    if w.moving:
        speed = rng.uniform(0.01, 2.0)
        ang = rng.uniform(0, 2 * math.pi)
        vx, vy = speed * math.cos(ang), speed * math.sin(ang)
    ev = []
    for _ in range(w.n_events):
        t = int(rng.integers(0, w.T))
        if rng.uniform() < 0.25:
            y_lo, x_lo, y_hi, x_hi = 0, 0, w.H, w.W
        else:
            h = int(rng.integers((w.H + 1) // 2, w.H + 1))
            wd = int(rng.integers((w.W + 1) // 2, w.W + 1))
            y_lo = int(rng.integers(0, w.H - h + 1))
            x_lo = int(rng.integers(0, w.W - wd + 1))
            y_hi, x_hi = y_lo + h, x_lo + wd
        f = rng.uniform(2.0, 10.0)
        if rng.uniform() < 0.5:
            f = 1.0 / f
        ev.append((t, y_lo, x_lo, y_hi, x_hi, f))
    events = np.array(ev, dtype=np.float64).reshape(-1, 6)
    return Scene(tex, float(x0), float(y0), vx, vy, events)


def make_stream(w: Workload, gt_stride: int | None = None):
    """Simulate the workload; returns (stream uint8 [T][pitch], gt float32 or None).

    gt, when asked for, holds the clipped intensity at every gt_stride-th step:
    shape [ceil(T/gt_stride)][H*W].
    """
    sc = scene(w)
    out = np.empty((w.T, w.pitch), dtype=np.uint8)
    gt = None
    if gt_stride:
        gt = np.empty((num_frames(w.T, gt_stride), w.P), dtype=np.float32)
    ev = np.ascontiguousarray(sc.events)
    rc = _load().spkgen_simulate(out.ctypes.data, w.pitch, w.H, w.W, w.T, sc.tex.ctypes.data, w.L,
                                 sc.x0, sc.y0, sc.vx, sc.vy, ev.shape[0],
                                 ev.ctypes.data if ev.size else None, w.ilo, w.ihi, w.theta,
                                 w.seed, w.noise_p, gt.ctypes.data if gt is not None else None,
                                 gt_stride or 0)
    if rc != 0:
        raise ValueError("spkgen_simulate rejected its arguments")
    return out, gt


def simulate_table(q: np.ndarray, r0: np.ndarray, theta: float = 1.0, H: int | None = None,
                   W: int | None = None) -> np.ndarray:
    """Eq. 2 for explicit intensities q [T][P] and initial accumulators r0 [P]."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    r0 = np.ascontiguousarray(r0, dtype=np.float64)
    T, P = q.shape
    if H is None:
        H, W = 1, P
    pt = pitch(H, W)
    out = np.empty((T, pt), dtype=np.uint8)
    rc = _load().spkgen_simulate_table(out.ctypes.data, pt, P, T, q.ctypes.data, r0.ctypes.data,
                                       theta)
    if rc != 0:
        raise ValueError("spkgen_simulate_table rejected its arguments")
    return out


def pack(bits: np.ndarray, H: int | None = None, W: int | None = None) -> np.ndarray:
    """Pack a 0/1 array [T][P] into the stream layout (LSB-first, 16-byte pitch)."""
    bits = np.asarray(bits).astype(np.uint8)
    T, P = bits.shape
    if H is None:
        H, W = 1, P
    pt = pitch(H, W)
    out = np.zeros((T, pt), dtype=np.uint8)
    packed = np.packbits(bits, axis=1, bitorder="little")
    out[:, :packed.shape[1]] = packed
    return out


def random_bits(T: int, P: int, density: float, seed: int) -> np.ndarray:
    """Independent Bernoulli(density) spikes [T][P] (uint8) from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.random((T, P)) < density).astype(np.uint8)


def uniform(seed: int, stream: int, a: int, b: int) -> float:
    """The counter-based uniform the simulator draws (exposed for the pins)."""
    return _load().spkgen_uniform(seed, stream, a, b)


def _load_cuda():
    global _culib
    if _culib is None:
        build()
        lib = ctypes.CDLL(_CU_SO)
        c = ctypes
        lib.spkgen_cuda_simulate.argtypes = [c.c_void_p, c.c_int64, c.c_int, c.c_int, c.c_int,
                                             c.c_void_p, c.c_int, c.c_double, c.c_double,
                                             c.c_double, c.c_double, c.c_int, c.c_void_p,
                                             c.c_double, c.c_double, c.c_double, c.c_uint64,
                                             c.c_double, c.c_void_p, c.c_int, c.c_void_p]
        lib.spkgen_cuda_simulate.restype = c.c_int
        _culib = lib
    return _culib


def make_stream_cuda(w: Workload, gt_stride: int | None = None, device: int = 0, stream=None):
    """make_stream on the GPU (gen.cu): the same bits, as torch CUDA tensors.

    Returns (stream uint8 [T][pitch], gt float32 [ceil(T/gt_stride)][H*W] or None).  The
    texture table is rendered on the host exactly as for make_stream.
    """
    import torch
    sc = scene(w)
    dev = f"cuda:{device}"
    tex = torch.from_numpy(sc.tex).to(dev)
    out = torch.empty((w.T, w.pitch), dtype=torch.uint8, device=dev)
    gt = None
    if gt_stride:
        gt = torch.empty((num_frames(w.T, gt_stride), w.P), dtype=torch.float32, device=dev)
    ev = np.ascontiguousarray(sc.events)
    cs = stream if stream is not None else torch.cuda.current_stream(device)
    rc = _load_cuda().spkgen_cuda_simulate(out.data_ptr(), w.pitch, w.H, w.W, w.T, tex.data_ptr(),
                                           w.L, sc.x0, sc.y0, sc.vx, sc.vy, ev.shape[0],
                                           ev.ctypes.data if ev.size else None, w.ilo, w.ihi,
                                           w.theta, w.seed, w.noise_p,
                                           gt.data_ptr() if gt is not None else None,
                                           gt_stride or 0, cs.cuda_stream)
    if rc != 0:
        raise ValueError(f"spkgen_cuda_simulate failed ({rc})")
    cs.synchronize()           # tex is freed when this function returns
    return out, gt
