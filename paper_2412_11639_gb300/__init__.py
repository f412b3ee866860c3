"""GB300-native spike-camera reconstruction (FSR / SSR of arXiv 2412.11639).

The work happens in libspk.so (CUDA, sm_103a) behind the C ABI of include/spk.h;
``spk`` is its ctypes binding and ``Reconstructor`` a convenience wrapper that takes
torch tensors for device memory and streams.
"""
from __future__ import annotations

from . import spk
from .build import build
from .spk import (SPK_F16, SPK_F32, SPK_U8, SPK_ZERO_HEAD, SPK_ZERO_TAIL, SpkError, spk_create, spk_destroy, spk_launch_count,
                  spk_last_error, spk_num_frames, spk_pitch, spk_reconstruct,
                  spk_reconstruct_host, spk_reconstruct_host_async, spk_run, spk_segments,
                  spk_stream_close, spk_stream_open, spk_stream_ready, spk_stream_steps,
                  spk_synchronize)

__all__ = ["spk", "build", "Reconstructor", "SpkError", "SPK_F32", "SPK_F16", "SPK_U8", "SPK_ZERO_HEAD",
           "SPK_ZERO_TAIL", "spk_create",
           "spk_destroy", "spk_pitch", "spk_num_frames", "spk_reconstruct",
           "spk_reconstruct_host", "spk_reconstruct_host_async", "spk_segments", "spk_synchronize", "spk_last_error",
           "spk_launch_count", "spk_run", "spk_stream_open", "spk_stream_close",
           "spk_stream_ready", "spk_stream_steps", "Stream"]


class Reconstructor:
    """One libspk context bound to a torch CUDA stream.

    order (the method): 1 = FSR, 2 = SSR, 3 = TFI, 4 = TFP (window tfp_window steps),
    5 = the general n-order stability tree with stability_order levels (3..5);
    frame k samples step k * stride; dtype torch.float32, torch.float16 or torch.uint8 (8-bit
    frames: threshold * N / D rounded half up, integral thresholds); edges 0 or SPK_ZERO_HEAD |
    SPK_ZERO_TAIL (frames up to the first / after the last spike read 0).  Device memory
    comes from torch; the reconstruction runs in libspk.
    """

    def __init__(self, order: int = 2, stride: int = 1, dtype=None, device: int = 0,
                 stream=None, tfp_window: int = 32, stability_order: int = 3, edges: int = 0):
        import torch
        self.torch = torch
        dtype = dtype or torch.float32
        kinds = {torch.float32: SPK_F32, torch.float16: SPK_F16, torch.uint8: SPK_U8}
        if dtype not in kinds:
            raise ValueError("dtype must be torch.float32, torch.float16 or torch.uint8")
        self.dtype = dtype
        self.order, self.stride, self.device = order, stride, device
        self.stream = stream or torch.cuda.current_stream(device)
        self.ctx = spk_create(order, stride, kinds[dtype], device, self.stream.cuda_stream, tfp_window,
                              stability_order, edges)

    def close(self):
        if self.ctx is not None:
            spk_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alloc_frames(self, H: int, W: int, T: int):
        return self.torch.empty((spk_num_frames(T, self.stride), H, W), dtype=self.dtype,
                                device=f"cuda:{self.device}")

    def __call__(self, stream, H: int, W: int, T: int, threshold: float = 1.0, out=None):
        """Reconstruct frames [T_out][H][W] from a device uint8 stream [T][pitch]."""
        if out is None:
            out = self.alloc_frames(H, W, T)
        spk_reconstruct(self.ctx, stream, H, W, T, threshold, out)
        return out

    def segments(self, stream, H: int, W: int, T: int, threshold: float = 1.0, cap=None,
                 spikes: bool = False):
        """Stable sequences per pixel: (counts [P], t_start, t_end, n, value [cap][P]);
        with spikes=True the spike counts K [P] come first."""
        torch = self.torch
        P = H * W
        dev = f"cuda:{self.device}"
        counts = torch.empty(P, dtype=torch.int32, device=dev)
        K = torch.empty(P, dtype=torch.int32, device=dev) if spikes else None
        if cap is None:
            spk_segments(self.ctx, stream, H, W, T, threshold, None, counts, None, None, None, None, 0)
            self.synchronize()
            cap = int(counts.max().item()) if P else 0
        arrs = [torch.empty((max(cap, 1), P), dtype=d, device=dev)
                for d in (torch.int32, torch.int32, torch.int32, torch.float32)]
        spk_segments(self.ctx, stream, H, W, T, threshold, K, counts, *arrs, cap)
        return (K, counts, *arrs) if spikes else (counts, *arrs)

    def synchronize(self):
        spk_synchronize(self.ctx)


class Stream:
    """A live stream on a Reconstructor: per-pixel state stays on the device between pieces.

    push(piece, n) reconstructs the next n steps (device uint8 [n][pitch]); frames go to
    self.frames ([T_out][H][W]) at their absolute index; ready() is the number of leading
    frames final for every pixel.
    """

    def __init__(self, rec: "Reconstructor", H: int, W: int, T: int, threshold: float = 1.0):
        self.rec, self.H, self.W, self.T, self.threshold = rec, H, W, T, threshold
        self.state = spk_stream_open(rec.ctx, H, W, T)
        self.frames = rec.alloc_frames(H, W, T)

    def job(self, piece, n: int):
        return (piece, self.H, self.W, n, self.threshold, self.frames, self.state)

    def push(self, piece, n: int):
        spk_run(self.rec.ctx, [self.job(piece, n)])

    @property
    def steps(self) -> int:
        return spk_stream_steps(self.state)

    def ready(self) -> int:
        return spk_stream_ready(self.rec.ctx, self.state)

    def close(self):
        if self.state is not None:
            spk_stream_close(self.rec.ctx, self.state)
            self.state = None
