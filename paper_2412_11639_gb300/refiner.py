"""The learned refiner: Python handle over spk_refiner_* (the network runs in libspk).

    x0 = features(rec, stream, H, W, T, plain)        # bf16 [T_out][H][2][W][8]
    ref = Refiner(seed=0)
    loss = ref.train_step(x0, plain, gt, lr=1e-3)     # one Adam step
    out = ref(x0, plain)                               # refined frames [T_out][H][W]

Device memory comes from torch; the features, the convolutions, the loss and the optimiser
are kernels of libspk.
"""
from __future__ import annotations

import numpy as np

from . import spk

FEAT_C = 16


def features(rec, stream, H: int, W: int, T: int, plain, threshold: float = 1.0):
    """Refiner input of every frame of `stream` (uses rec's frame stride): bf16, 16 channels
    as two channel-chunk planes, [T_out][H][2][W][8]."""
    torch = rec.torch
    T_out = plain.shape[0]
    x0 = torch.empty((T_out, H, FEAT_C // 8, W, 8), dtype=torch.bfloat16, device=plain.device)
    spk.spk_features(rec.ctx, stream, H, W, T, threshold, plain, x0)
    return x0


class Refiner:
    def __init__(self, device: int = 0, seed: int = 0, stream=None):
        import torch
        self.torch = torch
        self.device = device
        self.r = spk.spk_refiner_create(device, seed)
        self.stream = stream or torch.cuda.current_stream(device)
        self.n = spk.spk_refiner_num_params()

    def close(self):
        if self.r is not None:
            spk.spk_refiner_destroy(self.r)
            self.r = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float32)
        spk.spk_refiner_get_params(self.r, out, 0)
        return out

    def grads(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float32)
        spk.spk_refiner_get_params(self.r, out, 1)
        return out

    def set_params(self, p: np.ndarray):
        spk.spk_refiner_set_params(self.r, np.ascontiguousarray(p, dtype=np.float32))

    def save(self, path: str):
        np.save(path, self.params())

    def load(self, path: str):
        self.set_params(np.load(path))

    def __call__(self, x0, plain, out=None):
        N, H, W = plain.shape
        if out is None:
            out = self.torch.empty_like(plain)
        spk.spk_refiner_forward(self.r, self.stream.cuda_stream, x0, plain, N, H, W, out)
        return out

    def train_step(self, x0, plain, gt, lr: float, want_loss: bool = True) -> float:
        N, H, W = plain.shape
        return spk.spk_refiner_train_step(self.r, self.stream.cuda_stream, x0, plain, gt, N, H, W, lr,
                                          want_loss)


def fit(ref: Refiner, clips, steps: int, lr: float = 1e-3, batch: int = 8, seed: int = 0,
        lr_final: float | None = None):
    """Train on clips [(x0, plain, gt)] of device tensors ([N][H][2][W][8], [N][H][W], [N][H][W]).

    Each step takes `batch` consecutive frames of one clip (a contiguous view, no copy),
    clip and offset drawn from PCG64(seed); the learning rate decays linearly to lr_final
    (default lr / 10).  Returns the per-step losses.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lr_final = lr / 10 if lr_final is None else lr_final
    losses = []
    for s in range(steps):
        x0, plain, gt = clips[int(rng.integers(0, len(clips)))]
        n = min(batch, plain.shape[0])
        k = int(rng.integers(0, plain.shape[0] - n + 1))
        a = lr + (lr_final - lr) * s / max(1, steps - 1)
        losses.append(ref.train_step(x0[k:k + n], plain[k:k + n], gt[k:k + n], a,
                                     want_loss=(s % 10 == 0 or s == steps - 1)))
    return losses


CHECKPOINT = __import__("os").path.join(__import__("os").path.dirname(__file__), "weights",
                                        "refiner_dynamic.npy")


def simulator_clip(rec, w, device: int = 0):
    """(x0, plain, gt) of one simulated clip: the stream and its ground truth come from the
    GPU generator, the plain frames from rec, the features from spk_features."""
    import spkgen
    torch = rec.torch
    stream, gt = spkgen.make_stream_cuda(w, gt_stride=w.stride, device=device)
    plain = rec(stream, w.H, w.W, w.T)
    x0 = features(rec, stream, w.H, w.W, w.T, plain)
    del stream
    return x0, plain, gt.view(w.T_out, w.H, w.W)


def train_on_simulator(ref: Refiner, rec, base, n_clips: int, steps_per_clip: int = 4, batch: int = 16,
                       lr: float = 1e-3, lr_final: float = 5e-5, seed0: int = 1000, log=None):
    """Train on n_clips freshly simulated clips of recipe `base` (seeds seed0, seed0+1, ...),
    steps_per_clip Adam steps of `batch` consecutive frames each, learning rate decaying
    linearly from lr to lr_final.  Returns the mean loss of every clip's steps."""
    rng = np.random.Generator(np.random.PCG64(seed0))
    total = n_clips * steps_per_clip
    out = []
    s = 0
    for c in range(n_clips):
        x0, plain, gt = simulator_clip(rec, base.resized(seed=seed0 + c), ref.device)
        ls = []
        for _ in range(steps_per_clip):
            k = int(rng.integers(0, plain.shape[0] - batch + 1))
            a = lr + (lr_final - lr) * s / max(1, total - 1)
            ls.append(ref.train_step(x0[k:k + batch], plain[k:k + batch], gt[k:k + batch], a,
                                     want_loss=(c % 50 == 0)))
            s += 1
        if c % 50 == 0:
            out.append(float(np.mean(ls)))
            if log:
                log(f"clip {c}/{n_clips} loss {out[-1]:.4e}")
    return out
