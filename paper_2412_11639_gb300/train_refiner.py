"""Train the learned refiner on simulated streams and save its parameters.

    python -m paper_2412_11639_gb300.train_refiner [--clips 10000] [--out weights/refiner_dynamic.npy]

Clips follow the moving-scene recipe (250 x 400 pixels, 2000 steps, a frame every 10
steps, step events, dark noise) with seeds 1000, 1001, ...; the stream and its ground
truth come from the GPU generator, the plain SSR frames and the features from libspk, and
the network trains with libspk's kernels.  Seed 2 (the benchmark stream) is never used.
"""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--clips", type=int, default=10000)
    ap.add_argument("--steps-per-clip", type=int, default=2)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=5e-5)
    ap.add_argument("--T", type=int, default=2000)
    ap.add_argument("--seed", type=int, default=0, help="initial weights")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    import torch

    import spkgen
    from . import Reconstructor
    from .refiner import CHECKPOINT, Refiner, train_on_simulator
    base = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(T=a.T)
    rec = Reconstructor(order=2, stride=base.stride)
    ref = Refiner(seed=a.seed)
    t0 = time.perf_counter()
    losses = train_on_simulator(ref, rec, base, a.clips, a.steps_per_clip, a.batch, a.lr, a.lr_final,
                                log=lambda m: print(m, flush=True))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out = a.out or CHECKPOINT
    ref.save(out)
    print(json.dumps({"clips": a.clips, "recipe": f"{base.H}x{base.W}x{base.T} stride {base.stride}",
                      "steps": a.clips * a.steps_per_clip, "batch_frames": a.batch, "seconds": dt,
                      "first_loss": losses[0], "last_loss": losses[-1], "saved": out}), flush=True)
    ref.close()
    rec.close()


if __name__ == "__main__":
    main()
