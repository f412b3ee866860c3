"""Parity of the CUDA path (through the C ABI) with the fp64 CPU oracle.

Bars: spike counts K, sequence boundaries and interval counts bit-exact; fp32 values within
1e-6 relative of the oracle; fp16 frames equal to the round-to-nearest-even of the fp32
value and within one fp16 ulp of the oracle.
"""
import numpy as np
import pytest

import oracle
import spkgen
from conftest import load_golden

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_11639_gb300 as pkg
    pkg.build()
    return torch


def _padded_oracle_segments(r, P, cap):
    """Oracle sequences in the library's [cap][P] layout (-1 where absent)."""
    out = [np.full((cap, P), -1, dtype=np.int64) for _ in range(3)]
    val = np.full((cap, P), np.nan)
    pix = np.repeat(np.arange(P), r.nseg)
    j = np.arange(r.seg_ts.shape[0]) - np.repeat(r.seg_off[:-1], r.nseg)
    keep = j < cap
    out[0][j[keep], pix[keep]] = r.seg_ts[keep]
    out[1][j[keep], pix[keep]] = r.seg_te[keep]
    out[2][j[keep], pix[keep]] = r.seg_n[keep]
    val[j[keep], pix[keep]] = r.seg_val[keep]
    return out, val


def _run_gpu(torch, st, H, W, T, order, stride, dtype, theta=1.0, segments=True):
    import paper_2412_11639_gb300 as pkg
    R = pkg.Reconstructor(order=order, stride=stride, dtype=dtype)
    dev = torch.from_numpy(np.ascontiguousarray(st)).cuda()
    frames = R(dev, H, W, T, theta)
    seg = R.segments(dev, H, W, T, theta, spikes=True) if segments else None
    R.synchronize()
    res = frames.cpu().numpy().reshape(frames.shape[0], -1), (
        None if seg is None else [s.cpu().numpy() for s in seg])
    R.close()
    return res


def _check_segments(seg, r, P):
    K, counts, ts, te, n, v = seg
    assert np.array_equal(K, r.K), "spike counts differ"
    assert np.array_equal(counts, r.nseg), "sequence counts differ"
    cap = ts.shape[0]
    assert cap >= r.nseg.max(initial=0)
    (ots, ote, on), oval = _padded_oracle_segments(r, P, cap)
    mask = ots >= 0
    assert np.array_equal(ts[mask], ots[mask])
    assert np.array_equal(te[mask], ote[mask])
    assert np.array_equal(n[mask], on[mask])
    rel = np.abs(v[mask].astype(np.float64) - oval[mask]) / np.abs(oval[mask])
    assert rel.max(initial=0) <= REL_TOL


def _check_frames(frames, ref, dtype_name):
    assert frames.shape == ref.shape
    if dtype_name == "f32":
        f = frames.astype(np.float64)
        err = np.abs(f - ref)
        assert np.all(err <= REL_TOL * np.abs(ref)), err.max()
    else:
        expect = ref.astype(np.float32).astype(np.float16)
        assert np.array_equal(frames.view(np.uint16), expect.view(np.uint16))
        ulp = np.spacing(np.abs(ref).astype(np.float16)).astype(np.float64)
        assert np.all(np.abs(frames.astype(np.float64) - ref) <= ulp)


def _case(torch, st, H, W, T, order, stride, dtype_name="f32", theta=1.0, segments=True):
    dtype = torch.float32 if dtype_name == "f32" else torch.float16
    frames, seg = _run_gpu(torch, st, H, W, T, order, stride, dtype, theta, segments)
    r = oracle.reconstruct(st, H, W, T, theta, order, stride, segments=segments)
    _check_frames(frames, r.frames, dtype_name)
    if segments:
        _check_segments(seg, r, H * W)
    return r


@pytest.mark.parametrize("case", load_golden(), ids=lambda c: c["name"])
def test_golden_cases(torch_cuda, case):
    T = case["T"]
    bits = np.zeros((T, 300), dtype=np.uint8)
    for t in case["spikes"]:
        bits[t, 257] = 1      # second block of 256 pixels, ragged tail
    st = spkgen.pack(bits)
    frames, seg = _run_gpu(torch_cuda, st, 1, 300, T, case["order"], case["stride"],
                           torch_cuda.float32)
    K, counts, ts, te, n, v = seg
    assert K[257] == len(case["spikes"]) and np.all(K[np.arange(300) != 257] == 0)
    k = counts[257]
    got = list(zip(ts[:k, 257].tolist(), te[:k, 257].tolist(), n[:k, 257].tolist()))
    assert got == case["segments"]
    if case["frames"] is not None:
        assert np.allclose(frames[:, 257], [float(f) for f in case["frames"]], rtol=REL_TOL, atol=0)
    assert np.all(counts[np.arange(300) != 257] == 0)
    assert np.all(frames[:, np.arange(300) != 257] == 0)


@pytest.mark.parametrize("order", [1, 2])
def test_exhaustive_20_steps(torch_cuda, order):
    """All 2^20 patterns of 20 steps, one pattern per pixel."""
    T = 20
    P = 1 << T
    bits = ((np.arange(P)[None, :] >> np.arange(T)[:, None]) & 1).astype(np.uint8)
    st = spkgen.pack(bits)
    _case(torch_cuda, st, 1024, 1024, T, order, 1)
    _case(torch_cuda, st, 1024, 1024, T, order, 3, "f16", segments=False)


@pytest.mark.parametrize("H,W,T,stride,order,dtype,density", [
    (1, 1, 1, 1, 1, "f32", 0.5),
    (1, 7, 5, 1, 2, "f32", 0.6),
    (3, 11, 63, 2, 2, "f32", 0.5),      # T < one tile, P not a multiple of 8
    (5, 53, 65, 1, 1, "f16", 0.4),      # T = one tile + 1
    (4, 64, 130, 7, 2, "f32", 0.3),     # several tiles, ragged
    (17, 31, 1000, 1, 2, "f16", 0.5),   # ragged block of 256 pixels
    (16, 16, 4096, 10, 2, "f32", 0.05), # sparse
    (9, 100, 777, 3, 1, "f32", 0.9),    # dense
    (2, 200, 3001, 1, 2, "f32", 1.0),   # a spike every step
    (2, 200, 300, 1, 2, "f32", 0.0),    # no spikes
])
def test_random_streams(torch_cuda, H, W, T, stride, order, dtype, density):
    b = spkgen.random_bits(T, H * W, density, seed=H * 1000 + W + T)
    _case(torch_cuda, spkgen.pack(b, H, W), H, W, T, order, stride, dtype)


def test_theta_255(torch_cuda):
    b = spkgen.random_bits(500, 300, 0.4, seed=5)
    _case(torch_cuda, spkgen.pack(b), 1, 300, 500, 2, 4, "f32", theta=255.0)


@pytest.mark.parametrize("order", [1, 2])
def test_small_scene_workloads(torch_cuda, order):
    for name in ("dynamic_250x400x20000", "large_1000x1000x20000"):
        w = spkgen.WORKLOADS[name].resized(H=40, W=70, T=3000)
        st, _ = spkgen.make_stream(w)
        _case(torch_cuda, st, w.H, w.W, w.T, order, w.stride, w.out_dtype)


@pytest.mark.parametrize("order", [1, 2])
def test_static_250x400x2000_full(torch_cuda, order):
    """Full size, every pixel: one sequence each (Theorem 1) and every frame."""
    w = spkgen.WORKLOADS["static_250x400x2000"]
    st, _ = spkgen.make_stream(w)
    r = _case(torch_cuda, st, w.H, w.W, w.T, order, w.stride, w.out_dtype)
    assert np.all(r.nseg == 1)


@pytest.mark.parametrize("order", [2, 1])
def test_dynamic_250x400x20000_full(torch_cuda, order):
    """Full size, every pixel, every sequence and every frame."""
    w = spkgen.WORKLOADS["dynamic_250x400x20000"]
    st, _ = spkgen.make_stream(w)
    _case(torch_cuda, st, w.H, w.W, w.T, order, w.stride, w.out_dtype)


def test_large_1000x1000x20000_sampled(torch_cuda):
    """Full size in the benchmark's launch configuration: sequence counts of every pixel,
    sequences and frames of 2048 sampled pixels (fp16 frames of every step)."""
    torch = torch_cuda
    import paper_2412_11639_gb300 as pkg
    w = spkgen.WORKLOADS["large_1000x1000x20000"]
    st, _ = spkgen.make_stream(w)
    rng = np.random.default_rng(3)
    pix = np.sort(rng.choice(w.P, 2048, replace=False))
    r_all = oracle.reconstruct(st, w.H, w.W, w.T, 1.0, 2, w.stride, frames=False)
    r = oracle.reconstruct(st, w.H, w.W, w.T, 1.0, 2, w.stride, pixels=pix, segments=True)
    R = pkg.Reconstructor(order=2, stride=w.stride, dtype=torch.float16)
    dev = torch.from_numpy(st).cuda()
    del st
    frames = R(dev, w.H, w.W, w.T, 1.0)
    R.synchronize()
    idx = torch.from_numpy(pix).cuda()
    f_s = frames.view(frames.shape[0], -1).index_select(1, idx).cpu().numpy()
    del frames
    torch.cuda.empty_cache()
    K, counts, ts, te, n, v = R.segments(dev, w.H, w.W, w.T, 1.0, spikes=True)
    R.synchronize()
    assert np.array_equal(K.cpu().numpy(), r_all.K)
    assert np.array_equal(counts.cpu().numpy(), r_all.nseg)
    seg = [K.cpu().numpy()[pix], counts.cpu().numpy()[pix]] + [a.index_select(1, idx).cpu().numpy()
                                                                for a in (ts, te, n, v)]
    R.close()
    _check_segments(seg, r, len(pix))
    _check_frames(f_s, r.frames, "f16")


@pytest.mark.parametrize("order,stride,dtype", [(1, 1, "f32"), (2, 1, "f16"), (2, 7, "f32"), (1, 3, "f16")])
def test_record_ring_overflow(torch_cuda, order, stride, dtype):
    """One lane per warp never cuts (a constant interval of 4) and holds back the warp's
    full rows, while the other lanes cut at every interval (1, 3, 1, 3, ...): their record
    rings fill within a few words and write their oldest records alone."""
    T, W = 3000, 80
    bits = np.zeros((T, W), dtype=np.uint8)
    t = np.arange(T)
    for p in range(W):
        if p % 32 == 5:
            bits[t % 4 == p % 4, p] = 1
        else:
            bits[(t % 4 == 0) | (t % 4 == 1), p] = 1     # intervals 1, 3, 1, 3, ...
            bits[: p % 11, p] = 0                         # stagger the lanes
    _case(torch_cuda, spkgen.pack(bits), 1, W, T, order, stride, dtype)


@pytest.mark.parametrize("order", [1, 2])
def test_spike_counts_few_spikes(torch_cuda, order):
    """K of pixels with no spike, one spike (first, middle or last step), two spikes, a spike
    every step and random densities equals the number of set bits of the pixel's column
    (Def. 2: S_1 has K - 1 elements), and the oracle's K; pixels with K < 2 have no
    sequence and read 0 in every frame."""
    T, P = 300, 300
    bits = (spkgen.random_bits(T, P, 0.3, seed=9)).copy()
    bits[:, 0:40] = 0                     # K = 0
    bits[0, 40:48] = 1                    # K = 1 at the first step
    bits[137, 48:56] = 1                  # K = 1 in the middle
    bits[T - 1, 56:64] = 1                # K = 1 at the last step
    bits[[5, 250], 64:72] = 1             # K = 2
    bits[:, 72:80] = 1                    # K = T
    st = spkgen.pack(bits, 1, P)
    frames, seg = _run_gpu(torch_cuda, st, 1, P, T, order, 1, torch_cuda.float32)
    K, counts = seg[0], seg[1]
    assert np.array_equal(K, bits.sum(axis=0))
    assert np.array_equal(K, oracle.reconstruct(st, 1, P, T, 1.0, order, 1).K)
    assert np.all(counts[K < 2] == 0) and np.all(counts[K >= 2] >= 1)
    assert np.all(frames[:, K < 2] == 0)
