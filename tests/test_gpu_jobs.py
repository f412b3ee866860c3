"""Batched jobs (many uneven streams in one launch) and live streams (pieces with the
per-pixel state carried on the device) through the C ABI.

Bars: every job's frames equal the single-stream spk_reconstruct result bit for bit and the
fp64 oracle within 1e-6 relative; a stream pushed in pieces of any length equals the
whole stream bit for bit; ready() never decreases and reaches T_out.
"""
import numpy as np
import pytest

import oracle
import spkgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_11639_gb300 as pkg
    pkg.build()
    return torch, pkg


def _stream(kind, H, W, T, seed):
    if kind == "random":
        return spkgen.pack(spkgen.random_bits(T, H * W, 0.1 + 0.8 * ((seed * 37) % 10) / 10, seed), H, W)
    w = spkgen.WORKLOADS[kind].resized(H=H, W=W, T=T)
    return spkgen.make_stream(w)[0]


def _whole(env, st, H, W, T, order, stride, dtype):
    torch, pkg = env
    R = pkg.Reconstructor(order=order, stride=stride, dtype=dtype)
    f = R(torch.from_numpy(st).cuda(), H, W, T, 1.0)
    R.synchronize()
    out = f.cpu().numpy()
    R.close()
    return out


@pytest.mark.parametrize("order", [2, 1])
def test_batch_of_uneven_streams(env, order):
    torch, pkg = env
    rng = np.random.default_rng(order)
    specs = []
    kinds = ["random", "dynamic_250x400x20000", "large_1000x1000x20000", "static_250x400x2000"]
    for k in range(14):
        H, W = int(rng.integers(1, 40)), int(rng.integers(1, 90))
        T = int(rng.integers(1, 2500))
        specs.append((kinds[k % 4], H, W, T, k))
    R = pkg.Reconstructor(order=order, stride=3)
    streams, outs, jobs = [], [], []
    for kind, H, W, T, seed in specs:
        st = _stream(kind, H, W, T, seed)
        d = torch.from_numpy(st).cuda()
        o = R.alloc_frames(H, W, T)
        streams.append((st, d))
        outs.append(o)
        jobs.append((d, H, W, T, 1.0, o, None))
    n0 = pkg.spk_launch_count(R.ctx)
    pkg.spk_run(R.ctx, jobs)
    R.synchronize()
    assert pkg.spk_launch_count(R.ctx) - n0 == 1          # one launch for all of them
    for (kind, H, W, T, seed), (st, _), o in zip(specs, streams, outs):
        got = o.cpu().numpy()
        ref = _whole(env, st, H, W, T, order, 3, torch.float32)
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), (kind, H, W, T)
        r = oracle.reconstruct(st, H, W, T, 1.0, order, 3)
        f = got.reshape(got.shape[0], -1).astype(np.float64)
        assert np.all(np.abs(f - r.frames) <= 1e-6 * np.abs(r.frames))
    R.close()


@pytest.mark.parametrize("order,dtype_name,stride", [(2, "f32", 1), (1, "f32", 4), (2, "f16", 7)])
def test_stream_pieces_equal_whole(env, order, dtype_name, stride):
    torch, pkg = env
    dtype = torch.float32 if dtype_name == "f32" else torch.float16
    H, W, T = 24, 70, 3000
    for kind, seed in (("dynamic_250x400x20000", 1), ("random", 2), ("large_1000x1000x20000", 3)):
        st = _stream(kind, H, W, T, seed)
        ref = _whole(env, st, H, W, T, order, stride, dtype)
        R = pkg.Reconstructor(order=order, stride=stride, dtype=dtype)
        S = pkg.Stream(R, H, W, T)
        rng = np.random.default_rng(seed)
        t, last_ready = 0, 0
        while t < T:
            n = int(min(T - t, rng.choice([1, 5, 31, 32, 33, 64, 65, 200, 700])))
            piece = torch.from_numpy(np.ascontiguousarray(st[t:t + n])).cuda()
            S.push(piece, n)
            t += n
            assert S.steps == t
            ready = S.ready()
            assert ready >= last_ready
            last_ready = ready
        assert last_ready == ref.shape[0]
        got = S.frames.cpu().numpy()
        bits = np.uint16 if dtype_name == "f16" else np.uint32
        assert np.array_equal(got.view(bits), ref.view(bits)), kind
        S.close()
        R.close()


def test_live_streams_batched_together(env):
    """Continuous batching: pieces of several live streams share each launch; every stream
    still equals its own whole-stream result."""
    torch, pkg = env
    R = pkg.Reconstructor(order=2, stride=2)
    specs = [(16, 64, 2000, "dynamic_250x400x20000", 5), (9, 33, 1500, "random", 6),
             (30, 30, 2500, "large_1000x1000x20000", 7)]
    live = []
    for H, W, T, kind, seed in specs:
        st = _stream(kind, H, W, T, seed)
        live.append([st, pkg.Stream(R, H, W, T), 0, _whole(env, st, H, W, T, 2, 2, torch.float32)])
    rng = np.random.default_rng(0)
    while any(t < S.T for _, S, t, _ in live):
        jobs, keep = [], []
        for item in live:
            st, S, t, _ = item
            if t >= S.T:
                continue
            n = int(min(S.T - t, rng.integers(1, 400)))
            piece = torch.from_numpy(np.ascontiguousarray(st[t:t + n])).cuda()
            keep.append(piece)
            jobs.append(S.job(piece, n))
            item[2] = t + n
        pkg.spk_run(R.ctx, jobs)
    R.synchronize()
    for st, S, t, ref in live:
        assert S.ready() == ref.shape[0]
        assert np.array_equal(S.frames.cpu().numpy().view(np.uint32), ref.view(np.uint32))
        S.close()
    R.close()


def test_job_argument_errors(env):
    torch, pkg = env
    from paper_2412_11639_gb300 import spk
    R = pkg.Reconstructor(order=2, stride=1)
    S = pkg.Stream(R, 4, 8, 100)
    piece = torch.zeros((120, spk.spk_pitch(4, 8)), dtype=torch.uint8, device="cuda")
    with pytest.raises(spk.SpkError) as e:
        S.push(piece, 120)                                   # past T
    assert e.value.code == spk.SPK_ERR_ARG
    with pytest.raises(spk.SpkError) as e:
        pkg.spk_run(R.ctx, [S.job(piece, 10), S.job(piece, 10)])   # same stream twice
    assert e.value.code == spk.SPK_ERR_ARG
    assert S.steps == 0                                      # nothing was launched
    S.push(piece, 100)
    assert S.ready() == 100
    S.close()
    R.close()


def test_batch_captured_in_cuda_graph_and_autotuned(env):
    """A batch of whole streams captured once in a CUDA graph and replayed gives the same
    frames; the autotuner picks one of the tiles and every tile gives identical frames."""
    torch, pkg = env
    from paper_2412_11639_gb300 import spk
    rng = np.random.default_rng(9)
    side = torch.cuda.Stream()
    R = pkg.Reconstructor(order=2, stride=5, stream=side)
    jobs, outs, refs = [], [], []
    for k in range(10):
        H, W, T = int(rng.integers(4, 40)), int(rng.integers(8, 80)), int(rng.integers(100, 3000))
        st = _stream("dynamic_250x400x20000" if k % 2 else "random", H, W, T, k)
        d = torch.from_numpy(st).cuda()
        o = R.alloc_frames(H, W, T)
        jobs.append((d, H, W, T, 1.0, o, None))
        outs.append(o)
        refs.append(_whole(env, st, H, W, T, 2, 5, torch.float32))
    best = spk.spk_autotune(R.ctx, jobs)
    assert best in (32, 64, 128) and spk.spk_get_tile(R.ctx) == best
    for tile in (32, 64, 128):
        spk.spk_set_tile(R.ctx, tile)
        with torch.cuda.stream(side):
            pkg.spk_run(R.ctx, jobs)                 # also sets the kernel attributes
        torch.cuda.synchronize()
        for o, ref in zip(outs, refs):
            assert np.array_equal(o.cpu().numpy().view(np.uint32), ref.view(np.uint32)), tile
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            pkg.spk_run(R.ctx, jobs)
        for o in outs:                             # capture does not run the kernel
            o.fill_(-1.0)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        for o, ref in zip(outs, refs):
            assert np.array_equal(o.cpu().numpy().view(np.uint32), ref.view(np.uint32)), tile
    R.close()


def test_host_async_lanes_equal_sync(env):
    """Asynchronous host calls alternate between two lanes; each result equals the
    synchronous call on the same input."""
    torch, pkg = env
    from paper_2412_11639_gb300 import spk
    ws = [spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=33, W=70, T=2500, seed=s) for s in (5, 6, 7)]
    sts = [torch.from_numpy(spkgen.make_stream(w)[0]).pin_memory() for w in ws]
    R = pkg.Reconstructor(order=2, stride=10)
    outs = [torch.empty((ws[0].T_out, 33, 70), dtype=torch.float32).pin_memory() for _ in ws]
    for st, o in zip(sts, outs):
        spk.spk_reconstruct_host_async(R.ctx, st, 33, 70, 2500, 1.0, o)
    spk.spk_synchronize(R.ctx)
    for st, o in zip(sts, outs):
        ref = torch.empty_like(o)
        spk.spk_reconstruct_host(R.ctx, st, 33, 70, 2500, 1.0, ref)
        assert torch.equal(o, ref)
    R.close()


def test_host_calls_pinned_and_pageable_equal_device(env):
    """The synchronous host-buffer call writes the frames into page-locked output buffers
    directly from the kernel and copies them into pageable ones, the asynchronous one always
    copies; every way the frames equal the device-buffer reconstruction bit for bit (fp32
    and fp16)."""
    torch, pkg = env
    from paper_2412_11639_gb300 import spk
    w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=41, W=77, T=3100, seed=8)
    st = spkgen.make_stream(w)[0]
    for dtype, npdt in ((torch.float32, np.float32), (torch.float16, np.float16)):
        R = pkg.Reconstructor(order=2, stride=w.stride, dtype=dtype)
        want = R(torch.from_numpy(st).cuda(), w.H, w.W, w.T, 1.0)
        R.synchronize()
        want = want.cpu().numpy()
        pinned_in = torch.from_numpy(st).pin_memory()
        for pinned in (True, False):
            for call in (spk.spk_reconstruct_host, spk.spk_reconstruct_host_async):
                if pinned:
                    out = torch.full((w.T_out, w.H, w.W), -1.0, dtype=dtype).pin_memory()
                else:
                    out = np.full((w.T_out, w.H, w.W), -1.0, dtype=npdt)
                call(R.ctx, pinned_in if pinned else st, w.H, w.W, w.T, 1.0, out)
                spk.spk_synchronize(R.ctx)
                got = out.numpy() if pinned else out
                assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (dtype, pinned, call.__name__)
        R.close()
