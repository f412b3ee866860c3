"""8-bit frames and the frame edge policy of the CUDA path against the fp64 CPU oracle.

8-bit frames (SPK_U8) are threshold * N / D rounded half up and clamped to 255, an integer
decision, so the bar is bit-exact equality with the oracle's integer arithmetic for every
method (FSR, SSR, the n-order tree, TFI, TFP).  The edge policy (frames up to the first /
after the last spike read 0) changes which span covers a frame, so boundaries are exact
and fp32 values stay within 1e-6 relative of the oracle.
"""
import numpy as np
import pytest

import oracle
import spkgen

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6
HEAD, TAIL = oracle.ZERO_HEAD, oracle.ZERO_TAIL


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_11639_gb300 as pkg
    pkg.build()
    return torch, pkg


def _oracle(st, H, W, T, method, stride, theta, edges=0, u8=False, n=3, window=32):
    if method in (1, 2):
        return oracle.reconstruct(st, H, W, T, theta, method, stride, edges=edges, u8=u8).frames
    if method == 5:
        return oracle.reconstruct(st, H, W, T, theta, n, stride, edges=edges, u8=u8).frames
    if method == 3:
        return oracle.tfi(st, H, W, T, theta, stride, edges=edges, u8=u8)
    return oracle.tfp(st, H, W, T, window, theta, stride, u8=u8)


def _gpu(env, st, H, W, T, method, stride, theta, dtype, edges=0, n=3, window=32):
    torch, pkg = env
    R = pkg.Reconstructor(order=method, stride=stride, dtype=dtype, tfp_window=window,
                          stability_order=n, edges=edges)
    f = R(torch.from_numpy(np.ascontiguousarray(st)).cuda(), H, W, T, theta)
    R.synchronize()
    out = f.cpu().numpy().reshape(f.shape[0], -1)
    R.close()
    return out


def _edge_bits(T, P, density, seed):
    """Random columns with long empty heads and tails, plus pixels with K = 0, 1, 2 spikes."""
    b = spkgen.random_bits(T, P, density, seed).copy()
    rng = np.random.default_rng(seed)
    for p in range(P):
        a = int(rng.integers(0, T // 3 + 1))
        z = int(rng.integers(0, T // 3 + 1))
        b[:a, p] = 0
        b[T - z:, p] = 0
    b[:, 0:3] = 0                 # K = 0
    b[:, 3:6] = 0                 # K = 1
    b[T // 2, 3:6] = 1
    b[:, 6:9] = 0                 # K = 2
    b[[1, T - 2], 6:9] = 1
    return b


def _check_f32(got, ref):
    assert got.shape == ref.shape
    err = np.abs(got.astype(np.float64) - ref)
    assert np.all(err <= REL_TOL * np.abs(ref)), err.max()


@pytest.mark.parametrize("method", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("H,W,T,stride,density,theta", [
    (17, 31, 1000, 1, 0.5, 255.0),   # ragged block of 256 pixels
    (4, 64, 130, 7, 0.3, 255.0),     # several tiles, ragged
    (9, 100, 777, 3, 0.9, 1000.0),   # dense, values clamp at 255
    (3, 11, 63, 2, 0.5, 7.0),        # T below one tile, small integral scale
    (2, 200, 300, 1, 0.0, 255.0),    # no spikes
])
def test_u8_frames_exact(env, method, H, W, T, stride, density, theta):
    b = spkgen.random_bits(T, H * W, density, seed=H * 1000 + W + T)
    st = spkgen.pack(b, H, W)
    got = _gpu(env, st, H, W, T, method, stride, theta, env[0].uint8)
    ref = _oracle(st, H, W, T, method, stride, theta, u8=True)
    assert got.dtype == np.uint8
    assert np.array_equal(got.astype(np.int64), ref.astype(np.int64))


@pytest.mark.parametrize("method", [1, 2, 3, 5])
def test_u8_ties_round_half_up(env, method):
    """Constant intervals of 2 and 6 steps at theta = 255 give 127.5 and 42.5: both round up."""
    T, P = 600, 64
    bits = np.zeros((T, P), dtype=np.uint8)
    t = np.arange(T)
    for p in range(P):
        d = 2 if p % 2 == 0 else 6
        bits[(t + p) % d == 0, p] = 1
    st = spkgen.pack(bits, 1, P)
    got = _gpu(env, st, 1, P, T, method, 1, 255.0, env[0].uint8)
    ref = _oracle(st, 1, P, T, method, 1, 255.0, u8=True)
    assert np.array_equal(got.astype(np.int64), ref.astype(np.int64))
    assert set(np.unique(got[:, 0::2])) <= {0, 128} and set(np.unique(got[:, 1::2])) <= {0, 43}
    assert oracle.u8(255, 1, 2) == 128 and oracle.u8(255, 1, 6) == 43


@pytest.mark.parametrize("method", [1, 2, 3, 5])
@pytest.mark.parametrize("edges", [HEAD, TAIL, HEAD | TAIL])
@pytest.mark.parametrize("stride", [1, 7])
def test_edge_policies(env, method, edges, stride):
    H, W, T = 5, 61, 1500
    st = spkgen.pack(_edge_bits(T, H * W, 0.2, seed=31 + method), H, W)
    got = _gpu(env, st, H, W, T, method, stride, 1.0, env[0].float32, edges=edges)
    ref = _oracle(st, H, W, T, method, stride, 1.0, edges=edges)
    _check_f32(got, ref)
    plain = _oracle(st, H, W, T, method, stride, 1.0)
    assert (ref == 0).sum() > (plain == 0).sum()   # the policy zeroed some frames


@pytest.mark.parametrize("method", [1, 2, 3, 5])
def test_u8_with_edges(env, method):
    H, W, T = 7, 45, 2000
    st = spkgen.pack(_edge_bits(T, H * W, 0.3, seed=7 * method), H, W)
    got = _gpu(env, st, H, W, T, method, 3, 255.0, env[0].uint8, edges=HEAD | TAIL)
    ref = _oracle(st, H, W, T, method, 3, 255.0, edges=HEAD | TAIL, u8=True)
    assert np.array_equal(got.astype(np.int64), ref.astype(np.int64))


def test_tfp_ignores_edges(env):
    H, W, T = 3, 50, 400
    st = spkgen.pack(_edge_bits(T, H * W, 0.4, seed=4), H, W)
    a = _gpu(env, st, H, W, T, 4, 2, 1.0, env[0].float32, edges=HEAD | TAIL)
    b = _gpu(env, st, H, W, T, 4, 2, 1.0, env[0].float32)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_dynamic_250x400x20000_u8_edges_full(env):
    """The benchmark's stream, every pixel and every frame: SSR, 8-bit frames every 10 steps
    at theta = 255 with both edges zeroed."""
    w = spkgen.WORKLOADS["dynamic_250x400x20000"]
    st, _ = spkgen.make_stream(w)
    got = _gpu(env, st, w.H, w.W, w.T, 2, w.stride, 255.0, env[0].uint8, edges=HEAD | TAIL)
    ref = _oracle(st, w.H, w.W, w.T, 2, w.stride, 255.0, edges=HEAD | TAIL, u8=True)
    assert np.array_equal(got.astype(np.int64), ref.astype(np.int64))


@pytest.mark.parametrize("method,dtype_name,edges", [(2, "u8", HEAD | TAIL), (1, "f32", HEAD),
                                                     (3, "u8", TAIL), (2, "f32", HEAD | TAIL)])
def test_live_stream_pieces(env, method, dtype_name, edges):
    """A stream pushed in pieces of uneven length equals the whole-stream call bit for bit
    and the oracle; the first spike of many pixels falls in a later piece."""
    torch, pkg = env
    dtype = torch.uint8 if dtype_name == "u8" else torch.float32
    theta = 255.0 if dtype_name == "u8" else 1.0
    H, W, T, stride = 6, 50, 2500, 4
    st = spkgen.pack(_edge_bits(T, H * W, 0.25, seed=100 + method), H, W)
    whole = _gpu(env, st, H, W, T, method, stride, theta, dtype, edges=edges)
    R = pkg.Reconstructor(order=method, stride=stride, dtype=dtype, edges=edges)
    S = pkg.Stream(R, H, W, T, theta)
    rng = np.random.default_rng(method)
    t = 0
    while t < T:
        n = int(min(T - t, rng.choice([1, 31, 33, 64, 200, 701])))
        S.push(torch.from_numpy(np.ascontiguousarray(st[t:t + n])).cuda(), n)
        t += n
    R.synchronize()
    assert S.ready() == whole.shape[0]
    got = S.frames.cpu().numpy().reshape(whole.shape[0], -1)
    S.close()
    R.close()
    assert np.array_equal(got, whole)
    ref = _oracle(st, H, W, T, method, stride, theta, edges=edges, u8=dtype_name == "u8")
    if dtype_name == "u8":
        assert np.array_equal(got.astype(np.int64), ref.astype(np.int64))
    else:
        _check_f32(got, ref)


def test_batch_of_streams_u8(env):
    torch, pkg = env
    R = pkg.Reconstructor(order=2, stride=3, dtype=torch.uint8, edges=HEAD)
    rng = np.random.default_rng(12)
    jobs, keep = [], []
    for k in range(9):
        H, W, T = int(rng.integers(1, 30)), int(rng.integers(1, 80)), int(rng.integers(1, 1500))
        st = spkgen.pack(_edge_bits(T, H * W, 0.3, seed=k) if H * W >= 9 else
                         spkgen.random_bits(T, H * W, 0.5, seed=k), H, W)
        d = torch.from_numpy(st).cuda()
        o = R.alloc_frames(H, W, T)
        jobs.append((d, H, W, T, 255.0, o, None))
        keep.append((st, H, W, T, o))
    pkg.spk_run(R.ctx, jobs)
    R.synchronize()
    for st, H, W, T, o in keep:
        ref = _oracle(st, H, W, T, 2, 3, 255.0, edges=HEAD, u8=True)
        assert np.array_equal(o.cpu().numpy().reshape(ref.shape).astype(np.int64), ref.astype(np.int64))
    R.close()


def test_u8_needs_integral_threshold(env):
    torch, pkg = env
    R = pkg.Reconstructor(order=2, dtype=torch.uint8)
    st = torch.zeros((10, 16), dtype=torch.uint8, device="cuda")
    for bad in (1.5, 0.5, 70000.0):
        with pytest.raises(pkg.SpkError):
            R(st, 1, 8, 10, bad)
    R.close()


def test_host_calls_u8_edges(env):
    """The host-buffer call (pinned frames written in place) and the no-allocation call give
    the device call's 8-bit frames."""
    torch, pkg = env
    spk = pkg.spk
    H, W, T = 8, 40, 900
    st = spkgen.pack(_edge_bits(T, H * W, 0.3, seed=77), H, W)
    ref = _oracle(st, H, W, T, 2, 5, 255.0, edges=HEAD | TAIL, u8=True).astype(np.int64)
    R = pkg.Reconstructor(order=2, stride=5, dtype=torch.uint8, edges=HEAD | TAIL)
    T_out = spk.spk_num_frames(T, 5)
    pinned = torch.empty((T_out, H, W), dtype=torch.uint8).pin_memory()
    spk.spk_reconstruct_host(R.ctx, torch.from_numpy(st), H, W, T, 255.0, pinned)
    assert np.array_equal(pinned.numpy().reshape(T_out, -1).astype(np.int64), ref)
    R.close()
    host = np.zeros((T_out, H, W), dtype=np.uint8)
    spk.spk_reconstruct_host_noalloc(st, H, W, T, 255.0, host, method=2, frame_stride=5,
                                     out_dtype=spk.SPK_U8, edges=HEAD | TAIL)
    assert np.array_equal(host.reshape(T_out, -1).astype(np.int64), ref)
