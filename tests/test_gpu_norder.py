"""The general n-order stability tree (Sec. III-B, Fig. 1 caption) on the GPU against the
fp64 oracle: sequence boundaries and interval counts bit-exact, fp32 values within 1e-6
relative, fp16 frames the round-to-nearest-even of the fp32 value."""
import numpy as np
import pytest

import oracle
import spkgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-6


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2412_11639_gb300 as pkg
    pkg.build()
    return pkg


def _check(pkg, st, H, W, T, n, stride, f16=False):
    R = pkg.Reconstructor(order=5, stability_order=n, stride=stride,
                          dtype=torch.float16 if f16 else torch.float32)
    dev = torch.from_numpy(np.ascontiguousarray(st)).cuda()
    frames = R(dev, H, W, T).cpu().numpy().reshape(-1, H * W)
    K, counts, ts, te, nn, v = [a.cpu().numpy() for a in R.segments(dev, H, W, T, spikes=True)]
    R.synchronize()                      # raises on a device-side consistency failure
    R.close()
    r = oracle.reconstruct(st, H, W, T, 1.0, n, stride, segments=True)
    assert np.array_equal(K, r.K)
    assert np.array_equal(counts, r.nseg)
    for p in range(H * W):
        k = counts[p]
        ots, ote, onn, ov = r.segments(p)
        assert np.array_equal(ts[:k, p], ots) and np.array_equal(te[:k, p], ote), p
        assert np.array_equal(nn[:k, p], onn), p
        assert np.all(np.abs(v[:k, p] - ov) <= REL_TOL * np.abs(ov)), p
    if f16:
        assert np.array_equal(frames.view(np.uint16), r.frames.astype(np.float32).astype(np.float16).view(np.uint16))
    else:
        assert np.all(np.abs(frames - r.frames) <= REL_TOL * np.abs(r.frames))
    return r


def _deep_streams(P, T, seed):
    """One pixel per constructed stream: intervals 2 with 3s spaced by 1..4 intervals, so
    that S_2 and S_3 have several stable sequences; occasional FSR breaks."""
    rng = np.random.default_rng(seed)
    bits = np.zeros((T, P), dtype=np.uint8)
    for p in range(P):
        t = int(rng.integers(0, 4))
        while t < T:
            bits[t, p] = 1
            for _ in range(int(rng.integers(1, 5))):
                t += 2
                if t < T:
                    bits[t, p] = 1
            t += 3 if rng.uniform() > 0.05 else int(rng.integers(1, 7))
    return bits


@pytest.mark.parametrize("n", [3, 4, 5])
def test_norder_deep_streams(env, n):
    H, W, T = 3, 97, 1500
    bits = _deep_streams(H * W, T, 40 + n)
    r = _check(env, spkgen.pack(bits, H, W), H, W, T, n, 1)
    r2 = oracle.reconstruct(spkgen.pack(bits, H, W), H, W, T, 1.0, 2, 1, frames=False)
    assert (r.nseg > r2.nseg).sum() > H * W // 2      # the deeper levels do cut here


@pytest.mark.parametrize("n,H,W,T,stride,density,f16", [
    (3, 1, 7, 5, 1, 0.6, False),
    (3, 5, 53, 777, 3, 0.4, False),
    (4, 17, 31, 1000, 1, 0.5, True),
    (5, 4, 64, 2000, 7, 0.3, False),
    (3, 2, 200, 3001, 1, 1.0, False),      # a spike every step
    (4, 2, 200, 300, 1, 0.0, False),       # no spikes
])
def test_norder_random_streams(env, n, H, W, T, stride, density, f16):
    b = spkgen.random_bits(T, H * W, density, seed=n * 100 + W + T)
    _check(env, spkgen.pack(b, H, W), H, W, T, n, stride, f16)


@pytest.mark.parametrize("n", [3, 5])
def test_norder_scene_workload(env, n):
    w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=30, W=70, T=4000)
    st, _ = spkgen.make_stream(w)
    _check(env, st, w.H, w.W, w.T, n, w.stride)


def _push_pieces(pkg, R, S, st, T, rng, sizes=(1, 31, 32, 33, 64, 200, 701)):
    """Pushes the stream in pieces; returns (frames ready at the end, number of pieces)."""
    t, last_ready, pieces = 0, 0, 0
    while t < T:
        n = int(min(T - t, rng.choice(sizes)))
        pkg.spk_run(R.ctx, [S.job(torch.from_numpy(np.ascontiguousarray(st[t:t + n])).cuda(), n)])
        t += n
        pieces += 1
        assert S.steps == t
        ready = S.ready()
        assert ready >= last_ready
        last_ready = ready
    return last_ready, pieces


@pytest.mark.parametrize("n,ring0", [(3, 0), (4, 0), (5, 0), (3, 2), (5, 2)])
def test_norder_live_stream_pieces_equal_whole(env, n, ring0):
    """A live stream of the tree pushed in pieces of uneven length (node state and pending
    cuts carried on the device from piece to piece) equals the whole stream bit for bit and
    the oracle within 1e-6; started with rings of 2 cuts, pieces whose pixels need more run
    again, from a copy of the state taken before them, with rings twice as large."""
    from paper_2412_11639_gb300 import spk
    w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=12, W=70, T=3000)
    st, _ = spkgen.make_stream(w)
    bits = spkgen.pack(_deep_streams(3 * 40, 2500, seed=n), 3, 40)
    spk.spk_debug_norder_capacity(ring0)
    try:
        for stream, H, W, T in ((st, w.H, w.W, w.T), (bits, 3, 40, 2500)):
            R = env.Reconstructor(order=5, stability_order=n, stride=4)
            whole = R(torch.from_numpy(np.ascontiguousarray(stream)).cuda(), H, W, T).cpu().numpy()
            S = env.Stream(R, H, W, T)
            n0 = spk.spk_launch_count(R.ctx)
            rng = np.random.default_rng(n + 10 * ring0)
            ready, pieces = _push_pieces(env, R, S, stream, T, rng)
            launches = spk.spk_launch_count(R.ctx) - n0
            assert ready == whole.shape[0]
            assert launches > pieces if ring0 else launches == pieces   # reruns with larger rings
            got = S.frames.cpu().numpy()
            R.synchronize()
            assert np.array_equal(got.view(np.uint32), whole.view(np.uint32))
            r = oracle.reconstruct(stream, H, W, T, 1.0, n, 4)
            g = got.reshape(-1, H * W).astype(np.float64)
            assert np.all(np.abs(g - r.frames) <= REL_TOL * np.abs(r.frames))
            S.close()
            R.close()
    finally:
        spk.spk_debug_norder_capacity(0)


def test_norder_live_streams_and_whole_streams_in_one_launch(env):
    """Pieces of three live streams and two whole streams share each spk_run launch; every
    result equals its stream alone."""
    rng = np.random.default_rng(5)
    R = env.Reconstructor(order=5, stability_order=3, stride=3)
    live = []
    for k in range(3):
        H, W, T = int(rng.integers(2, 12)), int(rng.integers(5, 60)), int(rng.integers(500, 2500))
        w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=H, W=W, T=T, seed=70 + k)
        stream = spkgen.make_stream(w)[0]
        alone = R(torch.from_numpy(stream).cuda(), H, W, T).cpu().numpy()
        live.append([stream, env.Stream(R, H, W, T), 0, alone])
    whole = []
    while any(x[2] < x[1].T for x in live):
        jobs = []
        for x in live:
            stream, S, t, _ = x
            if t < S.T:
                n = int(min(S.T - t, rng.integers(1, 400)))
                jobs.append(S.job(torch.from_numpy(np.ascontiguousarray(stream[t:t + n])).cuda(), n))
                x[2] = t + n
        if len(whole) < 2:
            H, W, T = 5, 33, 700 + 300 * len(whole)
            stream = spkgen.pack(_deep_streams(H * W, T, seed=80 + len(whole)), H, W)
            d = torch.from_numpy(stream).cuda()
            o = R.alloc_frames(H, W, T)
            jobs.append((d, H, W, T, 1.0, o, None))
            whole.append((d, H, W, T, o))
        env.spk_run(R.ctx, jobs)
    R.synchronize()
    for stream, S, t, alone in live:
        assert np.array_equal(S.frames.cpu().numpy().view(np.uint32), alone.view(np.uint32))
        S.close()
    for d, H, W, T, o in whole:
        assert np.array_equal(o.cpu().numpy().view(np.uint32), R(d, H, W, T).cpu().numpy().view(np.uint32))
    R.close()


def test_live_stream_refusals(env):
    """TFP has no live streams; a stream opened for one method is refused by another."""
    from paper_2412_11639_gb300 import spk
    R = env.Reconstructor(order=4)
    with pytest.raises(spk.SpkError):
        env.Stream(R, 4, 8, 100)
    R.close()
    Rs = env.Reconstructor(order=2)
    S = env.Stream(Rs, 4, 8, 100)
    Rt = env.Reconstructor(order=5, stability_order=3)
    piece = torch.zeros((10, spkgen.pitch(4, 8)), dtype=torch.uint8, device="cuda")
    with pytest.raises(spk.SpkError):
        env.spk_run(Rt.ctx, [S.job(piece, 10)])
    S.close()
    Rs.close()
    Rt.close()


@pytest.mark.parametrize("n,ring0", [(3, 0), (4, 0), (5, 0), (3, 2), (5, 2)])
def test_norder_batch_of_uneven_streams(env, n, ring0):
    """spk_run: whole streams of uneven size in one launch (each job's pending-cut rings
    after the previous job's).  Every job equals its stream alone bit for bit and the
    oracle within 1e-6; started with rings of 2 cuts, the whole batch runs again with
    larger rings until every pixel fits."""
    from paper_2412_11639_gb300 import spk
    rng = np.random.default_rng(40 + n)
    spk.spk_debug_norder_capacity(ring0)
    try:
        R = env.Reconstructor(order=5, stability_order=n, stride=3)
        jobs, keep = [], []
        for k in range(8):
            H, W, T = int(rng.integers(1, 20)), int(rng.integers(1, 70)), int(rng.integers(1, 2500))
            if k == 0:                   # a scene whose deep cuts need rings of more than 4
                H, W, T = 12, 70, 3000
            if k % 2 == 0:
                w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=H, W=W, T=T)
                st = spkgen.make_stream(w)[0]
            else:
                st = spkgen.pack(_deep_streams(H * W, T, seed=k), H, W)
            d = torch.from_numpy(np.ascontiguousarray(st)).cuda()
            o = R.alloc_frames(H, W, T)
            jobs.append((d, H, W, T, 1.0, o, None))
            keep.append((st, d, H, W, T, o))
        n0 = spk.spk_launch_count(R.ctx)
        env.spk_run(R.ctx, jobs)
        R.synchronize()
        launches = spk.spk_launch_count(R.ctx) - n0
        assert launches == 1 if ring0 == 0 else launches >= 2
        for st, d, H, W, T, o in keep:
            got = o.cpu().numpy().reshape(-1, H * W)
            alone = R(d, H, W, T).cpu().numpy().reshape(-1, H * W)
            assert np.array_equal(got.view(np.uint32), alone.view(np.uint32)), (H, W, T)
            r = oracle.reconstruct(st, H, W, T, 1.0, n, 3)
            assert np.all(np.abs(got - r.frames) <= REL_TOL * np.abs(r.frames)), (H, W, T)
        R.close()
    finally:
        spk.spk_debug_norder_capacity(0)


@pytest.mark.parametrize("n", [3, 5])
def test_norder_rings_regrow(env, n):
    """Deep cuts wait in per-pixel rings; started with rings of 2 cuts, a call whose pixels
    need more runs again with rings twice as large until they fit, and the frames and
    sequences still equal the oracle's (the regrowth is visible as extra launches)."""
    from paper_2412_11639_gb300 import spk
    w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=12, W=70, T=3000)
    st, _ = spkgen.make_stream(w)
    spk.spk_debug_norder_capacity(2)
    try:
        R = env.Reconstructor(order=5, stability_order=n, stride=w.stride)
        dev = torch.from_numpy(np.ascontiguousarray(st)).cuda()
        n0 = spk.spk_launch_count(R.ctx)
        frames = R(dev, w.H, w.W, w.T).cpu().numpy().reshape(-1, w.P)
        R.synchronize()
        assert spk.spk_launch_count(R.ctx) - n0 >= 3       # 2 -> 4 -> 8 ... cuts per pixel
        R.close()
        r = _check(env, st, w.H, w.W, w.T, n, w.stride)
        assert np.all(np.abs(frames - r.frames) <= REL_TOL * np.abs(r.frames))
    finally:
        spk.spk_debug_norder_capacity(0)
