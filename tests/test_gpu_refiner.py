"""Learned refiner on the GPU: features, forward, gradients and Adam against plain PyTorch
fp32 on the CPU (tests/refnet.py), bitwise repeatable training, and training on simulator
streams against the plain reconstruction (PSNR, SSIM)."""
import math

import numpy as np
import pytest

import paper_2412_11639_gb300 as pkg
import spkgen
from paper_2412_11639_gb300 import quality, refiner, spk

torch = pytest.importorskip("torch")
import refnet  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    pkg.build()
    spk.load()


def planar(x):
    """[N][H][W][16] -> the library's channel-chunk planes [N][H][2][W][8]."""
    N, H, W, C = x.shape
    return np.ascontiguousarray(x.reshape(N, H, W, C // 8, 8).transpose(0, 1, 3, 2, 4))


def _bf16_bits(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).view(torch.int16).numpy()


def _cpu_features(stream, H, W, T, stride, plain, theta):
    """Channel 0 plain, 4..7 theta / x of the last four intervals ending at or before t_k."""
    P = H * W
    bits = np.unpackbits(stream[:T], axis=1, bitorder="little")[:, :P]
    T_out = (T + stride - 1) // stride
    f = np.zeros((T_out, P, 16), dtype=np.float32)
    f[:, :, 0] = plain.reshape(T_out, P)
    th = np.float32(theta)
    for p in range(P):
        s = np.flatnonzero(bits[:, p])
        for k in range(T_out):
            j = int(np.searchsorted(s, k * stride, side="right"))   # spikes at or before t_k
            for m in range(4):
                if j - m - 2 >= 0:
                    f[k, p, 4 + m] = th / np.float32(s[j - m - 1] - s[j - m - 2])
    return f.reshape(T_out, H, W, 16)


@pytest.mark.parametrize("H,W,T,stride,theta", [(23, 37, 700, 10, 1.0), (9, 130, 300, 1, 2.5)])
def test_features_exact(H, W, T, stride, theta):
    w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=H, W=W, T=T, stride=stride)
    stream, _ = spkgen.make_stream(w)
    rec = pkg.Reconstructor(order=2, stride=stride)
    dev = torch.from_numpy(stream).cuda()
    plain = rec(dev, H, W, T, theta)
    x0 = refiner.features(rec, dev, H, W, T, plain, theta)
    torch.cuda.synchronize()
    want = _cpu_features(stream, H, W, T, stride, plain.cpu().numpy(), theta)
    got = x0.view(torch.int16).cpu().numpy()
    assert np.array_equal(got, _bf16_bits(planar(want)))


# The hidden activations are stored in bf16 (a step of 2^-8 relative): where the kernels'
# fp32 accumulation order and PyTorch's round a value to different sides of a bf16 boundary,
# that activation differs by one bf16 step.  The forward is therefore held to one such step
# at the scale of the correction (observed: 2.5e-3); the gradients, whose reference rounds
# where the kernels do, to 1e-3 relative L2 (observed: 5e-5).
FWD_TOL = 2.0 ** -8
GRAD_TOL = 1e-3


def _rand_case(N, H, W, seed):
    rng = np.random.default_rng(seed)
    x0 = np.zeros((N, H, W, 16), dtype=np.float32)
    x0[..., 0] = rng.uniform(0.02, 1.0, (N, H, W))
    x0[..., 4:8] = rng.uniform(0.0, 1.0, (N, H, W, 4))
    x0 = torch.as_tensor(x0).to(torch.bfloat16).float().numpy()   # bf16 values
    plain = x0[..., 0].copy()
    gt = np.clip(plain + 0.05 * rng.standard_normal((N, H, W)), 0.02, 1.0).astype(np.float32)
    return x0, plain, gt


def _dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a)).cuda()
    return t.to(dtype) if dtype is not None else t


@pytest.mark.parametrize("N,H,W", [(2, 20, 150), (1, 3, 5), (3, 17, 128)])
def test_forward_matches_reference(N, H, W):
    ref = refiner.Refiner(seed=11)
    p = ref.params()
    # larger last layer than the init's 0.1 scale so that the correction is not tiny
    p[refnet.NPARAM - (9 * 32 * 16 + 16):] *= 10
    p[-16:] = 0.01
    ref.set_params(p)
    x0, plain, gt = _rand_case(N, H, W, seed=N * 1000 + W)
    out = ref(_dev(planar(x0), torch.bfloat16), _dev(plain))
    torch.cuda.synchronize()
    want, _, _ = refnet.forward(p, x0, plain)
    got = out.cpu().numpy()
    corr = np.abs(want - plain).max()
    assert corr > 1e-3
    err = np.abs(got - want).max()
    print(f"forward N={N} H={H} W={W}: max error {err:.3e} of correction range {corr:.3e} ({err / corr:.2e})")
    assert err <= FWD_TOL * corr + 1e-6, (err, corr)
    ref.close()


def test_tall_and_short_tasks_agree_bit_for_bit():
    """A forward over many frames walks tasks of 125 rows (fewer halo reloads), one over a
    few frames tasks of 32 rows; every output row is the same chain of MMAs either way, so
    1300 frames at once equal the same frames in chunks of 100, bit for bit."""
    ref = refiner.Refiner(seed=17)
    N, H, W = 1300, 130, 100
    g = torch.Generator(device="cuda").manual_seed(3)
    x0 = torch.rand((N, H, 2, W, 8), device="cuda", generator=g).to(torch.bfloat16)
    plain = torch.rand((N, H, W), device="cuda", generator=g)
    tall = ref(x0, plain)
    short = torch.empty_like(plain)
    for c in range(0, N, 100):
        ref(x0[c:c + 100], plain[c:c + 100], out=short[c:c + 100])
    torch.cuda.synchronize()
    assert torch.equal(tall.view(torch.int32), short.view(torch.int32))
    ref.close()


def test_gradients_and_loss_match_reference():
    N, H, W = 2, 21, 140
    ref = refiner.Refiner(seed=5)
    p = ref.params()
    p[refnet.NPARAM - (9 * 32 * 16 + 16):] *= 10
    ref.set_params(p)
    x0, plain, gt = _rand_case(N, H, W, seed=7)
    loss = ref.train_step(_dev(planar(x0), torch.bfloat16), _dev(plain), _dev(gt), lr=0.0)
    g = ref.grads()
    out_ref, loss_ref, g_ref = refnet.forward(p, x0, plain, gt)
    assert math.isclose(loss, loss_ref, rel_tol=1e-3)
    assert np.array_equal(ref.params(), p)                     # lr 0 leaves the weights
    for (wo, w, bo, b) in refnet.layers(p):
        for a, n in ((wo, w.numel()), (bo, b.numel())):
            gg, gr = g[a:a + n], g_ref[a:a + n]
            if not np.any(gr):
                assert np.abs(gg).max() <= 1e-9
                continue
            rel = np.linalg.norm(gg - gr) / np.linalg.norm(gr)
            print(f"gradient block at {a}: relative L2 {rel:.2e}")
            assert rel < GRAD_TOL, (a, rel)
    ref.close()


def test_training_is_deterministic():
    """Two refiners from one seed, trained with the same batches, end with identical weights
    bit for bit: the weight gradient reduces its per-block partial sums in a fixed order."""
    N, H, W = 4, 30, 200
    x0, plain, gt = _rand_case(N, H, W, seed=13)
    args = (_dev(planar(x0), torch.bfloat16), _dev(plain), _dev(gt))
    runs = []
    for _ in range(2):
        r = refiner.Refiner(seed=21)
        grads = []
        for step in range(4):
            r.train_step(*args, lr=1e-3, want_loss=False)
            grads.append(r.grads())
        runs.append((r.params(), grads))
        r.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    for ga, gb in zip(runs[0][1], runs[1][1]):
        assert np.array_equal(ga, gb)
    assert not np.array_equal(runs[0][1][0], runs[0][1][1])   # the weights did move


def test_adam_first_step_moves_by_lr_times_sign():
    # Adam's bias-corrected first step is lr * g / (|g| + eps): lr * sign(g) where |g| >> eps
    N, H, W = 1, 16, 64
    ref = refiner.Refiner(seed=3)
    p0 = ref.params()
    x0, plain, gt = _rand_case(N, H, W, seed=1)
    args = (_dev(planar(x0), torch.bfloat16), _dev(plain), _dev(gt))
    ref.train_step(*args, lr=0.0)
    g = ref.grads()
    ref.set_params(p0)                                        # also resets the Adam state
    ref.train_step(*args, lr=1e-3)
    d = ref.params() - p0
    big = np.abs(g) > 1e-5
    assert big.sum() > 1000
    assert np.allclose(d[big], -1e-3 * np.sign(g[big]), rtol=1e-3, atol=1e-9)
    assert np.all(np.abs(d) <= 1e-3 * (1 + 1e-5))
    ref.close()


def test_params_roundtrip_and_checkpoint(tmp_path):
    a = refiner.Refiner(seed=1)
    b = refiner.Refiner(seed=2)
    assert not np.array_equal(a.params(), b.params())
    a.save(str(tmp_path / "w.npy"))
    b.load(str(tmp_path / "w.npy"))
    assert np.array_equal(a.params(), b.params())
    x0, plain, _ = _rand_case(1, 8, 40, seed=2)
    oa = a(_dev(planar(x0), torch.bfloat16), _dev(plain))
    ob = b(_dev(planar(x0), torch.bfloat16), _dev(plain))
    assert torch.equal(oa, ob)
    with pytest.raises(spk.SpkError):
        spk.spk_refiner_set_params(a.r, np.zeros(5, dtype=np.float32))
    a.close()
    b.close()


def test_argument_errors():
    r = refiner.Refiner(seed=0)
    x0, plain, _ = _rand_case(1, 4, 8, seed=0)
    host = np.zeros((1, 4, 8), dtype=np.float32)
    with pytest.raises(spk.SpkError) as e:
        spk.spk_refiner_forward(r.r, None, _dev(planar(x0), torch.bfloat16), host, 1, 4, 8, _dev(plain))
    assert e.value.code == spk.SPK_ERR_ARG
    with pytest.raises(spk.SpkError):
        spk.spk_refiner_forward(r.r, None, _dev(planar(x0), torch.bfloat16), _dev(plain), 0, 4, 8, _dev(plain))
    r.close()


def _clip(rec, w):
    stream, gt = spkgen.make_stream(w, gt_stride=w.stride)
    dev = torch.from_numpy(stream).cuda()
    plain = rec(dev, w.H, w.W, w.T)
    x0 = refiner.features(rec, dev, w.H, w.W, w.T, plain)
    gt_d = torch.from_numpy(gt).cuda().view(w.T_out, w.H, w.W)
    return x0, plain, gt_d


def test_training_beats_plain_on_held_out_stream():
    base = spkgen.WORKLOADS["dynamic_250x400x20000"]
    rec = pkg.Reconstructor(order=2, stride=base.stride)
    # 12 small clips, 1500 steps: the held-out gain is about 5 dB (asserted > 0.3 dB); the
    # headline checkpoint, trained on 10^4 full-size clips, gains about 5.7 dB on the bench stream
    clips = [_clip(rec, base.resized(H=64, W=128, T=4000, seed=s)) for s in range(21, 33)]
    test = _clip(rec, base.resized(H=64, W=128, T=4000, seed=41))
    ref = refiner.Refiner(seed=0)
    losses = refiner.fit(ref, clips, steps=1500, lr=1e-3, batch=16)
    out = ref(test[0], test[1])
    torch.cuda.synchronize()
    k0 = 20                                    # skip the head fill before the first spans close
    gt = test[2][k0:].cpu().numpy()
    plain = test[1][k0:].cpu().numpy()
    refined = out[k0:].cpu().numpy()
    p_plain, p_ref = quality.psnr(plain, gt), quality.psnr(refined, gt)
    s_plain, s_ref = quality.ssim(plain, gt), quality.ssim(refined, gt)
    print(f"PSNR plain {p_plain:.2f} refined {p_ref:.2f}; SSIM plain {s_plain:.4f} refined {s_ref:.4f}; "
          f"loss {losses[0]:.3e} -> {losses[-1]:.3e}")
    assert p_ref > p_plain + 0.3
    assert s_ref > s_plain
    ref.close()


def test_packaged_checkpoint_matches_reference_on_a_scene():
    """The whole refiner path with the trained weights (features on the GPU, tcgen05
    forward) against the PyTorch restatement on the same features: same frames within the
    forward tolerance, and the refined frames beat the plain ones."""
    w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=40, W=150, T=3000)
    rec = pkg.Reconstructor(order=2, stride=w.stride)
    stream, gt = spkgen.make_stream(w, gt_stride=w.stride)
    dev = torch.from_numpy(stream).cuda()
    plain = rec(dev, w.H, w.W, w.T)
    x0 = refiner.features(rec, dev, w.H, w.W, w.T, plain)
    ref = refiner.Refiner()
    ref.load(refiner.CHECKPOINT)
    out = ref(x0, plain)
    spk.spk_refiner_synchronize(ref.r, ref.stream.cuda_stream)
    # the restatement reads the GPU's features back in NHWC order
    xh = x0.float().cpu().numpy().transpose(0, 1, 3, 2, 4).reshape(w.T_out, w.H, w.W, 16)
    p = ref.params()
    want, _, _ = refnet.forward(p, xh, plain.cpu().numpy())
    got = out.cpu().numpy()
    corr = np.abs(want - plain.cpu().numpy()).max()
    assert np.abs(got - want).max() <= FWD_TOL * corr + 1e-6
    g = gt.reshape(w.T_out, w.H, w.W)[20:]
    assert quality.psnr(got[20:], g) > quality.psnr(plain.cpu().numpy()[20:], g) + 2.0
    ref.close()
    rec.close()
