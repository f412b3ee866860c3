"""TFI and TFP (Sec. II baselines) on the GPU against the fp64 oracle: fp32 within 1e-6
relative, fp16 equal to the rounding of the fp32 value."""
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


def _run(env, st, H, W, T, method, stride, dtype, window=32):
    torch, pkg = env
    R = pkg.Reconstructor(order=method, stride=stride, dtype=dtype, tfp_window=window)
    f = R(torch.from_numpy(st).cuda(), H, W, T, 1.0)
    R.synchronize()
    out = f.cpu().numpy().reshape(f.shape[0], -1)
    R.close()
    return out


def _check(got, ref, f16):
    if f16:
        assert np.array_equal(got.view(np.uint16), ref.astype(np.float32).astype(np.float16).view(np.uint16))
    else:
        assert np.all(np.abs(got.astype(np.float64) - ref) <= 1e-6 * np.abs(ref))


@pytest.mark.parametrize("H,W,T,stride,density", [(1, 1, 1, 1, 0.5), (3, 11, 63, 2, 0.5),
                                                   (17, 31, 1000, 1, 0.3), (2, 200, 3001, 7, 0.9),
                                                   (4, 64, 500, 1, 0.0)])
def test_tfi_random(env, H, W, T, stride, density):
    b = spkgen.random_bits(T, H * W, density, seed=H + W + T)
    st = spkgen.pack(b, H, W)
    for f16 in (False, True):
        got = _run(env, st, H, W, T, 3, stride, env[0].float16 if f16 else env[0].float32)
        _check(got, oracle.tfi(st, H, W, T, 1.0, stride), f16)


@pytest.mark.parametrize("window", [1, 7, 32, 33, 64])
@pytest.mark.parametrize("stride", [1, 5])
def test_tfp_random(env, window, stride):
    H, W, T = 5, 53, 700
    b = spkgen.random_bits(T, H * W, 0.4, seed=window * 10 + stride)
    st = spkgen.pack(b, H, W)
    got = _run(env, st, H, W, T, 4, stride, env[0].float32, window)
    _check(got, oracle.tfp(st, H, W, T, window, 1.0, stride), False)


def test_baselines_on_scene_workloads(env):
    torch = env[0]
    w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=40, W=70, T=3000)
    st, _ = spkgen.make_stream(w)
    _check(_run(env, st, w.H, w.W, w.T, 3, w.stride, torch.float32),
           oracle.tfi(st, w.H, w.W, w.T, 1.0, w.stride), False)
    for L in (32, 64):
        _check(_run(env, st, w.H, w.W, w.T, 4, w.stride, torch.float32, L),
               oracle.tfp(st, w.H, w.W, w.T, L, 1.0, w.stride), False)
    w = spkgen.WORKLOADS["large_1000x1000x20000"].resized(H=30, W=50, T=2000)
    st, _ = spkgen.make_stream(w)
    _check(_run(env, st, w.H, w.W, w.T, 4, 1, torch.float16, 64), oracle.tfp(st, w.H, w.W, w.T, 64, 1.0, 1), True)
