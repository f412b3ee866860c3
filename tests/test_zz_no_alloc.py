"""The allocation-free host-buffer entry point (spk_reconstruct_host_noalloc).

It serves callers that may not allocate device memory (a foreign allocator owns the
device, or a camera loop cannot pay for cudaMalloc / cudaFree); it stages the stream and
frames in the library's fixed 16 MiB device array, which keeps the previous call's
contents.  Every method it accepts is checked against the fp64 oracle (fp32 within 1e-6
relative, fp16 the round-to-nearest-even of the fp32 value), calls follow each other on
different streams and settings so that nothing of one call leaks into the next, the
context-based spk_reconstruct_host gives the same frames, and a problem one block over the
array's capacity is refused before any device work.  Collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import spkgen

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6


@pytest.fixture(scope="module")
def spk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_11639_gb300 as pkg
    from paper_2412_11639_gb300 import spk as lib
    pkg.build()
    return lib


def _oracle_frames(st, H, W, T, method, stride, window, n):
    if method == 3:
        return oracle.tfi(st, H, W, T, 1.0, stride)
    if method == 4:
        return oracle.tfp(st, H, W, T, window, 1.0, stride)
    return oracle.reconstruct(st, H, W, T, 1.0, n if method == 5 else method, stride).frames


def _check_against_oracle(got, ref, f16):
    got = got.reshape(got.shape[0], -1)
    if f16:
        want = ref.astype(np.float32).astype(np.float16)
        assert np.array_equal(got.view(np.uint16), want.view(np.uint16))
    else:
        assert np.all(np.abs(got.astype(np.float64) - ref) <= REL_TOL * np.abs(ref))


def _host_entry_point(spk, st, H, W, T, method, stride, dtype, window, n):
    ctx = spk.spk_create(method, stride, dtype, 0, None, window, n)
    out = np.empty((spk.spk_num_frames(T, stride), H, W),
                   dtype=np.float16 if dtype == spk.SPK_F16 else np.float32)
    spk.spk_reconstruct_host(ctx, st, H, W, T, 1.0, out)
    spk.spk_destroy(ctx)
    return out


CASES = [
    # (recipe, H, W, T, method, stride, f16, tfp_window, stability_order): all fit 16 MiB
    ("dynamic_250x400x20000", 48, 100, 3000, 2, 10, False, 32, 3),   # SSR
    ("large_1000x1000x20000", 40, 70, 1500, 1, 1, True, 32, 3),      # FSR, fp16 every step
    ("dynamic_250x400x20000", 30, 64, 2000, 3, 3, False, 32, 3),     # TFI
    ("dynamic_250x400x20000", 30, 64, 2000, 4, 1, True, 32, 3),      # TFP-32
    ("dynamic_250x400x20000", 30, 50, 2500, 5, 5, False, 32, 3),     # third-order tree
]


def test_noalloc_every_method_against_oracle_in_a_row(spk):
    import torch
    side = torch.cuda.Stream()
    for k, (name, H, W, T, method, stride, f16, window, n) in enumerate(CASES):
        w = spkgen.WORKLOADS[name].resized(H=H, W=W, T=T, seed=100 + k)
        st, _ = spkgen.make_stream(w)
        dtype = spk.SPK_F16 if f16 else spk.SPK_F32
        got = np.full((spk.spk_num_frames(T, stride), H, W), np.nan,
                      dtype=np.float16 if f16 else np.float32)
        # alternate the default stream and a side stream between calls
        spk.spk_reconstruct_host_noalloc(st, H, W, T, 1.0, got, method=method, frame_stride=stride,
                                         out_dtype=dtype, device=0,
                                         stream=side.cuda_stream if k % 2 else None,
                                         tfp_window=window, stability_order=n)
        ref = _oracle_frames(st, H, W, T, method, stride, window, n)
        assert np.any(ref != 0)
        _check_against_oracle(got, ref, f16)
        host = _host_entry_point(spk, st, H, W, T, method, stride, dtype, window, n)
        assert np.array_equal(got.view(np.uint8), host.view(np.uint8)), (name, method)


def test_noalloc_capacity_boundary(spk):
    """64 x 64 pixels, fp32 every step: 992 steps need 256 + 507,904 + 16,252,928 bytes
    (fits the 16,777,216), 993 steps 768 bytes more than the array holds."""
    H, W = 64, 64
    assert spk.SPK_NOALLOC_SCRATCH_BYTES == 16 << 20
    w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=H, W=W, T=993, seed=7)
    st, _ = spkgen.make_stream(w)
    got = np.full((992, H, W), np.nan, dtype=np.float32)
    spk.spk_reconstruct_host_noalloc(np.ascontiguousarray(st[:992]), H, W, 992, 1.0, got, method=2)
    _check_against_oracle(got, oracle.reconstruct(st, H, W, 992, 1.0, 2, 1).frames, False)

    big = np.full((993, H, W), -7.0, dtype=np.float32)
    with pytest.raises(spk.SpkError) as e:
        spk.spk_reconstruct_host_noalloc(st, H, W, 993, 1.0, big, method=2)
    assert e.value.code == spk.SPK_ERR_ARG
    assert np.all(big == -7.0)          # refused before any device work


def test_noalloc_refuses_mismatched_host_buffers(spk):
    H, W, T = 8, 40, 100
    st = spkgen.pack(spkgen.random_bits(T, H * W, 0.4, seed=1), H, W)
    with pytest.raises(ValueError):       # fp16 buffer for fp32 output
        spk.spk_reconstruct_host_noalloc(st, H, W, T, 1.0, np.empty((T, H, W), np.float16))
    with pytest.raises(ValueError):       # one frame short
        spk.spk_reconstruct_host_noalloc(st, H, W, T, 1.0, np.empty((T - 1, H, W), np.float32))
    with pytest.raises(ValueError):       # strided view
        spk.spk_reconstruct_host_noalloc(st, H, W, T, 1.0, np.empty((T, H, 2 * W), np.float32)[:, :, ::2])
