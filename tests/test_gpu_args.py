"""Argument checks of the reconstruction calls on a GPU: every refused call returns
SPK_ERR_ARG before any launch, says what is wrong, writes nothing, and leaves the context
usable (sizes past the limits, empty sizes, bad thresholds, misaligned, overlapping,
NULL and host pointers)."""
import numpy as np
import pytest

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


def test_reconstruct_rejects_bad_arguments(env):
    torch, pkg = env
    from paper_2412_11639_gb300 import spk
    lib = spk.load()
    R = pkg.Reconstructor(order=2)
    H, W, T = 4, 40, 100
    pitch = spkgen.pitch(H, W)
    st = torch.from_numpy(spkgen.pack(spkgen.random_bits(T, H * W, 0.4, seed=2), H, W)).cuda()
    out = torch.full((T, H, W), -7.0, device="cuda")
    s0, o0 = st.data_ptr(), out.data_ptr()
    host = np.zeros(T * pitch + 32, dtype=np.uint8)
    h0 = host.ctypes.data + (-host.ctypes.data) % 16        # 16-byte aligned, pageable host
    cases = [
        ((s0, 0, W, T, 1.0, o0), "H, W, T"),
        ((s0, H, -3, T, 1.0, o0), "H, W, T"),
        ((s0, H, W, 0, 1.0, o0), "H, W, T"),
        ((s0, H, W, T, float("nan"), o0), "threshold"),
        ((s0, H, W, T, float("inf"), o0), "threshold"),
        ((s0, H, W, T, 0.0, o0), "threshold"),
        ((s0, H, W, T, -1.0, o0), "threshold"),
        ((s0 + 1, H, W, T, 1.0, o0), "aligned"),
        ((s0, H, W, T, 1.0, o0 + 4), "aligned"),
        ((s0, 46341, 46341, T, 1.0, o0), "too large"),      # H*W above 2^31 - 256
        ((s0, H, W, (1 << 30) + 1, 1.0, o0), "too large"),  # T above 2^30
        ((None, H, W, T, 1.0, o0), "NULL"),
        ((s0, H, W, T, 1.0, None), "NULL"),
        ((s0, H, W, T, 1.0, s0 + 16), "overlaps"),
        ((h0, H, W, T, 1.0, o0), "device memory"),
    ]
    n0 = spk.spk_launch_count(R.ctx)
    for args, what in cases:
        rc = lib.spk_reconstruct(R.ctx, *args)
        assert rc == spk.SPK_ERR_ARG, (args, rc)
        assert what in spk.spk_last_error(R.ctx), (args, spk.spk_last_error(R.ctx))
    assert spk.spk_launch_count(R.ctx) == n0                 # nothing launched
    R.synchronize()
    assert bool((out == -7.0).all())                         # nothing written
    f = R(st, H, W, T, 1.0, out=out)                         # the context still works
    R.synchronize()
    assert bool(torch.isfinite(f).all()) and spk.spk_launch_count(R.ctx) == n0 + 1
    R.close()


def test_segments_rejects_bad_arguments(env):
    torch, pkg = env
    from paper_2412_11639_gb300 import spk
    lib = spk.load()
    H, W, T = 2, 16, 64
    st = torch.from_numpy(spkgen.pack(spkgen.random_bits(T, H * W, 0.5, seed=4), H, W)).cuda()
    counts = torch.zeros(H * W, dtype=torch.int32, device="cuda")
    R = pkg.Reconstructor(order=2)
    assert lib.spk_segments(R.ctx, st.data_ptr(), H, W, T, 1.0, None, None, None, None, None, None,
                            0) == spk.SPK_ERR_ARG                    # counts NULL
    assert lib.spk_segments(R.ctx, st.data_ptr(), H, W, T, 1.0, None, counts.data_ptr(), None, None,
                            None, None, 4) == spk.SPK_ERR_ARG        # cap > 0 without arrays
    R.close()
    Rt = pkg.Reconstructor(order=4)                                  # TFP has no stable spans
    assert lib.spk_segments(Rt.ctx, st.data_ptr(), H, W, T, 1.0, None, counts.data_ptr(), None, None,
                            None, None, 0) == spk.SPK_ERR_ARG
    assert "TFP" in spk.spk_last_error(Rt.ctx)
    Rt.close()
