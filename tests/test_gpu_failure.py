"""Failure detection on the device without a fault: a bounded wait runs out, the kernel
returns, the host reads SPK_ERR_TIMEOUT, and the context keeps working."""
import numpy as np
import pytest

import spkgen

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_11639_gb300 as pkg
    from paper_2412_11639_gb300 import spk
    pkg.build()
    R = pkg.Reconstructor(order=2, stride=1)
    spk.spk_selftest_wait(R.ctx, 2_000_000)          # ~1 ms of waiting on nothing
    with pytest.raises(spk.SpkError) as e:
        R.synchronize()
    assert e.value.code == spk.SPK_ERR_TIMEOUT
    # the status word was cleared and the context still reconstructs
    b = spkgen.random_bits(100, 64, 0.5, seed=1)
    f = R(torch.from_numpy(spkgen.pack(b)).cuda(), 1, 64, 100, 1.0)
    R.synchronize()
    assert torch.isfinite(f).all()
    R.close()


def test_allocation_failures_report_oom_and_context_survives():
    """With the allocation hook armed, every allocating entry point returns SPK_ERR_OOM
    (context, live-stream state, host-call staging, asynchronous lanes), leaves nothing
    half-made, and the next call succeeds."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_11639_gb300 as pkg
    from paper_2412_11639_gb300 import spk
    pkg.build()
    H, W, T = 8, 40, 300
    st = spkgen.pack(spkgen.random_bits(T, H * W, 0.4, seed=3), H, W)
    host_in = torch.from_numpy(st).pin_memory()
    host_out = torch.empty((T, H, W), dtype=torch.float32).pin_memory()

    def expect_oom(call):
        spk.spk_debug_fail_allocations(1)
        with pytest.raises(spk.SpkError) as e:
            call()
        spk.spk_debug_fail_allocations(0)
        assert e.value.code == spk.SPK_ERR_OOM

    expect_oom(lambda: spk.spk_create(2, 1, spk.SPK_F32, 0, None))
    R = pkg.Reconstructor(order=2, stride=1)
    expect_oom(lambda: spk.spk_stream_open(R.ctx, H, W, T))
    expect_oom(lambda: spk.spk_reconstruct_host(R.ctx, host_in, H, W, T, 1.0, host_out))
    expect_oom(lambda: spk.spk_reconstruct_host_async(R.ctx, host_in, H, W, T, 1.0, host_out))
    # the same calls work once the hook is cleared, with the device result
    spk.spk_reconstruct_host(R.ctx, host_in, H, W, T, 1.0, host_out)
    want = R(torch.from_numpy(st).cuda(), H, W, T, 1.0)
    R.synchronize()
    assert torch.equal(host_out, want.cpu())
    s = spk.spk_stream_open(R.ctx, H, W, T)
    spk.spk_stream_close(R.ctx, s)
    R.close()
    with pytest.raises(spk.SpkError):
        spk.spk_debug_fail_allocations(-1)


def test_c_abi_from_plain_c(tmp_path):
    """A plain C program (tests/c/abi_demo.c) linked against libspk.so reconstructs a
    constant-interval stream through host buffers (and the asynchronous variant) and checks
    every frame and a few error codes."""
    import os
    import subprocess

    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_11639_gb300 as pkg
    from conftest import ROOT
    lib = pkg.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "abi_demo")
    subprocess.check_call(["gcc", "-O2", "-std=c11", os.path.join(ROOT, "tests", "c", "abi_demo.c"),
                           "-I", os.path.join(ROOT, "include"), os.path.join(libdir, "libspk.so"),
                           f"-Wl,-rpath,{libdir}", "-lm", "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert "abi_demo ok" in out.stdout
