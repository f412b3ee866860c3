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
