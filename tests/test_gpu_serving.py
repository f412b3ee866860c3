"""The continuous-batching request loop: streams arriving while others run are admitted
as memory and slots free up, share launches, and each result equals its stream
reconstructed alone (bit for bit)."""
import numpy as np
import pytest

import spkgen

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_11639_gb300 as pkg
    from paper_2412_11639_gb300.serving import Request, Server
    pkg.build()
    rng = np.random.default_rng(4)
    reqs, t = [], 0.0
    for k in range(10):
        H, W, T = int(rng.integers(8, 40)), int(rng.integers(16, 80)), int(rng.integers(300, 3000))
        w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=H, W=W, T=T, seed=100 + k)
        st, _ = spkgen.make_stream(w)
        t += float(rng.exponential(0.004))
        reqs.append(Request(k, st, H, W, arrival=t, rate=2.0e5))
    srv = Server(order=2, stride=3, max_streams=4, max_piece=256)
    budget = sorted(srv.mem_needed(r) for r in reqs)[-3:]
    srv.mem_budget = sum(budget)                       # at most ~3 streams at once
    stats = srv.run(reqs)
    assert stats.peak_active >= 2                      # streams overlapped on the device
    assert stats.launches > len(reqs)
    assert 0 < stats.p50_ms <= stats.p99_ms <= stats.max_ms
    R = pkg.Reconstructor(order=2, stride=3)
    for r in reqs:
        alone = R(torch.from_numpy(r.stream).cuda(), r.H, r.W, r.T, 1.0)
        R.synchronize()
        got = srv.results[r.rid]
        assert torch.equal(got.view(torch.int32), alone.view(torch.int32)), r.rid
    R.close()
    srv.close()
