"""The continuous-batching request loop: streams arriving while others run are admitted
as memory and slots free up, share launches, and each result equals its stream
reconstructed alone (bit for bit)."""
import numpy as np
import pytest

import spkgen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("order,n", [(2, 3), (5, 3)])
def test_served_results_equal_alone(order, n):
    """SSR, and the n-order tree (n = 3) whose live streams carry the tree's state."""
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
    srv = Server(order=order, stride=3, max_streams=4, max_piece=256, stability_order=n)
    budget = sorted(srv.mem_needed(r) for r in reqs)[-3:]
    srv.mem_budget = sum(budget)                       # at most ~3 streams at once
    stats = srv.run(reqs)
    assert stats.peak_active >= 2                      # streams overlapped on the device
    assert stats.launches > len(reqs)
    assert 0 < stats.p50_ms <= stats.p99_ms <= stats.max_ms
    R = pkg.Reconstructor(order=order, stride=3, stability_order=n)
    for r in reqs:
        alone = R(torch.from_numpy(r.stream).cuda(), r.H, r.W, r.T, 1.0)
        R.synchronize()
        got = srv.results[r.rid]
        assert torch.equal(got.view(torch.int32), alone.view(torch.int32)), r.rid
    R.close()
    srv.close()


def test_cancelled_requests_leave_and_the_rest_is_unchanged():
    """A request cancelled while waiting never runs; one cancelled while active gives its
    slot and state back at the next tick; every other result still equals its stream alone."""
    import threading

    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_11639_gb300 as pkg
    from paper_2412_11639_gb300.serving import Request, Server
    pkg.build()
    rng = np.random.default_rng(8)
    reqs = []
    for k in range(6):
        H, W, T = int(rng.integers(8, 32)), int(rng.integers(16, 64)), int(rng.integers(500, 2500))
        w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=H, W=W, T=T, seed=200 + k)
        st, _ = spkgen.make_stream(w)
        rate = 1.0e4 if k == 0 else 2.0e5               # request 0 runs for 50-250 ms
        reqs.append(Request(k, st, H, W, arrival=0.002 * k if k < 5 else 0.4, rate=rate))
    srv = Server(order=2, stride=3, max_streams=4, max_piece=256)
    srv.cancel(5)                                      # still waiting: dropped
    timer = threading.Timer(0.03, srv.cancel, args=(0,))  # active by then: leaves mid-stream
    timer.start()
    stats = srv.run(reqs)
    timer.join()
    assert stats.cancelled == 2
    assert 0 not in srv.results and 5 not in srv.results
    R = pkg.Reconstructor(order=2, stride=3)
    for r in reqs[1:5]:
        alone = R(torch.from_numpy(r.stream).cuda(), r.H, r.W, r.T, 1.0)
        R.synchronize()
        assert torch.equal(srv.results[r.rid].view(torch.int32), alone.view(torch.int32)), r.rid
    R.close()
    srv.close()
