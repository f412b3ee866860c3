"""The GPU twin of the stream generator (spkgen/gen.cu) writes the same bits as the C
generator: every stream byte and every ground-truth value, on small clips of each recipe."""
import numpy as np
import pytest

import spkgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,H,W,T", [("dynamic_250x400x20000", 37, 53, 3000),
                                        ("static_250x400x2000", 16, 129, 500),
                                        ("large_1000x1000x20000", 64, 64, 1000),
                                        ("dynamic_250x400x20000", 250, 400, 400)])
def test_gpu_generator_is_bit_exact(name, H, W, T):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    w = spkgen.WORKLOADS[name].resized(H=H, W=W, T=T)
    st, gt = spkgen.make_stream(w, gt_stride=7)
    dst, dgt = spkgen.make_stream_cuda(w, gt_stride=7)
    assert np.array_equal(dst.cpu().numpy(), st)
    assert np.array_equal(dgt.cpu().numpy().view(np.uint32), gt.view(np.uint32))
    assert st.any()
