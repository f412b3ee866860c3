"""The C-ABI library builds, loads and exports every symbol include/spk.h declares; host-side
argument checks reject bad calls before any device work.  CPU only (no compute calls)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT
import paper_2412_11639_gb300 as pkg
from paper_2412_11639_gb300 import spk


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "spk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spk_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return spk.load()


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n          # ctypes resolves exported symbols only
    assert set(names) == set(spk.EXPORTS)


def test_layout_helpers(lib):
    assert spk.spk_pitch(250, 400) == 12512          # ceil(100000/8)=12500 -> 12512
    assert spk.spk_pitch(1000, 1000) == 125008
    assert spk.spk_pitch(1, 1) == 16
    assert spk.spk_pitch(1, 128) == 16
    assert spk.spk_pitch(1, 129) == 32
    assert spk.spk_pitch(0, 5) == -1 and spk.spk_pitch(5, -1) == -1
    assert spk.spk_num_frames(20000, 10) == 2000
    assert spk.spk_num_frames(2001, 10) == 201
    assert spk.spk_num_frames(1, 7) == 1
    assert spk.spk_num_frames(0, 1) == -1 and spk.spk_num_frames(5, 0) == -1


def test_create_rejects_bad_config(lib):
    out = ctypes.c_void_p()
    assert lib.spk_create(ctypes.byref(out), None) == spk.SPK_ERR_ARG
    for cfg in (spk.spk_config(6, 1, 0, 0, None, 32, 3), spk.spk_config(0, 1, 0, 0, None, 32, 3),
                spk.spk_config(2, 0, 0, 0, None, 32, 3), spk.spk_config(1, 1, 7, 0, None, 32, 3),
                spk.spk_config(4, 1, 0, 0, None, 0, 3), spk.spk_config(4, 1, 0, 0, None, 65, 3),
                spk.spk_config(5, 1, 0, 0, None, 32, 2), spk.spk_config(5, 1, 0, 0, None, 32, 6),
                spk.spk_config(2, 1, 3, 0, None, 32, 3), spk.spk_config(2, 1, 0, 0, None, 32, 3, 4),
                spk.spk_config(2, 1, 2, 0, None, 32, 3, -1)):
        assert lib.spk_create(ctypes.byref(out), ctypes.byref(cfg)) == spk.SPK_ERR_ARG
        assert out.value is None
        assert spk.spk_last_error(None)


def test_null_context_calls(lib):
    assert lib.spk_destroy(None) == spk.SPK_OK
    assert lib.spk_reconstruct(None, None, 1, 1, 1, 1.0, None) == spk.SPK_ERR_ARG
    assert lib.spk_segments(None, None, 1, 1, 1, 1.0, None, None, None, None, None, None, 0) == spk.SPK_ERR_ARG
    assert lib.spk_synchronize(None) == spk.SPK_ERR_ARG
    assert lib.spk_launch_count(None) == 0


def test_no_gpu_is_reported_not_faked(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(spk.SpkError) as e:
        spk.spk_create(2, 1, spk.SPK_F32, 0, None)
    assert e.value.code == spk.SPK_ERR_CUDA


def test_package_has_no_oracle_dependency():
    """The product package never reaches the oracle (test infrastructure only)."""
    pdir = os.path.join(ROOT, "paper_2412_11639_gb300")
    for dp, _, files in os.walk(pdir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "oracle.c" not in txt, f


def test_noalloc_rejects_oversize_before_device_work(lib):
    """The allocation-free entry point refuses problems beyond its fixed scratch (the C side,
    called directly with a one-element frame buffer it must never touch), and the Python
    binding refuses host buffers smaller than the call would write."""
    import ctypes

    import numpy as np
    st = np.zeros((4000, spk.spk_pitch(1000, 1000)), dtype=np.uint8)
    out = np.full(1, -3.0, dtype=np.float32)
    cfg = spk.spk_config(spk.SPK_SSR, 1, spk.SPK_F32, 0, None, 32, 3)
    rc = lib.spk_reconstruct_host_noalloc(ctypes.byref(cfg), st.ctypes.data, 1000, 1000, 4000, 1.0,
                                          out.ctypes.data)
    assert rc == spk.SPK_ERR_ARG
    assert "scratch" in spk.spk_last_error(None)
    rc = lib.spk_reconstruct_host_noalloc(ctypes.byref(cfg), st.ctypes.data, 1, 8, 4, float("nan"),
                                          out.ctypes.data)
    assert rc == spk.SPK_ERR_ARG
    for theta in (1.5, 0.0, 65536.0):  # 8-bit frames need an integral threshold, 1 .. 65535
        cfg8 = spk.spk_config(spk.SPK_SSR, 1, spk.SPK_U8, 0, None, 32, 3)
        rc = lib.spk_reconstruct_host_noalloc(ctypes.byref(cfg8), st.ctypes.data, 1, 8, 4, theta,
                                              out.ctypes.data)
        assert rc == spk.SPK_ERR_ARG
    assert "integral" in spk.spk_last_error(None)
    assert out[0] == -3.0
    with pytest.raises(ValueError):
        spk.spk_reconstruct_host_noalloc(st, 1000, 1000, 4000, 1.0, out)


def test_refiner_host_checks(lib):
    import torch
    # 9 * Cin * Cout + Cout per layer for 16 -> 32 -> 32 -> 32 -> 32 -> 16
    assert spk.spk_refiner_num_params() == 9 * 16 * 32 + 32 + 3 * (9 * 32 * 32 + 32) + 9 * 32 * 16 + 16
    assert lib.spk_refiner_destroy(None) == spk.SPK_OK
    assert lib.spk_refiner_create(0, 0, None) == spk.SPK_ERR_ARG
    assert lib.spk_refiner_forward(None, None, None, None, 1, 1, 1, None) == spk.SPK_ERR_ARG
    assert lib.spk_refiner_train_step(None, None, None, None, None, 1, 1, 1, 0.0, None) == spk.SPK_ERR_ARG
    assert lib.spk_refiner_set_params(None, None, 0) == spk.SPK_ERR_ARG
    assert lib.spk_features(None, None, 1, 1, 1, 1.0, None, None) == spk.SPK_ERR_ARG
    if not torch.cuda.is_available():
        with pytest.raises(spk.SpkError) as e:
            spk.spk_refiner_create(0, 1)
        assert e.value.code == spk.SPK_ERR_CUDA


def test_packaged_refiner_checkpoint():
    import numpy as np
    from paper_2412_11639_gb300 import refiner
    p = np.load(refiner.CHECKPOINT)
    assert p.dtype == np.float32 and p.shape == (spk.spk_refiner_num_params(),)
    assert np.isfinite(p).all() and np.abs(p).max() < 10
