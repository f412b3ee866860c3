"""The kernel's own per-pixel scan (csrc/spk_scan.cuh), compiled for the host, against the
fp64 oracle -- on the CPU, no GPU needed (FSR, SSR, and the n-order tree of orders 3..5).

tests/c/scan_host.cpp drives PixelScan word by word as the CUDA kernel does (first spike,
whole-word absorption of steady ones, one spike() per remaining spike) and writes every
pixel's stable sequences.  They must equal the oracle's (Def. 2 greedy FSR, the two S_2
branches of SSR; Sec. III-B) exactly: spike times of every cut and interval counts.  The
program also checks the orderings the kernel's record ring depends on (a candidate at most
one place early, cut times unique, nothing before a reported frontier) and exits 3 if one
fails.
This pins the scan state machine itself; the GPU tests pin the kernel around it.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import spkgen
from conftest import ROOT


@pytest.fixture(scope="module")
def scan_host(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("scan_host") / "scan_host")
    subprocess.check_call(["g++", "-O2", "-std=c++17", os.path.join(ROOT, "tests", "c", "scan_host.cpp"),
                           "-o", exe])
    return exe


def run_host(exe, tmp_path, st, P, T, order, ring=None, layout=""):
    st = np.ascontiguousarray(st, dtype=np.uint8)
    src, dst = tmp_path / "stream.bin", tmp_path / "spans.bin"
    st.tofile(src)
    r = subprocess.run([exe, str(src), str(P), str(T), str(st.shape[1]), f"{order}{layout}", str(dst)]
                       + ([str(ring)] if ring else []), capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    raw = np.fromfile(dst, dtype=np.int32)
    counts = raw[:P]
    spans = raw[P:].reshape(-1, 3)
    assert spans.shape[0] == counts.sum()
    return counts, spans


def check_against_oracle(exe, tmp_path, st, H, W, T, order, layout=""):
    P = H * W
    counts, spans = run_host(exe, tmp_path, st, P, T, order, layout=layout)
    ref = oracle.reconstruct(st, H, W, T, 1.0, order, 1, frames=False, segments=True)
    assert np.array_equal(counts, ref.nseg), "sequence counts differ"
    assert np.array_equal(spans[:, 0], ref.seg_ts), "sequence starts differ"
    assert np.array_equal(spans[:, 1], ref.seg_te), "sequence ends differ"
    assert np.array_equal(spans[:, 2], ref.seg_n), "interval counts differ"
    return counts


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("recipe,H,W,T", [
    ("dynamic_250x400x20000", 20, 50, 3000),   # moving scene, step events, dark noise
    ("large_1000x1000x20000", 16, 40, 2500),   # moving scene down to I = 0.005
    ("static_250x400x2000", 16, 40, 2000),     # constant intensity per pixel (Theorem 1)
])
def test_scan_equals_oracle_on_scenes(scan_host, tmp_path, recipe, H, W, T, order):
    w = spkgen.WORKLOADS[recipe].resized(H=H, W=W, T=T)
    st, _ = spkgen.make_stream(w)
    counts = check_against_oracle(scan_host, tmp_path, st, H, W, T, order)
    if w.moving:
        assert counts.sum() > 10 * H * W  # cuts were exercised
    else:
        assert counts.max() == 1  # constant intensity: one stable sequence (Theorem 1)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("density", [0.1, 0.5, 0.9, 0.97])
def test_scan_equals_oracle_on_random_bits(scan_host, tmp_path, density, order):
    H, W, T = 10, 40, 1500  # T not a multiple of 32: a ragged last word
    bits = spkgen.random_bits(T, H * W, density, seed=int(density * 1000) + order)
    st = spkgen.pack(bits, H, W)
    check_against_oracle(scan_host, tmp_path, st, H, W, T, order)


@pytest.mark.parametrize("order", [1, 2])
def test_scan_equals_oracle_on_every_16_step_pattern(scan_host, tmp_path, order):
    T, P = 16, 1 << 16
    p = np.arange(P, dtype=np.int64)
    bits = np.stack([((p >> t) & 1).astype(np.uint8) for t in range(T)])  # [T][P]
    st = spkgen.pack(bits, 256, 256)
    check_against_oracle(scan_host, tmp_path, st, 256, 256, T, order)


@pytest.mark.parametrize("layout", ["", "l"])
@pytest.mark.parametrize("order", [3, 4, 5])
@pytest.mark.parametrize("recipe,H,W,T", [
    ("dynamic_250x400x20000", 12, 40, 2500),
    ("large_1000x1000x20000", 10, 40, 2000),
])
def test_tree_equals_oracle_on_scenes(scan_host, tmp_path, recipe, H, W, T, order, layout):
    """The n-order tree (Fig. 1 caption, Sec. III-B) of the same header, orders 3..5, with
    its node state in constant-indexed registers and indexed by node (local memory)."""
    w = spkgen.WORKLOADS[recipe].resized(H=H, W=W, T=T)
    st, _ = spkgen.make_stream(w)
    counts = check_against_oracle(scan_host, tmp_path, st, H, W, T, order, layout)
    assert counts.sum() > 10 * H * W


@pytest.mark.parametrize("layout", ["", "l"])
@pytest.mark.parametrize("order", [3, 5])
@pytest.mark.parametrize("density", [0.3, 0.7, 0.95])
def test_tree_equals_oracle_on_random_bits(scan_host, tmp_path, density, order, layout):
    H, W, T = 8, 40, 1200
    bits = spkgen.random_bits(T, H * W, density, seed=int(density * 1000) + 10 * order)
    st = spkgen.pack(bits, H, W)
    check_against_oracle(scan_host, tmp_path, st, H, W, T, order, layout)


@pytest.mark.parametrize("order", [3, 5])
def test_tree_ring_reports_full_and_large_ring_is_exact(scan_host, tmp_path, order):
    """The tree's pending-cut ring: a ring too small for a scene's deep cuts sets the full
    flag (exit status 4) instead of dropping cuts silently, and the largest number pending
    is reported; a ring of that size (rounded up to a power of two) reproduces the oracle."""
    w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=12, W=40, T=2500)
    st, _ = spkgen.make_stream(w)
    st = np.ascontiguousarray(st, dtype=np.uint8)
    src, dst = tmp_path / "stream.bin", tmp_path / "spans.bin"
    st.tofile(src)
    args = [scan_host, str(src), str(w.P), str(w.T), str(st.shape[1]), str(order), str(dst)]
    big = subprocess.run(args + [str(1 << 16)], capture_output=True, text=True, timeout=600)
    assert big.returncode == 0, big.stderr
    need = int(big.stderr.split("max_pending")[1].split()[0])
    assert need > 4
    small = subprocess.run(args + ["2"], capture_output=True, text=True, timeout=600)
    assert small.returncode == 4, small.stderr
    ring = 1 << (need - 1).bit_length()
    ref = oracle.reconstruct(st, w.H, w.W, w.T, 1.0, order, 1, frames=False, segments=True)
    counts, spans = run_host(scan_host, tmp_path, st, w.P, w.T, order, ring=ring)
    assert np.array_equal(counts, ref.nseg)
    assert np.array_equal(spans[:, 1], ref.seg_te)


def test_tree_state_sizes_agree(tmp_path):
    """The n-order tree's per-pixel node state, from the kernel's own type (TreeScan<n, 3> of
    the scan header, the first three levels in registers), agrees with the carried-state
    rows the C header documents for live streams (75, 131, 259 int32 for n = 3, 4, 5: 11
    scalars plus every node field) and with the serving loop's admission estimate."""
    src = tmp_path / "sizes.cpp"
    src.write_text('#include <cstdio>\n#include "' + os.path.join(ROOT, "paper_2412_11639_gb300", "csrc",
                                                               "spk_scan.cuh") + '"\n'
                   "template <int N> int rows() { using T = spk::TreeScan<N, 3>; return T::NF * (T::TOPN + T::DEEPN); }\n"
                   'int main() { std::printf("%d %d %d\\n", rows<3>(), rows<4>(), rows<5>()); }\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["g++", "-std=c++17", str(src), "-o", str(exe)])
    fields = [int(v) for v in subprocess.check_output([str(exe)], text=True).split()]
    assert [11 + f for f in fields] == [75, 131, 259]
    header = open(os.path.join(ROOT, "include", "spk.h")).read()
    assert "75, 131, 259 for" in header
    from paper_2412_11639_gb300 import serving
    for n, rows in zip((3, 4, 5), (75, 131, 259)):
        assert serving.stream_state_bytes(5, n) == 2 * 4 * rows + 2 * 2 * 64 * 4
    assert serving.stream_state_bytes(2) == 80
