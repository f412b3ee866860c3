"""Host logic of bench.py (CPU): the row slice used by --rows and the committed-profile
record the bench line reads its DRAM traffic and ALU-pipe figure from."""
import numpy as np

import bench
import spkgen


def test_cut_rows_keeps_the_first_rows_bit_for_bit():
    w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=6, W=13, T=40)  # 78 pixels, ragged byte
    bits = spkgen.random_bits(w.T, w.P, 0.4, seed=5)
    st = spkgen.pack(bits, w.H, w.W)
    for rows in (1, 3, 6):
        w2, st2 = bench.cut_rows(w, st, rows)
        assert (w2.H, w2.W, w2.T) == (rows, w.W, w.T)
        assert st2.shape == (w.T, spkgen.pitch(rows, w.W))
        P2 = rows * w.W
        got = np.unpackbits(st2, axis=1, bitorder="little")[:, :P2]
        assert np.array_equal(got, bits[:, :P2])


def test_recorded_profile_only_for_its_own_source_and_workload():
    traffic, alu = bench.recorded_profile("dynamic_250x400x20000", 2)
    kv = dict(l.strip().split("=", 1) for l in open(bench.TRAFFIC_FILE) if "=" in l and not l.startswith("#"))
    if kv["source_sha256"] == bench.kernel_source_sha():
        assert traffic == float(kv["dram_bytes_per_launch"]) and alu == float(kv["alu_pipe_active_pct"])
    else:
        assert (traffic, alu) == (None, None)
    assert bench.recorded_profile("large_1000x1000x20000", 2) == (None, None)
    assert bench.recorded_profile("dynamic_250x400x20000", 1) == (None, None)
