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
    rec = bench.recorded_profile("dynamic_250x400x20000", 2)
    kv = dict(l.strip().split("=", 1) for l in open(bench.TRAFFIC_FILE) if "=" in l and not l.startswith("#"))
    if kv["source_sha256"] == bench.kernel_source_sha():
        assert rec["traffic"] == float(kv["dram_bytes_per_launch"])
        assert rec["alu_pct"] == float(kv["alu_pipe_active_pct"])
        assert rec["alu_inst"] == float(kv["alu_warp_inst_per_launch"])
        # the ALU roofline: instructions over the live kernel time against the pipe's peak
        # at the sampled clock (2 warp instructions per SM per cycle)
        r = bench.alu_roofline(rec, 2.0, {"sm_mhz": 2000.0})
        assert r["bound"] == "alu"
        assert abs(r["achieved"] - rec["alu_inst"] / 2e-3 / 1e9) < 1e-9 * r["achieved"]
        assert abs(r["peak"] - rec["alu_peak_per_cycle"] * 2.0) < 1e-9
        assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    else:
        assert rec == {}
    assert bench.recorded_profile("large_1000x1000x20000", 2) == {}
    assert bench.recorded_profile("dynamic_250x400x20000", 1) == {}
    assert bench.alu_roofline({}, 2.0, None) is None
