"""Pins of the oracle (and of the stream generator) against what the paper and the
mathematics fix, independently of the oracle's own code.  CPU only.

* closed form of Eq. 2 for a constant intensity (spike times, Lemma 1's two intervals);
* Lemma 2: the interval stream is regenerated by an integrator G_1 (Eq. 13-14);
* Theorem 1: a constant-intensity stream is one stable sequence under FSR and SSR;
* the Eq. 4 estimate lies within Q/D of the true rate, exactly when theta/Q is integral;
* step edges large enough to leave the {a, a+1} set are split, small ones are not;
* structural invariants on the moving-scene recipe (tiling, sums, zero-order stability,
  greedy maximality, SSR refines FSR, SSR sequences are second-order stable);
* TFI (Sec. II) as the special case of one-interval sequences;
* hand-derived golden cases, and the set-based literal reading of Def. 2 (exhaustive on
  all 2^16 patterns of 16 steps and on random 4x4x64 streams).
"""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle
import spkgen
from oracle import bruteforce as bf
from conftest import load_golden


def _const_stream(Q, r0, T, theta=1.0):
    Q = np.asarray(Q, dtype=np.float64)
    r0 = np.asarray(r0, dtype=np.float64)
    q = np.broadcast_to(Q, (T, Q.shape[0])).copy()
    return spkgen.simulate_table(q, r0, theta)


def _bits(stream, p, T):
    return [(int(stream[n, p >> 3]) >> (p & 7)) & 1 for n in range(T)]


# ----------------------------------------------------------------- Eq. 2 closed form ----
def test_eq2_spike_times_closed_form():
    """Constant Q <= theta, residual r0: spike k (k = 1, 2, ...) fires at step
    ceil((k theta - r0) / Q) - 1.  Dyadic Q and r0 keep fp64 accumulation exact."""
    rng = np.random.default_rng(11)
    T = 600
    Q = rng.integers(1, 257, 64) / 256.0          # (0, 1] in steps of 1/256
    r0 = rng.integers(0, 256, 64) / 256.0 * Q     # [0, Q) ... dyadic
    r0 = np.floor(r0 * 1024) / 1024
    st = _const_stream(Q, r0, T)
    for p in range(64):
        got = oracle.spike_times(st, T, p).tolist()
        q, r = Fraction(Q[p]), Fraction(r0[p])
        exp = []
        k = 1
        while True:
            n = math.ceil((k - r) / q) - 1
            if n >= T:
                break
            exp.append(n)
            k += 1
        assert got == exp, p


def test_lemma1_two_intervals():
    """Lemma 1 (Eq. 7-9): with fixed Q, every interval is floor(T*) or floor(T*) + 1,
    T* = theta / Q (exact rational value of the fp64 Q)."""
    rng = np.random.default_rng(12)
    T = 3000
    Q = rng.uniform(0.02, 1.0, 200)
    r0 = rng.uniform(0, 1, 200)
    st = _const_stream(Q, r0, T)
    for p in range(200):
        s = oracle.spike_times(st, T, p)
        x = set(np.diff(s).tolist())
        f = math.floor(Fraction(1) / Fraction(Q[p]))
        assert x <= {f, f + 1}, (p, Q[p], x)


def test_lemma2_interval_stream_is_integrate_and_fire():
    """Lemma 2 (Eq. 10-14): after a fire the residual r decides the next interval:
    floor(T*) ('-' firing value) iff r + Q_1 >= M_1th with Q_1 = (1-b) Q, M_1th = Q,
    then r drops by M_1th; otherwise the interval is floor(T*) + 1.  Exact rationals."""
    rng = np.random.default_rng(13)
    T = 4000
    Q = rng.integers(5, 1000, 40) / 1024.0
    r0 = np.zeros(40)
    st = _const_stream(Q, r0, T)
    for p in range(40):
        s = oracle.spike_times(st, T, p)
        q = Fraction(Q[p])
        Tstar = 1 / q
        f = math.floor(Tstar)
        b = Tstar - f
        # residual after the first fire at s_0
        r = (s[0] + 1) * q - 1
        Q1, M1 = (1 - b) * q, q
        M = r                       # status of G_1 after its own reset
        gen = []
        for _ in range(len(s) - 1):
            M = M + Q1
            if M >= M1:
                gen.append(f)
                M -= M1
            else:
                gen.append(f + 1)
        assert np.diff(s).tolist() == gen, p


# --------------------------------------------------------------------- Theorem 1 ----
@pytest.mark.parametrize("order", [1, 2])
def test_theorem1_constant_intensity_is_one_sequence(order):
    rng = np.random.default_rng(14)
    T, P = 2000, 512
    Q = rng.uniform(0.02, 1.0, P)
    r0 = rng.uniform(0, 1, P)
    st = _const_stream(Q, r0, T)
    r = oracle.reconstruct(st, 1, P, T, 1.0, order, 1, frames=False, segments=True)
    assert np.all(r.K >= 2)
    assert np.all(r.nseg == 1)


@pytest.mark.parametrize("order", [1, 2])
def test_theorem1_static_workload(order):
    """Every pixel of the static 250x400x2000 workload sees a constant intensity."""
    w = spkgen.WORKLOADS["static_250x400x2000"]
    st, _ = spkgen.make_stream(w)
    r = oracle.reconstruct(st, w.H, w.W, w.T, 1.0, order, 1, frames=False)
    assert np.all(r.nseg == 1)


def test_estimate_bound_and_exact_cases():
    """Over a sequence D Q - N theta = r_end - r_start with residuals in [0, Q), so
    |theta N / D - Q| < Q / D; exact when theta / Q is an integer (all intervals equal)."""
    rng = np.random.default_rng(15)
    T, P = 2000, 300
    Q = rng.uniform(0.02, 1.0, P)
    Q[:40] = 1.0 / rng.integers(1, 50, 40)
    Q[:40] = 1.0 / np.round(1.0 / Q[:40])
    r0 = rng.uniform(0, 1, P) * Q
    st = _const_stream(Q, r0, T)
    r = oracle.reconstruct(st, 1, P, T, 1.0, 2, 1, frames=False, segments=True)
    for p in range(P):
        ts, te, n, v = r.segments(p)
        D = int(te[0] - ts[0])
        assert abs(v[0] - Q[p]) < Q[p] / D + 1e-15, p
    for p in range(40):
        ts, te, n, v = r.segments(p)
        inv = round(1.0 / Q[p])
        if abs(1.0 / Q[p] - inv) < 1e-12 and Fraction(Q[p]) == Fraction(1, inv):
            assert Fraction(int(n[0]), int(te[0] - ts[0])) == Fraction(1, inv)


# --------------------------------------------------------------------- step edges ----
@pytest.mark.parametrize("order", [1, 2])
def test_step_edge_is_split(order):
    """I1 -> I2 with |theta/I1 - theta/I2| >= 4 leaves every {a, a+1} set: FSR makes one
    or two cuts at the edge (2 or 3 sequences); SSR never has fewer sequences.  Eq. 2 over
    the steps (t_start, t_end] of any sequence gives theta N = sum Q(n) + r_start - r_end
    with residuals below the charge of their own spike step, so every value is within
    max Q / D of the mean charge over the sequence."""
    rng = np.random.default_rng(16)
    T, P, te = 2000, 256, 1000
    I1 = rng.uniform(0.05, 1.0, P)
    I2 = np.where(rng.uniform(size=P) < 0.5, I1 / rng.uniform(2, 8, P), I1 * rng.uniform(2, 8, P))
    I2 = np.clip(I2, 0.02, 1.0)
    ok = np.abs(1 / I1 - 1 / I2) >= 4
    q = np.empty((T, P))
    q[:te] = I1
    q[te:] = I2
    st = spkgen.simulate_table(q, rng.uniform(0, 1, P) * I1)
    r1 = oracle.reconstruct(st, 1, P, T, 1.0, 1, 1, frames=False, segments=True)
    r = oracle.reconstruct(st, 1, P, T, 1.0, order, 1, frames=False, segments=True)
    assert ok.sum() > 100
    for p in np.nonzero(ok)[0]:
        assert r1.nseg[p] in (2, 3), p
        assert r.nseg[p] >= r1.nseg[p]
        ts, tend, n, v = r.segments(p)
        for j in range(len(ts)):
            seg_q = q[ts[j] + 1: tend[j] + 1, p]
            D = tend[j] - ts[j]
            qmax = q[ts[j]: tend[j] + 1, p].max()    # residuals are below Q of their step
            assert abs(v[j] - seg_q.mean()) < qmax / D + 1e-12, (p, j)
        # the outer sequences lie on one side of the edge except for one interval
        assert abs(v[0] - I1[p]) < 2 * max(I1[p], I2[p]) / (tend[0] - ts[0]) + 1e-12
        assert abs(v[-1] - I2[p]) < 2 * max(I1[p], I2[p]) / (tend[-1] - ts[-1]) + 1e-12


def test_small_step_stays_one_sequence():
    """I 0.5 -> 1.0 gives intervals 2 then 1: the set {1, 2} is zero-order stable, so
    neither FSR nor SSR splits it (a step the stability rule cannot see)."""
    T = 400
    q = np.empty((T, 1))
    q[:200] = 0.5
    q[200:] = 1.0
    st = spkgen.simulate_table(q, np.array([0.5]))
    for order in (1, 2):
        r = oracle.reconstruct(st, 1, 1, T, 1.0, order, 1, frames=False)
        assert r.nseg[0] == 1


# ------------------------------------------------------------ structural invariants ----
def _check_structure(st, T, P, order):
    r = oracle.reconstruct(st, 1, P, T, 1.0, order, 1, frames=False, segments=True)
    r1 = oracle.reconstruct(st, 1, P, T, 1.0, 1, 1, frames=False, segments=True)
    for p in range(P):
        s = oracle.spike_times(st, T, p)
        ts, te, n, v = r.segments(p)
        if len(s) < 2:
            assert len(ts) == 0
            continue
        x = np.diff(s)
        # tiling of (s_1, s_K], sums
        assert ts[0] == s[0] and te[-1] == s[-1]
        assert np.all(ts[1:] == te[:-1])
        assert n.sum() == len(s) - 1
        assert (te - ts).sum() == s[-1] - s[0]
        assert np.allclose(v, n / (te - ts), rtol=1e-15)
        idx = np.searchsorted(s, ts)
        for j in range(len(ts)):
            seg = x[idx[j]: idx[j] + n[j]]
            assert seg.sum() == te[j] - ts[j]
            assert seg.max() - seg.min() <= 1                        # Def. 2 zero order
            if order >= 2:
                a = seg.min()
                for val in (a, a + 1):                               # second order inside
                    pos = np.nonzero(seg == val)[0]
                    if len(pos) >= 3:
                        d = np.diff(pos)
                        assert d.max() - d.min() <= 1, (p, j)
        # FSR greedy maximality: the element after a sequence breaks the rule
        f_ts, f_te, f_n, _ = r1.segments(p)
        fidx = np.searchsorted(s, f_ts)
        for j in range(len(f_ts) - 1):
            seg = x[fidx[j]: fidx[j] + f_n[j] + 1]
            assert seg.max() - seg.min() > 1
        # SSR refines FSR
        assert set(f_te.tolist()) <= set(te.tolist())
    return r


@pytest.mark.parametrize("order", [1, 2])
def test_structure_moving_scene(order):
    w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=8, W=64, T=3000)
    st, _ = spkgen.make_stream(w)
    r = _check_structure(st, w.T, w.P, order)
    assert r.nseg.mean() > 5


def test_structure_random_streams():
    for seed in range(4):
        b = spkgen.random_bits(500, 64, 0.15 + 0.2 * seed, seed)
        _check_structure(spkgen.pack(b), 500, 64, 2)


# ------------------------------------------------------------------------ TFI case ----
def test_tfi_special_case():
    """Alternating intervals 2, 8, 2, 8, ... violate the rule at every step, so every
    sequence holds one interval and Eq. 4 reduces to TFI's theta / interval (Sec. II)."""
    s = [0]
    for i in range(40):
        s.append(s[-1] + (2 if i % 2 == 0 else 8))
    T = s[-1] + 3
    bits = np.zeros((T, 1), dtype=np.uint8)
    bits[s, 0] = 1
    st = spkgen.pack(bits)
    for order in (1, 2):
        r = oracle.reconstruct(st, 1, 1, T, 1.0, order, 1, frames=False, segments=True)
        ts, te, n, v = r.segments(0)
        assert np.all(n == 1)
        assert np.allclose(v, 1.0 / np.diff(s), rtol=0, atol=0)


# ---------------------------------------------------------------- golden, by hand ----
@pytest.mark.parametrize("case", load_golden(), ids=lambda c: c["name"])
def test_golden_cases(case):
    T = case["T"]
    bits = np.zeros((T, 3), dtype=np.uint8)
    for t in case["spikes"]:
        bits[t, 1] = 1          # the case sits in pixel 1 of 3 (neighbours stay silent)
    st = spkgen.pack(bits)
    r = oracle.reconstruct(st, 1, 3, T, 1.0, case["order"], case["stride"], segments=True)
    ts, te, n, v = r.segments(1)
    got = list(zip(ts.tolist(), te.tolist(), n.tolist()))
    assert got == case["segments"]
    # Eq. 4 as theta / mean interval: two fp64 roundings at most
    for (a, b, c), val in zip(case["segments"], v):
        assert math.isclose(val, c / (b - a), rel_tol=1e-15)
    if case["frames"] is not None:
        assert np.allclose(r.frames[:, 1], [float(f) for f in case["frames"]], rtol=1e-15, atol=0)
    # the literal reading agrees too
    assert [s[:3] for s in bf.segments(bits[:, 1].tolist(), case["order"])] == case["segments"]
    if case["frames"] is not None:
        assert bf.frames(bits[:, 1].tolist(), case["order"], case["stride"]) == case["frames"]


# -------------------------------------------------------------- literal Def. 2 check ----
@pytest.mark.parametrize("order", [1, 2])
def test_bruteforce_exhaustive_16_steps(order):
    T = 16
    P = 1 << T
    bits = ((np.arange(P)[None, :] >> np.arange(T)[:, None]) & 1).astype(np.uint8)
    r = oracle.reconstruct(spkgen.pack(bits), 1, P, T, 1.0, order, 1, frames=False,
                           segments=True)
    for p in range(P):
        exp = bf.segments(bits[:, p].tolist(), order)
        ts, te, n, _ = r.segments(p)
        assert list(zip(ts.tolist(), te.tolist(), n.tolist())) == [e[:3] for e in exp], p


@pytest.mark.parametrize("order", [1, 2])
def test_bruteforce_random_4x4x64(order):
    rng = np.random.default_rng(17)
    for seed in range(120):
        b = spkgen.random_bits(64, 16, rng.uniform(0.2, 0.9), 1000 + seed)
        stride = int(rng.integers(1, 6))
        r = oracle.reconstruct(spkgen.pack(b, 4, 4), 4, 4, 64, 1.0, order, stride, segments=True)
        for p in range(16):
            exp = bf.segments(b[:, p].tolist(), order)
            ts, te, n, v = r.segments(p)
            assert list(zip(ts.tolist(), te.tolist(), n.tolist())) == [e[:3] for e in exp]
            assert np.allclose(v, [float(e[3]) for e in exp], rtol=1e-15, atol=0)
            fr = bf.frames(b[:, p].tolist(), order, stride)
            assert np.allclose(r.frames[:, p], [float(f) for f in fr], rtol=1e-15, atol=0)


def test_ssr_changes_random_streams():
    """SSR must actually cut: on random streams it refines FSR for many pixels."""
    b = spkgen.random_bits(64, 1024, 0.5, 7)
    st = spkgen.pack(b)
    r1 = oracle.reconstruct(st, 1, 1024, 64, 1.0, 1, 1, frames=False)
    r2 = oracle.reconstruct(st, 1, 1024, 64, 1.0, 2, 1, frames=False)
    assert np.all(r2.nseg >= r1.nseg)
    assert (r2.nseg > r1.nseg).sum() > 100


def test_theta_scales_values():
    """Eq. 4's 255 is the threshold argument: values scale linearly with theta."""
    b = spkgen.random_bits(200, 32, 0.4, 8)
    st = spkgen.pack(b)
    r1 = oracle.reconstruct(st, 1, 32, 200, 1.0, 2, 3)
    r255 = oracle.reconstruct(st, 1, 32, 200, 255.0, 2, 3)
    assert np.allclose(r255.frames, 255.0 * r1.frames, rtol=1e-15)


# ----------------------------------------------------------------- TFI / TFP (Sec. II) ----
def test_tfi_tfp_against_literal_reading():
    for seed in range(40):
        b = spkgen.random_bits(80, 8, 0.05 + 0.02 * seed, 300 + seed)
        st = spkgen.pack(b)
        for stride in (1, 3):
            f = oracle.tfi(st, 1, 8, 80, 1.0, stride)
            for p in range(8):
                assert np.allclose(f[:, p], [float(v) for v in bf.tfi_frames(b[:, p].tolist(), stride)],
                                   rtol=1e-15, atol=0)
            for L in (1, 7, 32):
                g = oracle.tfp(st, 1, 8, 80, L, 1.0, stride)
                for p in range(8):
                    assert np.allclose(g[:, p], [float(v) for v in bf.tfp_frames(b[:, p].tolist(), L, stride)],
                                       rtol=1e-15, atol=0)


def test_tfi_is_fsr_of_single_intervals_and_tfp_tracks_rate():
    """TFI equals the FSR frames of a stream whose every interval breaks the rule; TFP of a
    constant intensity Q over a full window counts floor or ceil of L Q spikes (Eq. 2)."""
    s = [0]
    for i in range(30):
        s.append(s[-1] + (2 if i % 2 == 0 else 8))
    T = s[-1] + 5
    bits = np.zeros((T, 1), dtype=np.uint8)
    bits[s, 0] = 1
    st = spkgen.pack(bits)
    assert np.array_equal(oracle.tfi(st, 1, 1, T, 1.0, 1), oracle.reconstruct(st, 1, 1, T, 1.0, 1, 1).frames)
    rng = np.random.default_rng(21)
    Q = rng.uniform(0.05, 1.0, 64)
    q = np.broadcast_to(Q, (600, 64)).copy()
    st = spkgen.simulate_table(q, rng.uniform(0, 1, 64) * Q)
    for L in (32, 64):
        g = oracle.tfp(st, 1, 64, 600, L, 1.0, 1)[L:]
        cnt = np.rint(g * L)
        assert np.all((cnt >= np.floor(L * Q)) & (cnt <= np.ceil(L * Q)))


# ------------------------------------------------ general n-order tree (Fig. 1, Sec. III-B) ----
def _times(b, p):
    return np.flatnonzero(b[:, p]).astype(np.int32)


def _trip(segs):
    return [tuple(e[:3]) for e in segs]


def test_norder_general_code_is_fsr_and_ssr_at_orders_1_and_2():
    """The tree's code at n = 1 and 2 gives the FSR and SSR sequences of the specialised
    (separately pinned) oracle, and the literal tree gives the literal FSR and SSR."""
    rng = np.random.default_rng(3)
    for seed in range(60):
        T = int(rng.integers(20, 300))
        b = spkgen.random_bits(T, 8, rng.uniform(0.1, 0.9), 500 + seed)
        st = spkgen.pack(b)
        for n in (1, 2):
            r = oracle.reconstruct(st, 1, 8, T, 1.0, n, 1, frames=False, segments=True)
            for p in range(8):
                ts, te, nn, v = r.segments(p)
                got = oracle.segments_n(_times(b, p), n)
                assert _trip(got) == list(zip(ts.tolist(), te.tolist(), nn.tolist()))
                assert np.array_equal([g[3] for g in got], v)
                assert _trip(bf.segments_n(b[:, p].tolist(), n)) == _trip(bf.segments(b[:, p].tolist(), n))


def _third_order_streams(count, seed):
    """Streams whose S_2 has several stable sequences of its own: intervals 2 and 3 in
    patterns with changing spacings, so that the third level has something to cut."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        x = []
        while sum(x) < 400:
            gap = int(rng.integers(1, 5))          # occurrences of 3 spaced by 1..4 intervals of 2
            x += [2] * gap + [3]
            if rng.uniform() < 0.05:
                x.append(int(rng.integers(1, 7)))   # occasional FSR break
        s = np.concatenate([[int(rng.integers(0, 3))], np.cumsum(x) + 2])
        out.append(s[s < 420].astype(np.int32))
    return out


@pytest.mark.parametrize("n", [3, 4, 5])
def test_norder_matches_literal_tree(n):
    """C tree == set-based literal tree: on all 2^14 patterns of 14 steps, random streams,
    and streams built so that levels 3 and up do cut."""
    T = 14
    P = 1 << T
    bits = ((np.arange(P)[None, :] >> np.arange(T)[:, None]) & 1).astype(np.uint8)
    r = oracle.reconstruct(spkgen.pack(bits), 1, P, T, 1.0, n, 1, frames=False, segments=True)
    for p in range(0, P, 3):
        ts, te, nn, _ = r.segments(p)
        assert list(zip(ts.tolist(), te.tolist(), nn.tolist())) == _trip(bf.segments_n(bits[:, p].tolist(), n))
    differ = 0
    for s in _third_order_streams(40, 11 + n):
        T = int(s[-1]) + 1
        bits1 = np.zeros(T, dtype=np.uint8)
        bits1[s] = 1
        want = bf.segments_n(bits1.tolist(), n)
        got = oracle.segments_n(s, n)
        assert _trip(got) == _trip(want)
        assert np.allclose([g[3] for g in got], [float(w[3]) for w in want], rtol=1e-15, atol=0)
        differ += _trip(got) != _trip(oracle.segments_n(s, 2))
    assert differ >= 10            # the third level does cut these streams


def test_norder_constant_intensity_is_one_sequence():
    """Theorem 1 through the tree: by Lemma 2 every S_k of a constant intensity is the
    interval stream of an integrate-and-fire G_{k-1} with a constant rate, hence stable,
    so no level cuts: one sequence for every order."""
    rng = np.random.default_rng(9)
    Q = rng.uniform(0.03, 1.0, 128)
    T = 3000
    st = _const_stream(Q, rng.uniform(0, 1, 128) * Q, T)
    for n in (3, 4, 6):
        r = oracle.reconstruct(st, 1, 128, T, 1.0, n, 1, frames=False)
        assert np.all(r.nseg[r.K >= 2] == 1), n


def test_norder_refines_and_saturates():
    """Each level can only add cuts (the sequences of order n+1 refine those of order n), and
    past the depth at which every stream is empty nothing changes."""
    b = spkgen.random_bits(300, 256, 0.45, 77)
    st = spkgen.pack(b)
    prev = None
    for n in range(1, 9):
        r = oracle.reconstruct(st, 1, 256, 300, 1.0, n, 1, frames=False, segments=True)
        if prev is not None:
            for p in range(0, 256, 7):
                ends = set(r.segments(p)[1].tolist())
                assert set(prev.segments(p)[1].tolist()) <= ends
        prev = r
    r12 = oracle.reconstruct(st, 1, 256, 300, 1.0, 12, 1, frames=False)
    r32 = oracle.reconstruct(st, 1, 256, 300, 1.0, 32, 1, frames=False)
    assert np.array_equal(r12.nseg, r32.nseg)


def test_constant_span_is_tfp_over_that_span():
    """A pixel with one stable sequence (constant intensity): its value theta N / D is TFP
    with the window equal to the sequence, read at the sequence's last spike (the N spikes
    in (t_start, t_end] over D steps) -- the special case of Sec. II."""
    rng = np.random.default_rng(31)
    Q = rng.uniform(0.1, 1.0, 64)
    T = 60
    st = _const_stream(Q, rng.uniform(0, 1, 64) * Q, T)
    r = oracle.reconstruct(st, 1, 64, T, 1.0, 2, 1, frames=False, segments=True)
    checked = 0
    for p in range(64):
        if r.nseg[p] != 1:
            continue
        ts, te, n, v = (a[0] for a in r.segments(p))
        D = int(te - ts)
        if D > 64:
            continue
        f = oracle.tfp(st, 1, 64, T, D, 1.0, 1, pixels=[p])
        assert f[int(te), 0] == pytest.approx(float(v), rel=1e-15)
        assert v == pytest.approx(n / D, rel=1e-15)
        checked += 1
    assert checked > 40


# ------------------------------------------------------------ 8-bit frames, edge policy ----
def test_u8_is_round_half_up_of_the_exact_ratio():
    """The 8-bit value of a sequence (the decoder's 8-bit output, Sec. III-C; Eq. 4 with
    its 8-bit scale): theta * N / D rounded half up and clamped to 255, checked against
    exact rationals, ties included."""
    from fractions import Fraction
    rng = np.random.default_rng(17)
    cases = [(255, 1, 2), (255, 3, 7), (1, 1, 2), (1, 3, 2), (2, 5, 4), (255, 20, 2), (7, 9, 14)]
    cases += [(int(t), int(n), int(d)) for t, n, d in zip(rng.choice([1, 2, 7, 255, 1000], 3000),
                                                          rng.integers(1, 5000, 3000), rng.integers(1, 20000, 3000))]
    for theta, N, D in cases:
        want = min(255, int((Fraction(theta * N, D) + Fraction(1, 2)) // 1))
        assert oracle.u8(theta, N, D) == want, (theta, N, D)
    assert oracle.u8(1, 1, 2) == 1 and oracle.u8(1, 1, 3) == 0 and oracle.u8(3, 1, 2) == 2   # ties round up


@pytest.mark.parametrize("order", [1, 2, 3])
def test_u8_frames_are_the_covering_sequences_u8(order):
    w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=6, W=30, T=1500)
    st, _ = spkgen.make_stream(w)
    for theta in (255, 1):
        r = oracle.reconstruct(st, w.H, w.W, w.T, float(theta), order, w.stride, segments=True)
        u = oracle.reconstruct(st, w.H, w.W, w.T, float(theta), order, w.stride, u8=True)
        f, g = r.frames, u.frames
        assert np.all(g == np.round(g)) and g.min() >= 0 and g.max() <= 255
        ok = f <= 255.5
        assert np.all(np.abs(g[ok] - f[ok]) <= 0.5 + 1e-9)        # the nearest integer
        assert np.all(g[~ok] == 255)
        for p in range(w.P):                                    # and exactly the sequence's u8
            ts, te, n, _ = r.segments(p)
            vals = {oracle.u8(theta, int(a), int(b) - int(c)) for a, b, c in zip(n, te, ts)}
            assert set(np.unique(g[:, p])) <= vals | {0.0}


@pytest.mark.parametrize("order", [1, 2, 4])
def test_edge_policies_zero_only_the_edges(order):
    """ZERO_HEAD makes the frames up to the first spike 0, ZERO_TAIL those after the last
    spike; every other frame keeps its value (the frame policy of A4, with the edges off)."""
    w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=5, W=40, T=1200)
    st, _ = spkgen.make_stream(w)
    bits = np.zeros((w.T, w.P), dtype=np.uint8)
    bits[100:900:7, :] = 1                         # every pixel: spikes from 100 to 897 only
    st2 = spkgen.pack(bits, w.H, w.W)
    for s in (st, st2):
        base = oracle.reconstruct(s, w.H, w.W, w.T, 1.0, order, 3).frames
        tk = np.arange(base.shape[0])[:, None] * 3
        s1 = np.array([oracle.spike_times(s, w.T, p)[0] for p in range(w.P)])[None, :]
        sK = np.array([oracle.spike_times(s, w.T, p)[-1] for p in range(w.P)])[None, :]
        for edges in (oracle.ZERO_HEAD, oracle.ZERO_TAIL, oracle.ZERO_HEAD | oracle.ZERO_TAIL):
            f = oracle.reconstruct(s, w.H, w.W, w.T, 1.0, order, 3, edges=edges).frames
            zero = np.zeros_like(base, dtype=bool)
            if edges & oracle.ZERO_HEAD:
                zero |= tk <= s1
            if edges & oracle.ZERO_TAIL:
                zero |= tk > sK
            assert np.all(f[zero] == 0) and np.array_equal(f[~zero], base[~zero])
        if s is st2:
            assert (tk <= s1).any() and (tk > sK).any()
        t0 = oracle.tfi(s, w.H, w.W, w.T, 1.0, 3)
        t1 = oracle.tfi(s, w.H, w.W, w.T, 1.0, 3, edges=oracle.ZERO_HEAD | oracle.ZERO_TAIL)
        zero = (tk <= s1) | (tk > sK)
        assert np.all(t1[zero] == 0) and np.array_equal(t1[~zero], t0[~zero])
