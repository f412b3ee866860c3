"""ORACLE (test infrastructure only): a literal, set-based reading of Def. 2 for tiny inputs.

Independent of ``oracle.c``: instead of running min/max registers it re-tests the
zero-order rule on explicit Python sets, builds every interval stream S_1, S_2 as an
explicit list, and finds each stable sequence as the longest stable prefix (O(n^2)).

* Def. 2 (Sec. III-A): a sequence is zero-order stable when it holds one value, or two
  values whose difference is 1.
* FSR (Sec. III-B): S_1 is broken where the zero-order rule would be violated; the
  violating element opens the next stable sequence (Sec. III-C).
* SSR (Sec. III-B, Fig. 1): inside every FSR sequence, S_2 is the interval stream of S_1
  for the '-' firing value (the smaller one) and for the '+' firing value (the larger
  one); each S_2 is broken by the same rule, and every break of S_2 becomes a break of
  S_1 placed after the S_1 element at which the violating S_2 interval starts.
* Eq. 4: intensity = theta / mean interval of the stable sequence.
"""
from __future__ import annotations

from fractions import Fraction


def zero_order_stable(seq) -> bool:
    """Def. 2: one distinct value, or two distinct values differing by exactly 1."""
    s = set(seq)
    return len(s) == 1 or (len(s) == 2 and max(s) - min(s) == 1)


def greedy_stable_sequences(seq):
    """Split seq into consecutive longest stable prefixes; returns [(i0, i1)] inclusive."""
    out = []
    i0 = 0
    while i0 < len(seq):
        i1 = i0
        while i1 + 1 < len(seq) and zero_order_stable(seq[i0:i1 + 2]):
            i1 += 1
        out.append((i0, i1))
        i0 = i1 + 1
    return out


def interval_stream(seq, firing):
    """Positions of `firing` in seq and the distances between consecutive ones (Def. 2)."""
    pos = [i for i, v in enumerate(seq) if v == firing]
    return pos, [pos[j + 1] - pos[j] for j in range(len(pos) - 1)]


def spike_times(bits):
    return [n for n, b in enumerate(bits) if b]


def segments(bits, order: int = 1, theta=1):
    """Stable sequences of one pixel's 0/1 list: [(t_start, t_end, N, value)] (value exact)."""
    s = spike_times(bits)
    if len(s) < 2:
        return []
    x = [s[i + 1] - s[i] for i in range(len(s) - 1)]  # S_1
    ends = set()                                       # S_1 indices that close a sequence
    for (i0, i1) in greedy_stable_sequences(x):
        ends.add(i1)
        if order >= 2:
            seq = x[i0:i1 + 1]
            a = min(seq)
            for v in (a, a + 1):                       # '-' then '+'
                pos, d = interval_stream(seq, v)
                for (j0, _j1) in greedy_stable_sequences(d)[1:]:
                    ends.add(i0 + pos[j0])             # d_j0 starts after element pos[j0]
    out = []
    i0 = 0
    for i in sorted(ends):
        N = i - i0 + 1
        ts, te = s[i0], s[i + 1]
        out.append((ts, te, N, Fraction(theta) * N / (te - ts)))
        i0 = i + 1
    return out


def frames(bits, order: int = 1, stride: int = 1, theta=1):
    """Frame k samples t_k = k*stride: covering sequence's value, head fill / tail hold."""
    T = len(bits)
    segs = segments(bits, order, theta)
    T_out = (T + stride - 1) // stride
    out = []
    for k in range(T_out):
        t = k * stride
        if not segs:
            out.append(Fraction(0))
            continue
        if t <= segs[0][0]:
            out.append(segs[0][3])
            continue
        if t > segs[-1][1]:
            out.append(segs[-1][3])
            continue
        out.append(next(v for (ts, te, _n, v) in segs if ts < t <= te))
    return out


def tfi_frames(bits, stride: int = 1, theta=1):
    """TFI (Sec. II): theta over the interval between the two adjacent spikes around t_k."""
    s = spike_times(bits)
    T = len(bits)
    out = []
    for k in range((T + stride - 1) // stride):
        t = k * stride
        if len(s) < 2:
            out.append(Fraction(0))
            continue
        # the interval (s_j, s_j+1] holding t; clamp to the first / last interval
        j = next((j for j in range(len(s) - 1) if s[j] < t <= s[j + 1]), None)
        if j is None:
            j = 0 if t <= s[0] else len(s) - 2
        out.append(Fraction(theta) / (s[j + 1] - s[j]))
    return out


def tfp_frames(bits, window: int, stride: int = 1, theta=1):
    """TFP (Sec. II): theta * spikes in the `window` steps ending at t_k / window."""
    T = len(bits)
    return [Fraction(theta) * sum(bits[u] for u in range(max(0, k * stride - window + 1), k * stride + 1))
            / window for k in range((T + stride - 1) // stride)]


def _ends_n(seq, depth: int, n: int):
    """Cut positions ('a cut after element i') of a level-`depth` stream under the n-order
    tree: its own greedy stable sequences, and, below level n, the cuts its two sub-streams
    ('-' = the smaller value, '+' = the larger, inside each of its stable sequences) send up,
    each placed after the element at which the breaking sub-stream element ends."""
    ends = set()
    for (i0, i1) in greedy_stable_sequences(seq):
        ends.add(i1)
        if depth < n:
            part = seq[i0:i1 + 1]
            a = min(part)
            for v in (a, a + 1):
                pos, d = interval_stream(part, v)
                if len(d) < 2:
                    continue
                for e in _ends_n(d, depth + 1, n):
                    if e < len(d) - 1:
                        ends.add(i0 + pos[e + 1])
    return ends


def segments_n(bits, n: int, theta=1):
    """segments() under the general n-order tree (Fig. 1 caption, Sec. III-B)."""
    s = spike_times(bits)
    if len(s) < 2:
        return []
    x = [s[i + 1] - s[i] for i in range(len(s) - 1)]
    out, i0 = [], 0
    for i in sorted(_ends_n(x, 1, n)):
        N = i - i0 + 1
        ts, te = s[i0], s[i + 1]
        out.append((ts, te, N, Fraction(theta) * N / (te - ts)))
        i0 = i + 1
    return out
