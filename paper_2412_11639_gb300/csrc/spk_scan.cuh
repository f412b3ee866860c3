// Per-pixel online stability scan (FSR / SSR, Sec. III-B) -- device code.
//
// One instance follows one pixel through time, one spike at a time, and reports every
// final stable sequence, in time order, to a sink: sink(t_start, t_end, N).
//
// S_1 (Def. 2, Eq. 5) is never stored: each new spike yields one interval x = t - t_prev.
//
// FSR (order 1).  The open sequence keeps the range [lo, hi] of its intervals; an
// interval that would widen it beyond 1 (Def. 2's zero-order rule) closes the sequence at
// the spike where that interval starts and opens the next one with it (Sec. III-C).
//
// SSR (order 2).  Inside the open FSR sequence there are at most two values: v0 (the
// first) and v1 (= v0 +- 1, once seen).  Each value is one of the two second-order
// streams of Fig. 1 ('-' for the smaller, '+' for the larger): its S_2 elements are the
// index distances d between consecutive occurrences.  Each branch keeps the range
// [dlo, dhi] of its open S_2 sequence (dlo = 0 while it has no distance yet) and the
// index q and end time tq of its last occurrence.  A distance that breaks the rule cuts
// S_1 after element q, i.e. at time tq, and restarts [dlo, dhi] with it.  The cut lies
// in the past, so it is held as pending until no earlier cut can still appear: a later
// cut from a branch can only fall at or after that branch's tq (if it has a distance)
// and an FSR cut only at or after the latest spike.  Cuts at or before
//   S = min(t_latest, tq of every branch with a distance)
// are final.  At most one cut stays pending after each step (a branch can run ahead of
// the other only through a distance of 1); two slots hold the momentary pair.
//
// The hierarchy reading: SSR refines FSR sequences (the cuts of both branches are
// united, the branches are independent, and an FSR cut resets both).
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define SPK_DEV __device__ __forceinline__
#else
#define SPK_DEV inline
#endif

namespace spk {

template <int ORDER>
struct PixelScan {
    int last_t;   // latest spike time, -1 before the first spike
    int nint;     // intervals seen so far (index of the next S_1 element)
    int v0, v1;   // order 1: [lo, hi]; order 2: first value and the other value (0: none)
    int c_t, c_i; // last final cut: its spike time and the index of the interval before it
    // order 2 only
    int q0, tq0, dlo0, dhi0;
    int q1, tq1, dlo1, dhi1;
    int pa_t, pa_i, pb_t, pb_i;  // pending cuts, pa before pb; time -1 = empty
    int err;                      // set if the pending list would overflow (never expected)

    SPK_DEV void init() {
        last_t = -1;
        nint = 0;
        v0 = v1 = 0;
        c_t = c_i = 0;
        q0 = tq0 = dlo0 = dhi0 = 0;
        q1 = tq1 = dlo1 = dhi1 = 0;
        pa_t = pb_t = -1;
        pa_i = pb_i = 0;
        err = 0;
    }

    template <class Sink>
    SPK_DEV void cut(int ct, int ci, Sink &sink) {
        sink(c_t, ct, ci - c_i);
        c_t = ct;
        c_i = ci;
    }

    SPK_DEV void open_fsr(int x, int i, int t) {
        v0 = x;
        v1 = 0;
        q0 = i;
        tq0 = t;
        dlo0 = 0;
        dlo1 = 0;
    }

    SPK_DEV void add_pending(int ct, int ci) {
        if (pa_t < 0) {
            pa_t = ct;
            pa_i = ci;
        } else if (pb_t < 0) {
            if (ct < pa_t) {
                pb_t = pa_t;
                pb_i = pa_i;
                pa_t = ct;
                pa_i = ci;
            } else {
                pb_t = ct;
                pb_i = ci;
            }
        } else {
            err = 1;
        }
    }

    template <class Sink>
    SPK_DEV void settle(Sink &sink) {
        int S = last_t;
        if (dlo0 != 0) S = min(S, tq0);
        if (dlo1 != 0) S = min(S, tq1);
        if (pa_t >= 0 && pa_t <= S) {
            cut(pa_t, pa_i, sink);
            pa_t = pb_t;
            pa_i = pb_i;
            pb_t = -1;
            if (pa_t >= 0 && pa_t <= S) {
                cut(pa_t, pa_i, sink);
                pa_t = -1;
            }
        }
    }

    template <class Sink>
    SPK_DEV void flush_pending(Sink &sink) {
        if (pa_t >= 0) cut(pa_t, pa_i, sink);
        if (pb_t >= 0) cut(pb_t, pb_i, sink);
        pa_t = pb_t = -1;
    }

    // The first spike of the stream opens the first sequence (no interval yet).
    SPK_DEV void first_spike(int t) {
        last_t = t;
        c_t = t;
        c_i = -1;
        v0 = ORDER == 1 ? (1 << 30) : 0;   // order 1: empty range [lo, hi] = [2^30, -2^30]
        v1 = ORDER == 1 ? -(1 << 30) : 0;
    }

    // Every later spike t > last_t.  The common case -- the interval continues the open
    // sequence and no S_2 distance breaks -- takes no data-dependent branch except the
    // rarely taken exits, so the lanes of a warp stay converged.
    template <class Sink>
    SPK_DEV void spike(int t, Sink &sink) {
        const int x = t - last_t;
        const int i = nint;
        if (ORDER == 1) {
            const int lo = min(v0, x), hi = max(v1, x);
            if (hi - lo > 1) {  // FSR break: the sequence ends at spike last_t
                cut(last_t, i - 1, sink);
                v0 = v1 = x;
            } else {
                v0 = lo;
                v1 = hi;
            }
            nint = i + 1;
            last_t = t;
            return;
        } else {
            const bool b1 = (x == v1);
            if (!(b1 || x == v0)) {
                rare(t, x, sink);
                return;
            }
            nint = i + 1;
            last_t = t;
            // one S_2 step of the branch of value x
            const int q = b1 ? q1 : q0, tq = b1 ? tq1 : tq0;
            const int lo = b1 ? dlo1 : dlo0, hi = b1 ? dhi1 : dhi0;
            const int d = i - q;
            const int nlo = min(lo, d), nhi = max(hi, d);
            const bool restart = (lo == 0) || (nhi - nlo > 1);
            const int wlo = restart ? d : nlo, whi = restart ? d : nhi;
            if (lo != 0 && nhi - nlo > 1) add_pending(tq, q);  // S_2 breaks: cut after q
            if (b1) {
                q1 = i;
                tq1 = t;
                dlo1 = wlo;
                dhi1 = whi;
            } else {
                q0 = i;
                tq0 = t;
                dlo0 = wlo;
                dhi0 = whi;
            }
            if (pa_t >= 0) settle(sink);
        }
    }

    // order 2, an interval outside {v0, v1}: the first interval, the first occurrence of
    // the second value, or an FSR break
    template <class Sink>
    SPK_DEV void rare(int t, int x, Sink &sink) {
        const int i = nint++;
        const int prev = last_t;
        last_t = t;
        if (v0 != 0 && v1 == 0 && (x == v0 + 1 || x == v0 - 1)) {
            v1 = x;  // first occurrence of the second value: no distance yet
            q1 = i;
            tq1 = t;
            dlo1 = 0;
            if (pa_t >= 0) settle(sink);
            return;
        }
        if (v0 != 0) {  // FSR break: the open sequence ends with interval i-1, at spike prev
            flush_pending(sink);
            cut(prev, i - 1, sink);
        }
        open_fsr(x, i, t);
    }

    // end of the stream: everything still open is final
    template <class Sink>
    SPK_DEV void finish(Sink &sink) {
        if (nint >= 1) {
            if (ORDER >= 2) flush_pending(sink);
            cut(last_t, nint - 1, sink);
        }
    }
};

}  // namespace spk
