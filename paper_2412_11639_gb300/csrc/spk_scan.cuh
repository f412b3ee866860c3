// Per-pixel online stability scan (FSR / SSR, Sec. III-B; the TFI baseline of Sec. II as
// ORDER 3, where every interval is its own span) -- device code.
//
// One instance follows one pixel through time, one spike at a time.  Every cut of S_1 it
// finds is handed to a sink as a candidate sink.cand(t_cut, i_cut): the spike time at
// which one stable sequence ends and the next begins, and the index of the last S_1
// element before it.  Stable sequences are the spans between consecutive cuts, starting
// at the first spike (t0, index -1) and ending at the last spike.
//
// S_1 (Def. 2, Eq. 5) is never stored: each new spike yields one interval x = t - t_prev.
//
// FSR (order 1).  The open sequence keeps the range [lo, hi] of its intervals; an
// interval that would widen it beyond 1 (Def. 2's zero-order rule) cuts at the spike
// where that interval starts and opens the next sequence with it (Sec. III-C).
//
// SSR (order 2).  Inside the open FSR sequence there are at most two values: v0 (the
// first) and v1 (= v0 +- 1, once seen).  Each value is one of the two second-order
// streams of Fig. 1 ('-' for the smaller, '+' for the larger): its S_2 elements are the
// index distances d between consecutive occurrences.  Each branch keeps the range
// [dlo, dhi] of its open S_2 sequence (dlo = 0 while it has no distance yet) and the
// index q and end time tq of its last occurrence.  A distance that breaks the rule cuts
// S_1 after element q, i.e. at time tq, and restarts [dlo, dhi] with it.  The hierarchy
// reading: SSR refines FSR sequences (the cuts of both branches are united, the branches
// are independent, and an FSR cut resets both).
//
// Order of candidates.  An S_2 cut lies in the past, so candidates can arrive out of
// time order, but by one place at most: a branch can run ahead of the other only through
// a distance of 1, which breaks its S_2 at most once before the other branch's next
// occurrence.  A candidate is final once no earlier cut can still appear; later cuts of a
// branch fall at or after its tq (if it has a distance) and FSR cuts at or after the
// latest spike, so every cut at or before
//   S = min(t_latest, tq of each branch with a distance)      (frontier())
// is final.  Sinks keep candidates sorted (one swap) and consume only final ones.
//
// The common step takes no data-dependent branch except the one that hands a candidate
// to the sink, so the 32 lanes of a warp stay converged.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define SPK_DEV __device__ __forceinline__
#else
#define SPK_DEV inline
#endif

namespace spk {

constexpr int NO_VALUE = -100;  // v0 before the first interval: never equals an interval

template <int ORDER>
struct PixelScan {
    int last_t;   // latest spike time, -1 before the first spike
    int nint;     // intervals seen so far (index of the next S_1 element)
    int v0, v1;   // order 1: [lo, hi]; order 2: first value and the other value (0: none)
    // order 2 only: the two S_2 branches
    int q0, tq0, dlo0, dhi0;
    int q1, tq1, dlo1, dhi1;

    SPK_DEV void init() {
        last_t = -1;
        nint = 0;
        v0 = v1 = 0;
        q0 = tq0 = dlo0 = dhi0 = 0;
        q1 = tq1 = dlo1 = dhi1 = 0;
    }

    // The stream's first spike opens the first sequence (no interval yet).
    SPK_DEV void first_spike(int t) {
        last_t = t;
        v0 = ORDER == 1 ? (1 << 30) : NO_VALUE;  // order 1: empty range [2^30, -2^30]
        v1 = ORDER == 1 ? -(1 << 30) : 0;
    }

    // Cuts at or before the frontier are final.
    SPK_DEV int frontier() const {
        int S = last_t;
        if (ORDER >= 2) {
            if (dlo0 != 0) S = min(S, tq0);
            if (dlo1 != 0) S = min(S, tq1);
        }
        return S;
    }

    // Every later spike t > last_t.
    template <class Sink>
    SPK_DEV void spike(int t, Sink &sink) {
        const int x = t - last_t;
        const int i = nint;
        if (ORDER == 3) {  // TFI (Sec. II): every interval is its own span
            if (i > 0) sink.cand(last_t, i - 1);
        } else if (ORDER == 1) {
            const int lo = min(v0, x), hi = max(v1, x);
            const bool brk = hi - lo > 1;
            if (brk) sink.cand(last_t, i - 1);  // the sequence ends at spike last_t
            v0 = brk ? x : lo;
            v1 = brk ? x : hi;
        } else {
            const bool isv0 = (x == v0), isv1 = (x == v1);
            const int dv = x - v0;
            const bool nv1 = (v1 == 0) && (dv == 1 || dv == -1);  // second value appears
            const bool brk = !(isv0 || isv1 || nv1);                 // FSR break (or first)
            // one S_2 step of the branch of value x
            const int q = isv1 ? q1 : q0, tq = isv1 ? tq1 : tq0;
            const int lo = isv1 ? dlo1 : dlo0, hi = isv1 ? dhi1 : dhi0;
            const int d = i - q;
            const int nlo = min(lo, d), nhi = max(hi, d);
            const bool wide = nhi - nlo > 1;
            const bool viol = (isv0 || isv1) && lo != 0 && wide;  // S_2 breaks before d
            const bool rst = lo == 0 || wide;
            const int wlo = rst ? d : nlo, whi = rst ? d : nhi;
            if (viol || (brk && v0 > 0))  // S_2 cut after q, or FSR cut at the previous spike
                sink.cand(viol ? tq : last_t, viol ? q : i - 1);
            const bool u0 = isv0 || brk, u1 = isv1 || nv1;
            q0 = u0 ? i : q0;
            tq0 = u0 ? t : tq0;
            dlo0 = brk ? 0 : (isv0 ? wlo : dlo0);
            dhi0 = isv0 ? whi : dhi0;
            q1 = u1 ? i : q1;
            tq1 = u1 ? t : tq1;
            dlo1 = (brk || nv1) ? 0 : (isv1 ? wlo : dlo1);
            dhi1 = isv1 ? whi : dhi1;
            v1 = nv1 ? x : (brk ? 0 : v1);
            v0 = brk ? x : v0;
        }
        nint = i + 1;
        last_t = t;
    }

    // 32 spikes at steps base .. base+31 (an all-ones time word).  If the pixel is in the
    // steady state those spikes cannot cut -- its previous interval was 1, value 1
    // already belongs to the open FSR sequence and its S_2 branch holds the distance 1
    // (or has no distance yet) -- they are absorbed in O(1) and true is returned: 32
    // intervals of 1, each an S_2 distance of 1.  Otherwise nothing changes.
    SPK_DEV bool absorb_ones(int base) {
        if (ORDER == 3 || last_t != base - 1) return false;
        if (ORDER == 1) {
            if (v0 != 1) return false;  // [lo, hi] = [1, 1 or 2] already holds 1
        } else {
            const int last = nint - 1;
            if (v0 == 1 && q0 == last && dlo0 <= 1) {
                q0 = last + 32;
                tq0 = base + 31;
                if (dlo0 == 0) dlo0 = dhi0 = 1;
            } else if (v1 == 1 && q1 == last && dlo1 <= 1) {
                q1 = last + 32;
                tq1 = base + 31;
                if (dlo1 == 0) dlo1 = dhi1 = 1;
            } else {
                return false;
            }
        }
        nint += 32;
        last_t = base + 31;
        return true;
    }

    // end of the stream: the last sequence ends at the last spike
    template <class Sink>
    SPK_DEV void finish(Sink &sink) {
        if (nint >= 1) sink.cand(last_t, nint - 1);
    }
};

}  // namespace spk
