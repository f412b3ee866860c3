// Per-pixel online stability scan (FSR / SSR, Sec. III-B; the TFI baseline of Sec. II as
// ORDER 3, where every interval is its own span) -- device code.
//
// One instance follows one pixel through time, one spike at a time.  Every cut of S_1 it
// finds is handed to a sink as a candidate (t_cut, i_cut): the spike time at which one
// stable sequence ends and the next begins, and the index of the last S_1 element before
// it.  An SSR (or TFI) spike hands its outcome over as sink.put(emit, t_cut, i_cut),
// whether or not it cuts (the sink keeps the pair only if emit), so that the step has no
// branch; the caller makes room for one record before each such spike.  FSR spikes, which
// cut rarely, and the end of the stream call sink.cand(t_cut, i_cut) only for a cut.
// Stable sequences are the spans between consecutive cuts, starting at the first spike
// (t0, index -1) and ending at the last spike.
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
// branch fall at or after its tq (if it has a distance; branch 1 only while the second
// value is set) and FSR cuts at or after the latest spike, so every cut at or before
//   S = min(t_latest, tq of each branch with a distance)      (frontier())
// is final.  Sinks keep candidates sorted (one swap) and consume only final ones.
//
// The SSR step takes no data-dependent branch, so the 32 lanes of a warp stay converged
// and the loop body over a word's spikes is one straight-line block.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define SPK_DEV __device__ __forceinline__
#else
#define SPK_DEV inline
#include <algorithm>
#endif

namespace spk {
#if !defined(__CUDACC__)
using std::max;  // host builds of this header (the scan's CPU check in tests/c)
using std::min;
#endif

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
            if (dlo1 != 0 && v1 != 0) S = min(S, tq1);  // branch 1 exists only with v1
        }
        return S;
    }

    // Every later spike t > last_t.
    template <class Sink>
    SPK_DEV void spike(int t, Sink &sink) {
        const int x = t - last_t;
        const int i = nint;
        if (ORDER == 3) {  // TFI (Sec. II): every interval is its own span
            sink.put(i > 0, last_t, i - 1);
        } else if (ORDER == 1) {
            const int lo = min(v0, x), hi = max(v1, x);
            const bool brk = hi - lo > 1;
            // the sequence ends at spike last_t (rare: FSR keeps the branch, which measured
            // faster than the predicated hand-off of SSR for this lighter step)
            if (brk) sink.cand(last_t, i - 1);
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
            // S_2 cut after q, or FSR cut at the previous spike
            sink.put(viol || (brk && v0 > 0), viol ? tq : last_t, viol ? q : i - 1);
            // the branch this element belongs to takes (i, t, range); an opening element (FSR
            // break: branch 0; the other value's first occurrence: branch 1) has no distance
            const bool u0 = isv0 || brk, u1 = isv1 || nv1;
            const int nlo0 = (brk || nv1) ? 0 : wlo;
            q0 = u0 ? i : q0;
            tq0 = u0 ? t : tq0;
            dlo0 = u0 ? nlo0 : dlo0;
            dhi0 = u0 ? whi : dhi0;
            q1 = u1 ? i : q1;
            tq1 = u1 ? t : tq1;
            dlo1 = u1 ? nlo0 : dlo1;  // (left as is by an FSR break: unused until v1 is set)
            dhi1 = u1 ? whi : dhi1;
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

// General n-order stability (the tree in the caption of Fig. 1, Sec. III-B), orders 3..5.
//
// Every stream of the tree is segmented online by the same greedy zero-order rule as
// S_1: node 0 is S_1, and the children of node k are the '-' and '+' streams of the
// values of its open stable sequence (heap order: 2k + 1 for the sequence's first value,
// 2k + 2 for the other one), whose elements are the index distances between consecutive
// occurrences of that value inside the sequence.  Every element carries the cut "after
// this element" expressed on S_1 -- (spike time, S_1 index) of the S_1 element at which
// it ends -- so that a node whose new element breaks its sequence emits the cut of its
// previous element, and a break of a node ends (resets) the sequences of all its
// descendants.  The levels stop at the order n.
//
// Cuts of deep nodes lie arbitrarily far in the past, so they wait, sorted and without
// duplicates, in a per-pixel list until they are final: a node can only emit the cut of
// its latest element, so every cut at or before the minimum of those over the nodes with
// an open sequence (frontier()) is final and goes to the sink in order.  The list is a
// ring of pcap entries (a power of two) in storage the caller provides, entry j of slot s
// at pt[s * ps], pi[s * ps]; a push that finds it full sets bad bit 2 (the caller runs the
// pixel again with a larger ring), an ordering fault bad bit 1.
// The walk down the tree runs one block of code per LEVEL, not per node: a lane's node on
// level L is r (0 .. 2^(L-1) - 1, heap index 2^(L-1) - 1 + r) and its state is gathered
// from and scattered back to the level's nodes, so the lanes of a warp stay converged
// whichever branches their elements take, and the code stays small.  The first RL levels
// are indexed by constants only (select chains), so their state lives in registers; deeper
// levels are indexed by r (per-thread local memory), for trees too large for registers.
constexpr int TREE_MIN = 3, TREE_MAX = 5;  // orders of the tree (1 and 2 are PixelScan)
constexpr int TREE_BAD_ORDER = 1;
constexpr int TREE_BAD_FULL = 2;

template <int N, int RL>
struct TreeScan {
    static_assert(N >= TREE_MIN && N <= TREE_MAX && RL >= 1 && RL <= N, "tree order");
    static constexpr int NODES = (1 << N) - 1;
    static constexpr int TOPN = (1 << RL) - 1;                          // nodes in registers
    static constexpr int DEEPN = NODES > TOPN ? NODES - TOPN : 1;        // nodes in local memory
    // per-node fields
    enum { CNT,   // elements in the node's open sequence (0: none)
           V0,    // its first value
           V1,    // the other value (0: none yet)
           Q0,    // last occurrence (node element index) of V0, -1: none
           Q1,    // last occurrence of V1, -1: none
           JN,    // next element index of the node's stream
           PCT,   // cut after the node's latest element: spike time ...
           PCI,   // ... and S_1 index
           NF };
    int top[NF][TOPN];          // levels 1 .. RL, heap order
    int *deep;                  // levels RL+1 .. N: [NF][DEEPN] in the caller's per-thread
                                // storage (kept out of this object, so that the object's
                                // constant-indexed state is promoted to registers)
    int last_t, nint;           // S_1 bookkeeping, as in PixelScan
    int *pt, *pi;               // pending cuts, increasing t: a ring in the caller's storage
    int ps, pcap;               // its slot stride and capacity (a power of two)
    int ph, np;                 // first slot and number of pending cuts
    int thead, tlast;           // times of the first and the last pending cut (np > 0)
    int rel_t;                  // last cut handed to the sink
    int bad;                    // TREE_BAD_FULL: the ring was too small; TREE_BAD_ORDER: a cut arrived behind the frontier

    // field F of node r on level L
    template <int L, int F>
    SPK_DEV int get(int r) const {
        constexpr int B = (1 << (L - 1)) - 1, M = 1 << (L - 1);
        if constexpr (L > RL) {
            return deep[F * DEEPN + B - TOPN + r];
        } else if constexpr (M == 1) {
            return top[F][B];
        } else {
            int v = top[F][B];
#pragma unroll
            for (int i = 1; i < M; ++i) v = r == i ? top[F][B + i] : v;
            return v;
        }
    }
    template <int L, int F>
    SPK_DEV void put(int r, int v) {
        constexpr int B = (1 << (L - 1)) - 1, M = 1 << (L - 1);
        if constexpr (L > RL) {
            deep[F * DEEPN + B - TOPN + r] = v;
        } else if constexpr (M == 1) {
            top[F][B] = v;
        } else {
#pragma unroll
            for (int i = 0; i < M; ++i)
                if (r == i) top[F][B + i] = v;
        }
    }

    SPK_DEV void init(int *deep_store, int *pend_t, int *pend_i, int stride, int cap) {
        last_t = -1;
        nint = 0;
#pragma unroll
        for (int k = 0; k < TOPN; ++k) {
#pragma unroll
            for (int f = 0; f < NF; ++f) top[f][k] = 0;
            top[Q0][k] = top[Q1][k] = -1;
        }
        deep = deep_store;
        if constexpr (NODES > TOPN)
            for (int k = 0; k < DEEPN; ++k) {
                for (int f = 0; f < NF; ++f) deep[f * DEEPN + k] = 0;
                deep[Q0 * DEEPN + k] = deep[Q1 * DEEPN + k] = -1;
            }
        pt = pend_t;
        pi = pend_i;
        ps = stride;
        pcap = cap;
        ph = np = 0;
        thead = tlast = 0;
        rel_t = -1;
        bad = 0;
    }
    SPK_DEV int64_t slot(int j) const {  // storage index of the j-th pending cut
        return static_cast<int64_t>((ph + j) & (pcap - 1)) * ps;
    }
    SPK_DEV void first_spike(int t) { last_t = t; }

    // 32 spikes at steps base .. base+31 (an all-ones time word): 32 intervals of 1.  If the
    // path of value 1 is steady -- every node on it already holds 1 in its open sequence
    // and (above the last level) its previous element was a 1 as well, so that each of the
    // 32 elements sends a distance of 1 one level down -- no node can break, and the word
    // is absorbed in O(levels).  Otherwise nothing changes and false is returned.
    template <int L>
    SPK_DEV bool ones_steady(int r) const {
        const int a0 = get<L, V0>(r);
        if (get<L, CNT>(r) == 0 || (a0 != 1 && get<L, V1>(r) != 1)) return false;
        if constexpr (L < N) {
            const int b = a0 == 1 ? 0 : 1;
            if ((b ? get<L, Q1>(r) : get<L, Q0>(r)) != get<L, JN>(r) - 1) return false;
            return ones_steady<L + 1>(2 * r + b);
        } else {
            return true;
        }
    }
    template <int L>
    SPK_DEV void ones_take(int r, int base) {
        put<L, CNT>(r, get<L, CNT>(r) + 32);
        put<L, PCT>(r, base + 31);
        put<L, PCI>(r, nint + 31);
        if constexpr (L < N) {
            const int j = get<L, JN>(r) + 32;
            put<L, JN>(r, j);
            const int b = get<L, V0>(r) == 1 ? 0 : 1;
            if (b) put<L, Q1>(r, j - 1);
            else put<L, Q0>(r, j - 1);
            ones_take<L + 1>(2 * r + b, base);
        }
    }
    SPK_DEV bool absorb_ones(int base) {
        if (last_t != base - 1 || !ones_steady<1>(0)) return false;
        ones_take<1>(0, base);
        nint += 32;
        last_t = base + 31;
        return true;
    }

    SPK_DEV int frontier() const {
        int S = last_t;
#pragma unroll
        for (int k = 0; k < TOPN; ++k)
            if (top[CNT][k] && top[PCT][k] < S) S = top[PCT][k];
        if constexpr (NODES > TOPN)
            for (int k = 0; k < DEEPN; ++k)
                if (deep[CNT * DEEPN + k] && deep[PCT * DEEPN + k] < S) S = deep[PCT * DEEPN + k];
        return S;
    }
    // Most cuts come after every pending one (a level-1 break, or the first pending cut):
    // they are appended without reading the ring, whose first and last times are kept in
    // registers; only a cut that lands inside the list walks it.
    SPK_DEV void push(int t, int i) {
        if (t <= rel_t) {               // handed over already (equal) -- earlier would be a fault
            if (t < rel_t) bad |= TREE_BAD_ORDER;
            return;
        }
        if (np > 0 && t == tlast) return;  // the same cut from two levels
        int j = np;
        if (np > 0 && t < tlast) {
            --j;                         // the last entry is tlast > t
            while (j > 0 && pt[slot(j - 1)] > t) --j;
            if (j > 0 && pt[slot(j - 1)] == t) return;
        }
        if (np == pcap) {
            bad |= TREE_BAD_FULL;
            return;
        }
        for (int m = np; m > j; --m) {
            const int64_t a = slot(m), b = slot(m - 1);
            pt[a] = pt[b];
            pi[a] = pi[b];
        }
        const int64_t s = slot(j);
        pt[s] = t;
        pi[s] = i;
        if (j == 0) thead = t;
        if (j == np) tlast = t;
        ++np;
    }
    // the sequences of every descendant of node r of level L end
    template <int L>
    SPK_DEV void reset_below(int r) {
        if constexpr (L < N) {
#pragma unroll
            for (int M = L + 1; M <= N; ++M) {
                const int B = (1 << (M - 1)) - 1;
                if (M <= RL) {
#pragma unroll
                    for (int i = 0; i < (1 << (M - 1)); ++i)
                        if ((i >> (M - L)) == r) {
                            top[CNT][B + i] = 0;
                            if (M < N) top[Q0][B + i] = top[Q1][B + i] = -1;
                        }
                } else {
                    const int lo = B - TOPN + (r << (M - L));
                    for (int i = 0; i < (1 << (M - L)); ++i) {
                        deep[CNT * DEEPN + lo + i] = 0;
                        if (M < N) deep[Q0 * DEEPN + lo + i] = deep[Q1 * DEEPN + lo + i] = -1;
                    }
                }
            }
        }
    }
    // element x, whose own cut is (ct, ci), arrives at node r of level L; then the distance
    // it closes travels down the branch of its value
    template <int L>
    SPK_DEV void element(int x, int r, int ct, int ci) {
        int c = get<L, CNT>(r), a0 = get<L, V0>(r), a1 = get<L, V1>(r);
        int b0 = -1, b1 = -1;
        if constexpr (L < N) {
            b0 = get<L, Q0>(r);
            b1 = get<L, Q1>(r);
        }
        if (c == 0) {
            a0 = x;
            a1 = 0;
        } else if (x != a0 && x != a1) {
            if (a1 == 0 && (x - a0 == 1 || a0 - x == 1)) {
                a1 = x;
            } else {                     // zero-order rule broken: the sequence ends after
                push(get<L, PCT>(r), get<L, PCI>(r));  // the previous element, x opens the next
                a0 = x;
                a1 = 0;
                c = 0;
                b0 = b1 = -1;
                reset_below<L>(r);
            }
        }
        put<L, CNT>(r, c + 1);
        put<L, V0>(r, a0);
        put<L, V1>(r, a1);
        put<L, PCT>(r, ct);
        put<L, PCI>(r, ci);
        if constexpr (L < N) {
            const int j = get<L, JN>(r);
            put<L, JN>(r, j + 1);
            const int b = x == a0 ? 0 : 1;
            const int prev = b ? b1 : b0;
            put<L, Q0>(r, b ? b0 : j);
            put<L, Q1>(r, b ? j : b1);
            if (prev >= 0) element<L + 1>(j - prev, 2 * r + b, ct, ci);
        }
    }
    template <class Sink>
    SPK_DEV void spike(int t, Sink &) {
        element<1>(t - last_t, 0, t, nint);
        ++nint;
        last_t = t;
    }
    // hand every final pending cut to the sink, in time order
    template <class Sink>
    SPK_DEV void release(Sink &sink, int S) {
        while (np > 0 && thead <= S) {
            sink.cand(thead, pi[slot(0)]);
            rel_t = thead;
            ph = (ph + 1) & (pcap - 1);
            if (--np > 0) thead = pt[slot(0)];
        }
    }
    template <class Sink>
    SPK_DEV void release(Sink &sink) { release(sink, frontier()); }
    template <class Sink>
    SPK_DEV void finish(Sink &sink) {
        if (nint >= 1) push(last_t, nint - 1);
        release(sink, 0x7fffffff);
    }
};

}  // namespace spk
