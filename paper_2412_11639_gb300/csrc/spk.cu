// libspk: GB300 (sm_103a) spike-camera reconstruction -- kernels and the C ABI of spk.h.
//
// One kernel does the whole hot path of Sec. III-B for a block of 256 consecutive pixels:
//   1. TMA (cp.async.bulk.tensor) stages [64 steps] x [32 bytes] tiles of the bit-packed
//      stream into shared memory through a 4-stage mbarrier pipeline fed by one producer
//      warp (the paper's FPGA sequence buffer, Sec. III-C, does the same transposition of
//      frame-major bits into per-pixel time sequences);
//   2. each compute warp turns its 32 x 32 bit tile (32 steps x 32 pixels) into one
//      32-step time word per lane with a 5-stage shuffle transpose;
//   3. each lane runs the stability scan (spk_scan.cuh: FSR, SSR, the TFI baseline, or
//      the general n-order tree) over the spikes of its time word (ffs per spike) and
//      hands every cut to a per-lane shared-memory queue;
//   4. final cuts are converted in place into records (last frame index, value =
//      threshold * N / D, Eq. 4) -- the analogue of the FPGA encoder's (duration,
//      intensity) records;
//   5. every 256 steps the warp writes the frame rows every lane has resolved, one
//      coalesced row (32 consecutive pixels) per store; a lane whose queue runs full
//      writes its oldest record on its own.
// The TFP baseline and the refiner's input features use the same pipeline in kernels of
// their own; the learned refiner lives in refiner.cu.
// Values are known only when a sequence closes, which may be thousands of steps later
// (a static pixel is one sequence), so rows are written when resolved, not when sampled.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <type_traits>

#include "../../include/spk.h"
#include "spk_scan.cuh"

namespace {

constexpr int NCW = 8;                   // compute warps per block
constexpr int BLOCK_PIX = NCW * 32;      // pixels per block
constexpr int ROW_BYTES = BLOCK_PIX / 8; // bytes of one frame row per block (TMA box x)
constexpr int TT_DEFAULT = 64;           // steps per TMA tile (box y); 32, 64 or 128
constexpr int NS = 4;                    // pipeline stages
constexpr int QCAP = 32;        // records per lane
constexpr int FLUSH_WORDS = 8;  // 32-step words between two row flushes of a warp
constexpr int NTHREADS = (NCW + 1) * 32; // + one producer warp
constexpr unsigned FULL = 0xffffffffu;
constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz: bounded waits

// device status bits
constexpr int DEV_TIMEOUT = 1;
constexpr int DEV_INTERNAL = 2;
constexpr int DEV_PEND_FULL = 4;   // an n-order tree's pending-cut ring was too small (the host reruns)
constexpr int NORDER_CAP0 = 64;    // initial pending-cut ring per pixel (entries, a power of two)

template <int TT>
struct Smem {
    uint8_t stage[NS][TT][ROW_BYTES];
    unsigned long long full[NS];
    unsigned long long empty[NS];
    int rec_t[NCW][QCAP][32];
    int rec_i[NCW][QCAP][32];
};
template <int TT>
constexpr size_t smem_bytes() { return sizeof(Smem<TT>) + 128; }  // + alignment slack for TMA

// One job: a piece of one stream (the whole stream, or the next steps of a live stream
// whose per-pixel state is carried in device memory between launches).
constexpr int JOB_FIRST = 1;  // the piece starts the stream (no carried state)
constexpr int JOB_LAST = 2;   // the piece ends the stream (tail hold, every frame written)
constexpr int CARRY_INTS = 20;  // carried state per pixel, stored [CARRY_INTS][P]

struct Job {
    int64_t P;      // pixels
    void *out;      // frames [T_out][P], absolute frame index
    int *carry;     // [CARRY_INTS][P] (streams) or nullptr
    int *ready;     // after the launch: min over pixels of frames written (streams) or nullptr
    int n;          // steps in this piece (rows of its tensor map)
    int ntiles;     // ceil(n / tile)
    int t_base;     // absolute step of the piece's first row
    int T_out;      // frames of the whole stream
    int stride;     // frame stride
    uint32_t div_m; // t / stride = umulhi(t, div_m) >> div_s for 0 <= t < 2^31 (stride >= 2)
    int div_s;
    float theta;    // threshold of Eq. 4
    int window;     // TFP window in steps
    int order_n;    // levels of the n-order tree (method SPK_NORDER)
    int edges;      // frame edge policy (EDGE_ZERO_HEAD | EDGE_ZERO_TAIL)
    int flags;      // JOB_FIRST | JOB_LAST
    int block0;     // first block of this job in the flat grid
    int64_t pend_px;  // n-order tree, whole streams: the job's first pixel in the context's rings
    int *pend;        // n-order tree: the job's pending-cut rings [P][pend_cap][2]
    int pend_cap;
};

template <int MAXJ>
struct Batch {
    CUtensorMap maps[MAXJ];  // one per job: the piece, [n][pitch] bytes
    Job jobs[MAXJ];
    int njobs;
    int *status;
    int32_t *spikes;                            // segments mode (one job): K per pixel, or nullptr
    int32_t *counts, *seg_ts, *seg_te, *seg_n;  // segments mode: the stable sequences
    float *seg_v;
    int cap;
};

// ------------------------------------------------------------------ PTX helpers ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// generic-proxy shared loads, ordered before a later async-proxy (TMA) refill of the stage
__device__ __forceinline__ uint32_t lds_u32(const void *p) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
    return v;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false (and the status word flagged) if the phase never completes
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, int *status,
                                          long long limit = WAIT_CYCLES) {
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) {
            atomicOr(status, DEV_TIMEOUT);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map,
                                            unsigned long long *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// 32 x 32 bit transpose across a warp: lane l holds row l (bit b = element [l][b]);
// afterwards lane l holds column l (bit t = element [t][l]).  Five block swaps.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
#pragma unroll
    for (int j = 16; j >= 1; j >>= 1) {
        const uint32_t m = j == 16 ? 0x0000FFFFu
                         : j == 8  ? 0x00FF00FFu
                         : j == 4  ? 0x0F0F0F0Fu
                         : j == 2  ? 0x33333333u
                                   : 0x55555555u;
        uint32_t y = __shfl_xor_sync(FULL, x, j);
        x = (lane & j) ? (((y >> j) & m) | (x & ~m)) : ((x & m) | ((y & m) << j));
    }
    return x;
}

template <typename OutT> __device__ __forceinline__ OutT to_out(float v);
template <> __device__ __forceinline__ float to_out<float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_out<__half>(float v) { return __float2half_rn(v); }

// Eq. 4 with the scale generalised: theta / (D / N) = theta * N / D, correctly rounded
// (theta * N is exact for theta = 1 and N < 2^24).
__device__ __forceinline__ float seq_value(float theta, int n, int d) {
    return __fdiv_rn(__fmul_rn(theta, static_cast<float>(n)), static_cast<float>(d));
}

// 8-bit output (the decoder's 8-bit frames, Sec. III-C, with the 8-bit scale of Eq. 4):
// theta * N / D rounded half up and clamped to 255, exactly, in integers (theta integral).
__device__ __forceinline__ int seq_u8(int theta, int n, int d) {
    const long long v = (2LL * theta * n + d) / (2LL * d);
    return v > 255 ? 255 : static_cast<int>(v);
}
// a span's value as a record stores it: the fp32 bits, or the 8-bit value for uint8_t frames
template <typename OutT>
__device__ __forceinline__ int value_bits(float theta, int n, int d) {
    if constexpr (std::is_same_v<OutT, uint8_t>) return seq_u8(static_cast<int>(theta), n, d);
    else return __float_as_int(seq_value(theta, n, d));
}
template <typename OutT>
__device__ __forceinline__ OutT from_bits(int b) {
    if constexpr (std::is_same_v<OutT, uint8_t>) return static_cast<uint8_t>(b);
    else return to_out<OutT>(__int_as_float(b));
}
// frame edge policy bits (spk_config.edges)
constexpr int EDGE_ZERO_HEAD = SPK_ZERO_HEAD, EDGE_ZERO_TAIL = SPK_ZERO_TAIL;

// --------------------------------------------------------------------- sinks ----
// Cuts of one lane, in time order, in a per-lane shared-memory ring.  Stable spans run
// between consecutive cuts, so span j has N = i_j - i_{j-1} intervals over
// D = t_j - t_{j-1} steps; the first starts at the first spike with index -1.  A candidate
// arrives as (t_cut, i_cut); one that arrives one place early (a retroactive S_2 cut) is
// swapped in front of the last cut.  Every cut but the last is final, and the last is
// final once it is at or before the scan's frontier.  Final cuts are converted in place,
// in order, into (last frame of the span, value of the span), so that writing a frame row
// costs one comparison per lane and a new span two shared-memory loads.  The pixel's last
// record is TAIL: it holds the last value for the frames after the last spike (0 if there
// is no span).
constexpr int TAIL = INT_MAX;

template <typename OutT>
struct FrameSink {
    int *rt;       // &rec_t[warp][0][lane], slot stride 32: t_cut, or the last frame once converted
    int *ri;       // i_cut, or the value's bits once converted
    OutT *col;     // out + p: frame k at col[k * P]
    int64_t P;
    float theta;
    int stride;
    uint32_t div_m;
    int div_s;
    int T_out;
    int head, tail;  // ring positions (monotone)
    int sorted;      // records before this position are in time order
    int conv;        // records before this position are converted
    int W;           // frames < W are written
    int kf;          // frames < kf are covered by converted records
    int bad;         // set if a flush found no record for a frame (never expected)
    int ct, ci;      // the last converted cut (the first spike and -1 before the first)
    int cvb;         // value bits (value_bits) of the last converted span (0 before the first)
    int zero_tail;   // frames after the last spike read 0 (edge policy)
    int cur_ke;      // cursor: the record at head covers frames up to cur_ke, value cur_o
    OutT cur_o;

    __device__ __forceinline__ int slot(int j) const { return (j & (QCAP - 1)) * 32; }
    __device__ __forceinline__ int frame_of(int t) const {  // t / stride, t >= 0
        return stride == 1 ? t : static_cast<int>(__umulhi(static_cast<uint32_t>(t), div_m) >> div_s);
    }
    __device__ __forceinline__ void load() {
        const int s = slot(head);
        cur_ke = rt[s];
        cur_o = from_bits<OutT>(ri[s]);
    }
    // A candidate that arrived one place early is swapped in front of its predecessor
    // (converted records are final and never move).
    __device__ __forceinline__ void sort_new() {
        for (int j = max(sorted - 1, conv); j + 1 < tail; ++j) {
            const int a = slot(j), b = slot(j + 1);
            const int ta = rt[a], tb = rt[b];
            if (tb < ta) {
                const int ia = ri[a];
                rt[a] = tb;
                ri[a] = ri[b];
                rt[b] = ta;
                ri[b] = ia;
            }
        }
        sorted = tail;
    }
    // records [conv, R) are final and sorted: (t_cut, i_cut) -> (last frame, value)
    __device__ __forceinline__ void convert(int R) {
        for (; conv < R; ++conv) {
            const int s = slot(conv);
            const int t = rt[s];
            int ke;
            if (t == TAIL) {
                ke = T_out - 1;
                if (zero_tail) cvb = 0;
            } else {
                const int i = ri[s];
                cvb = value_bits<OutT>(theta, i - ci, t - ct);
                ct = t;
                ci = i;
                ke = frame_of(t);
            }
            rt[s] = ke;
            ri[s] = cvb;
            kf = max(kf, ke + 1);
        }
    }
    // convert every final record: all but the last, and the last if it is at or before
    // the frontier
    __device__ __forceinline__ void convert_final(int frontier) {
        int R = tail;
        if (R > conv && rt[slot(R - 1)] > frontier) --R;
        convert(R);
    }
    // Edge policy: frames up to the first spike t0 read 0.  At the first spike the ring is
    // empty; a converted record (last frame frame_of(t0), value 0) goes ahead of the first
    // span, which then covers only the frames after t0.
    __device__ __forceinline__ void zero_head(int t0) {
        const int s = slot(tail);
        const int ke = frame_of(t0);
        rt[s] = ke;
        ri[s] = 0;
        ++tail;
        sorted = conv = tail;
        kf = max(kf, ke + 1);
    }
    __device__ __forceinline__ void drain_one() {  // ring full: write the oldest record alone
        sort_new();
        convert(head + 2);  // the ring holds QCAP records, so these two are final
        load();
        const int kl = min(cur_ke, T_out - 1);
        for (int k = W; k <= kl; ++k) col[static_cast<int64_t>(k) * P] = cur_o;
        if (kl + 1 > W) W = kl + 1;
        ++head;
    }
    __device__ __forceinline__ void cand(int t, int i) {
        if (tail - head == QCAP) drain_one();
        const int s = slot(tail);
        rt[s] = t;
        ri[s] = i;
        ++tail;
    }
    // Room for one more record (a spike's put): the oldest goes out if the ring is full.
    __device__ __forceinline__ void reserve() {
        if (tail - head == QCAP) drain_one();
    }
    // A spike's outcome, after reserve(): the slot at tail is free, so the record is
    // stored under a predicate and tail advances by emit -- no branch in the spike loop.
    __device__ __forceinline__ void put(bool emit, int t, int i) {
        const int s = slot(tail);
        if (emit) {
            rt[s] = t;
            ri[s] = i;
        }
        tail += emit ? 1 : 0;
    }
};

// Verification sink: the spans themselves, in time order (a one-candidate hold restores
// the order of a candidate that arrives one place early).
struct SegSink {
    int32_t *ts, *te, *n;
    float *v;
    int64_t P, p;
    float theta;
    int cap, cnt;
    int ct, ci;        // last emitted cut (the first spike and -1 at the start)
    int ht, hi, held;  // held candidate
    __device__ __forceinline__ void emit(int t, int i) {
        if (cnt < cap) {
            const int64_t o = static_cast<int64_t>(cnt) * P + p;
            ts[o] = ct;
            te[o] = t;
            n[o] = i - ci;
            v[o] = seq_value(theta, i - ci, t - ct);
        }
        ++cnt;
        ct = t;
        ci = i;
    }
    __device__ __forceinline__ void cand(int t, int i) {
        if (!held) {
            ht = t;
            hi = i;
            held = 1;
        } else if (t < ht) {
            emit(t, i);
        } else {
            emit(ht, hi);
            ht = t;
            hi = i;
        }
    }
    __device__ __forceinline__ void put(bool e, int t, int i) {
        if (e) cand(t, i);
    }
    __device__ __forceinline__ void done() {
        if (held) emit(ht, hi);
        held = 0;
    }
};

// Warp-wide write of resolved frame rows.  Normal: rows below the warp minimum of the
// resolved counts (full rows).  Forced (a ring is nearly full, or the stream ended):
// every lane up to its own resolved count.
template <typename OutT>
__device__ __forceinline__ void flush_rows(FrameSink<OutT> &sk, int frontier, bool valid, bool final_flush) {
    if (valid) {
        if (sk.sorted < sk.tail) sk.sort_new();
        sk.convert_final(frontier);
    }
    const int F = valid ? max(sk.W, sk.kf) : INT_MAX;
    const int Wl = valid ? sk.W : INT_MAX;
    const int used = valid ? sk.tail - sk.head : 0;
    const int Fmin = __reduce_min_sync(FULL, F);
    const int Wmin = __reduce_min_sync(FULL, Wl);
    const bool forced = final_flush || __reduce_max_sync(FULL, used) > QCAP - 8;
    int khi, lim;
    if (forced) {
        khi = __reduce_max_sync(FULL, valid ? F : 0);
        lim = F;
    } else {
        khi = Fmin;
        lim = Fmin;
    }
    if (Wmin >= khi) return;  // nothing to write (warp-uniform)
    const int klo = valid ? sk.W : INT_MAX;
    if (!valid) lim = 0;
    if (sk.W < lim) sk.load();
    // one row per iteration for the whole warp, so that the lanes' stores coalesce
    OutT *ptr = sk.col + static_cast<int64_t>(Wmin) * sk.P;
    for (int k = Wmin; k < khi; ++k, ptr += sk.P) {
        if (k >= klo && k < lim) {
            while (k > sk.cur_ke) {  // the next converted record
                if (sk.head + 1 >= sk.conv) {  // none covers frame k: inconsistent, never expected
                    sk.bad = 1;
                    break;
                }
                ++sk.head;
                sk.load();
            }
            *ptr = sk.cur_o;
        }
    }
    if (lim > sk.W) sk.W = lim;
}

// ------------------------------------------------------------------- the kernel ----
// Carried state of one pixel between pieces of a stream: the scan registers, the frames
// written, the last final cut (start of the open span) and up to two pending candidates.
template <int ORDER, typename OutT>
__device__ __forceinline__ void carry_load(const int *c, int64_t P, int64_t p, spk::PixelScan<ORDER> &sc,
                                           FrameSink<OutT> &fs) {
    c += p;
    sc.last_t = c[0 * P];
    sc.nint = c[1 * P];
    sc.v0 = c[2 * P];
    sc.v1 = c[3 * P];
    sc.q0 = c[4 * P];
    sc.tq0 = c[5 * P];
    sc.dlo0 = c[6 * P];
    sc.dhi0 = c[7 * P];
    sc.q1 = c[8 * P];
    sc.tq1 = c[9 * P];
    sc.dlo1 = c[10 * P];
    sc.dhi1 = c[11 * P];
    fs.W = fs.kf = c[12 * P];
    fs.ct = c[13 * P];
    fs.ci = c[14 * P];
    const int npend = c[15 * P];
    if (npend > 0) {
        fs.rt[fs.slot(0)] = c[16 * P];
        fs.ri[fs.slot(0)] = c[17 * P];
    }
    if (npend > 1) {
        fs.rt[fs.slot(1)] = c[18 * P];
        fs.ri[fs.slot(1)] = c[19 * P];
    }
    fs.tail = fs.sorted = npend;
}

template <int ORDER, typename OutT>
__device__ __forceinline__ void carry_store(int *c, int64_t P, int64_t p, const spk::PixelScan<ORDER> &sc,
                                            const FrameSink<OutT> &fs, int npend, int pj) {
    c += p;
    c[0 * P] = sc.last_t;
    c[1 * P] = sc.nint;
    c[2 * P] = sc.v0;
    c[3 * P] = sc.v1;
    c[4 * P] = sc.q0;
    c[5 * P] = sc.tq0;
    c[6 * P] = sc.dlo0;
    c[7 * P] = sc.dhi0;
    c[8 * P] = sc.q1;
    c[9 * P] = sc.tq1;
    c[10 * P] = sc.dlo1;
    c[11 * P] = sc.dhi1;
    c[12 * P] = fs.W;
    c[13 * P] = fs.ct;
    c[14 * P] = fs.ci;
    c[15 * P] = npend;
    c[16 * P] = npend > 0 ? fs.rt[fs.slot(pj)] : 0;
    c[17 * P] = npend > 0 ? fs.ri[fs.slot(pj)] : 0;
    c[18 * P] = npend > 1 ? fs.rt[fs.slot(pj + 1)] : 0;
    c[19 * P] = npend > 1 ? fs.ri[fs.slot(pj + 1)] : 0;
}

// Carried state of one pixel of the n-order tree between pieces of a live stream, [rows][P]:
// the scan's scalars (its pending-cut ring stays in the stream's ring buffer), the frame
// sink's frames written and last final cut (every released cut is final, so none is pending
// at a piece end), and every node field.
constexpr int TREE_ROW_PH = 2, TREE_ROW_NP = 3, TREE_CARRY_FIXED = 11;
template <class Tree>
constexpr int tree_carry_rows() { return TREE_CARRY_FIXED + Tree::NF * (Tree::TOPN + Tree::DEEPN); }

template <class Tree, typename OutT>
__device__ __forceinline__ void tree_carry_load(const int *c, int64_t P, int64_t p, Tree &sc, FrameSink<OutT> &fs) {
    c += p;
    sc.last_t = c[0 * P];
    sc.nint = c[1 * P];
    sc.ph = c[2 * P];
    sc.np = c[3 * P];
    sc.thead = c[4 * P];
    sc.tlast = c[5 * P];
    sc.rel_t = c[6 * P];
    sc.bad = c[7 * P];
    fs.W = fs.kf = c[8 * P];
    fs.ct = c[9 * P];
    fs.ci = c[10 * P];
    const int *t = c + static_cast<int64_t>(TREE_CARRY_FIXED) * P;
#pragma unroll
    for (int f = 0; f < Tree::NF; ++f)
#pragma unroll
        for (int k = 0; k < Tree::TOPN; ++k) sc.top[f][k] = t[static_cast<int64_t>(f * Tree::TOPN + k) * P];
    if constexpr (Tree::NODES > Tree::TOPN) {
        const int *d = t + static_cast<int64_t>(Tree::NF * Tree::TOPN) * P;
        for (int k = 0; k < Tree::NF * Tree::DEEPN; ++k) sc.deep[k] = d[static_cast<int64_t>(k) * P];
    }
}

template <class Tree, typename OutT>
__device__ __forceinline__ void tree_carry_store(int *c, int64_t P, int64_t p, const Tree &sc,
                                                 const FrameSink<OutT> &fs) {
    c += p;
    c[0 * P] = sc.last_t;
    c[1 * P] = sc.nint;
    c[2 * P] = sc.ph;
    c[3 * P] = sc.np;
    c[4 * P] = sc.thead;
    c[5 * P] = sc.tlast;
    c[6 * P] = sc.rel_t;
    c[7 * P] = sc.bad;
    c[8 * P] = fs.W;
    c[9 * P] = fs.ct;
    c[10 * P] = fs.ci;
    int *t = c + static_cast<int64_t>(TREE_CARRY_FIXED) * P;
#pragma unroll
    for (int f = 0; f < Tree::NF; ++f)
#pragma unroll
        for (int k = 0; k < Tree::TOPN; ++k) t[static_cast<int64_t>(f * Tree::TOPN + k) * P] = sc.top[f][k];
    if constexpr (Tree::NODES > Tree::TOPN) {
        int *d = t + static_cast<int64_t>(Tree::NF * Tree::TOPN) * P;
        for (int k = 0; k < Tree::NF * Tree::DEEPN; ++k) d[static_cast<int64_t>(k) * P] = sc.deep[k];
    }
}

// A live stream's pending-cut rings grown from old_cap to new_cap cuts per pixel: each
// pixel's np pending cuts, first at slot ph, move to slots 0 .. np-1 of its new ring and
// its carried ph becomes 0.
__global__ void tree_ring_grow_kernel(const int *old_ring, int old_cap, int *new_ring, int new_cap, int *carry,
                                      int64_t P) {
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < P;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int ph = carry[TREE_ROW_PH * P + p], np = carry[TREE_ROW_NP * P + p];
        const int *o = old_ring + p * 2 * old_cap;
        int *n = new_ring + p * 2 * new_cap;
        for (int j = 0; j < np && j < new_cap; ++j) {
            const int sl = (ph + j) & (old_cap - 1);
            n[2 * j] = o[2 * sl];
            n[2 * j + 1] = o[2 * sl + 1];
        }
        carry[TREE_ROW_PH * P + p] = 0;
    }
}

// ORDER: 1 FSR, 2 SSR, 3 TFI, TREE_ORDER0 + n the n-order tree (n = 3..5 levels)
constexpr int TREE_ORDER0 = 10;
// The tree's first levels keep their node state in registers (7 nodes), deeper ones in local
// memory.  n = 3 fits two blocks per SM in 96 registers (bench stream 12.8 ms; one block:
// 14.7 ms); n = 4 and 5 take one (146 and 162 registers: 23.1 and 35.5 ms; two blocks with
// spills: 33.4 and 56.8 ms).
constexpr int TREE_REG_LEVELS = 3;
constexpr int tree_min_blocks(int order) { return order == TREE_ORDER0 + 3 ? 2 : 1; }

template <int ORDER, typename OutT, bool SEGMENTS, int MAXJ, int TT>
__global__ void __launch_bounds__(NTHREADS, ORDER > TREE_ORDER0 ? tree_min_blocks(ORDER) : 3)
    spk_scan_kernel(const __grid_constant__ Batch<MAXJ> prm) {
    constexpr int WPT = TT / 32;  // 32-step words per tile
    extern __shared__ uint8_t smem_raw[];
    Smem<TT> &sm = *reinterpret_cast<Smem<TT> *>(smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127));
    __shared__ int s_job;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        int jb = 0;  // the job whose block range holds this block
        for (int k = 1; k < prm.njobs; ++k)
            if (static_cast<int>(blockIdx.x) >= prm.jobs[k].block0) jb = k;
        s_job = jb;
        for (int s = 0; s < NS; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], NCW * 32);  // every consumer lane releases
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int jb = s_job;
    const Job &job = prm.jobs[jb];
    const int blk = static_cast<int>(blockIdx.x) - job.block0;  // block within the job

    if (warp == NCW) {  // ---------------------------------------- producer warp ----
        if (lane == 0) {
            const CUtensorMap *map = &prm.maps[jb];
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
            int issued = 0;
            for (int j = 0; j < job.ntiles; ++j) {
                const int s = j % NS;
                if (j >= NS && !mbar_wait(&sm.empty[s], ((j / NS) - 1) & 1, prm.status)) break;
                mbar_arrive_expect_tx(&sm.full[s], TT * ROW_BYTES);
                tma_load_2d(&sm.stage[s][0][0], map, &sm.full[s], blk * ROW_BYTES, j * TT);
                issued = j + 1;
            }
            // let every copy land before this warp leaves (matters only after an error)
            for (int j = issued > NS ? issued - NS : 0; j < issued; ++j)
                if (!mbar_wait(&sm.full[j % NS], (j / NS) & 1, prm.status)) break;
        }
        return;
    }

    // ------------------------------------------------------------- compute warps ----
    const int64_t p = static_cast<int64_t>(blk) * BLOCK_PIX + warp * 32 + lane;
    const bool valid = p < job.P;
    constexpr bool TREE = ORDER > TREE_ORDER0;
    constexpr int TN = TREE ? ORDER - TREE_ORDER0 : spk::TREE_MIN;
    using Tree = spk::TreeScan<TN, TN < TREE_REG_LEVELS ? TN : TREE_REG_LEVELS>;
    using Scan = std::conditional_t<TREE, Tree, spk::PixelScan<TREE ? 1 : ORDER>>;
    Scan sc;
    int tree_deep[TREE ? Tree::NF * Tree::DEEPN : 1];  // the tree's deep levels (local memory)
    if constexpr (TREE) {  // the pixel's ring: pend_cap (t, i) pairs, contiguous
        int *ring = job.pend + static_cast<int64_t>(valid ? p : 0) * 2 * job.pend_cap;
        sc.init(tree_deep, ring, ring + 1, 2, job.pend_cap);
    } else {
        sc.init();
    }

    FrameSink<OutT> fs;
    SegSink ss;
    if constexpr (SEGMENTS) {
        ss = SegSink{prm.seg_ts, prm.seg_te, prm.seg_n, prm.seg_v, job.P, p, job.theta, prm.cap, 0, 0, -1, 0, 0, 0};
    } else {
        fs.rt = &sm.rec_t[warp][0][lane];
        fs.ri = &sm.rec_i[warp][0][lane];
        fs.col = static_cast<OutT *>(job.out) + (valid ? p : 0);
        fs.P = job.P;
        fs.theta = job.theta;
        fs.stride = job.stride;
        fs.T_out = job.T_out;
        fs.div_m = job.div_m;
        fs.div_s = job.div_s;
        fs.head = fs.tail = fs.sorted = fs.conv = fs.W = fs.kf = fs.bad = 0;
        fs.ct = fs.cur_ke = 0;
        fs.ci = -1;
        fs.cvb = 0;
        fs.zero_tail = (job.edges & EDGE_ZERO_TAIL) != 0;
        fs.cur_o = from_bits<OutT>(0);
        if (!(job.flags & JOB_FIRST) && valid) {
            // (one-job launches of the tree are whole streams: live pieces come in batches)
            if constexpr (!TREE) carry_load(job.carry, job.P, p, sc, fs);
            else if constexpr (MAXJ > 1) tree_carry_load(job.carry, job.P, p, sc, fs);
        }
    }

    bool ok = true;
    const int ntiles = job.ntiles, t_base = job.t_base;  // kept in registers
    for (int j = 0; j < ntiles; ++j) {
        const int s = j % NS;
        // warp-uniform outcome: every lane leaves together if any lane's wait gave up
        if (!__all_sync(FULL, mbar_wait(&sm.full[s], (j / NS) & 1, prm.status))) {
            ok = false;
            break;
        }
        uint32_t r[WPT];
#pragma unroll
        for (int h = 0; h < WPT; ++h) r[h] = lds_u32(&sm.stage[s][lane + 32 * h][warp * 4]);
        // each lane orders its own reads before the producer may refill this stage
        fence_proxy_async_smem();
        mbar_arrive(&sm.empty[s]);
#pragma unroll
        for (int h = 0; h < WPT; ++h) {
            uint32_t w = warp_transpose32(r[h], lane);
            if (!valid) w = 0;
            const int base = t_base + j * TT + h * 32;
            if (sc.last_t < 0 && w) {  // the stream's first spike opens the first sequence
                const int t0 = base + __ffs(w) - 1;
                sc.first_spike(t0);
                if constexpr (SEGMENTS) {
                    ss.ct = t0;  // the first span starts here
                } else {
                    fs.ct = t0;
                    if (job.edges & EDGE_ZERO_HEAD) fs.zero_head(t0);
                }
                w &= w - 1;
            }
            if (w == 0xffffffffu && sc.absorb_ones(base)) w = 0;  // steady run of 1-intervals
            while (w) {
                const int b = __ffs(w) - 1;
                w &= w - 1;
                if constexpr (SEGMENTS) {
                    sc.spike(base + b, ss);
                } else {
                    // FSR cuts rarely: its spike keeps a branch to cand(), which makes room itself;
                    // the tree keeps its own list
                    if constexpr (ORDER == 2 || ORDER == 3) fs.reserve();
                    sc.spike(base + b, fs);
                }
            }
            if constexpr (TREE) {  // the tree's final cuts go to the sink in order
                if constexpr (SEGMENTS) sc.release(ss);
                else sc.release(fs);
            }
            // rows go out every FW words: fewer warp reductions of the flush (TFI cuts at every
            // spike and would overflow the record ring between sparse flushes: every word)
            constexpr int FW = ORDER == 3 ? 1 : FLUSH_WORDS;
            if constexpr (!SEGMENTS)
                if (((j * WPT + h) % FW) == FW - 1 || (j == ntiles - 1 && h == WPT - 1))
                    flush_rows(fs, sc.frontier(), valid, false);
        }
    }
    if (!ok) return;

    if constexpr (SEGMENTS) {
        sc.finish(ss);
        ss.done();
        if (valid) prm.counts[p] = ss.cnt;
        // K, the number of spikes (S_1 has K - 1 elements, Def. 2): the scan's own count
        if (valid && prm.spikes) prm.spikes[p] = sc.last_t >= 0 ? sc.nint + 1 : 0;
        if constexpr (TREE)
            if (valid && sc.bad)
                atomicOr(prm.status, (sc.bad & spk::TREE_BAD_ORDER ? DEV_INTERNAL : 0) |
                                         (sc.bad & spk::TREE_BAD_FULL ? DEV_PEND_FULL : 0));
    } else if (job.flags & JOB_LAST) {
        sc.finish(fs);
        if constexpr (TREE)
            if (valid && sc.bad)
                atomicOr(prm.status, (sc.bad & spk::TREE_BAD_ORDER ? DEV_INTERNAL : 0) |
                                         (sc.bad & spk::TREE_BAD_FULL ? DEV_PEND_FULL : 0));
        if (valid) fs.cand(TAIL, 0);  // tail hold (0 without spans)
        flush_rows(fs, INT_MAX, valid, true);
        if (valid && fs.bad) atomicOr(prm.status, DEV_INTERNAL);
    } else {
        // piece end: convert the final cuts and write every resolved frame; the last
        // converted cut starts the open span, the rest are pending candidates
        flush_rows(fs, sc.frontier(), valid, true);
        if (valid) {
            if constexpr (!TREE) {
                const int npend = fs.tail - fs.conv;
                if (npend > 2 || fs.bad) atomicOr(prm.status, DEV_INTERNAL);
                carry_store(job.carry, job.P, p, sc, fs, npend > 2 ? 2 : npend, fs.conv);
            } else if constexpr (MAXJ > 1) {
                if (fs.tail != fs.conv || fs.bad) atomicOr(prm.status, DEV_INTERNAL);
                if (sc.bad)
                    atomicOr(prm.status, (sc.bad & spk::TREE_BAD_ORDER ? DEV_INTERNAL : 0) |
                                             (sc.bad & spk::TREE_BAD_FULL ? DEV_PEND_FULL : 0));
                tree_carry_store(job.carry, job.P, p, sc, fs);
            }
        }
    }
    if constexpr (!SEGMENTS) {
        if (job.ready) {  // frames written for every pixel of the stream
            const int wmin = __reduce_min_sync(FULL, valid ? fs.W : INT_MAX);
            if (lane == 0) atomicMin(job.ready, wmin);
        }
    }
}

// ------------------------------------------------------------------ TFP kernel ----
// TFP (Sec. II): frame k = theta * (spikes in the L steps (t_k - L, t_k]) / L.  The same
// TMA pipeline and transpose feed one lane per pixel; a frame needs no future, so every
// frame row is written (coalesced) as soon as the scan passes its sampling step.
template <int TT>
struct StageSmem {
    uint8_t stage[NS][TT][ROW_BYTES];
    unsigned long long full[NS];
    unsigned long long empty[NS];
};

template <typename OutT, int MAXJ, int TT>
__global__ void __launch_bounds__(NTHREADS, 3) spk_tfp_kernel(const __grid_constant__ Batch<MAXJ> prm) {
    constexpr int WPT = TT / 32;
    extern __shared__ uint8_t smem_raw[];
    StageSmem<TT> &sm = *reinterpret_cast<StageSmem<TT> *>(smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127));
    __shared__ int s_job;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        int jb = 0;
        for (int k = 1; k < prm.njobs; ++k)
            if (static_cast<int>(blockIdx.x) >= prm.jobs[k].block0) jb = k;
        s_job = jb;
        for (int s = 0; s < NS; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], NCW * 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int jb = s_job;
    const Job &job = prm.jobs[jb];
    const int blk = static_cast<int>(blockIdx.x) - job.block0;
    if (warp == NCW) {  // producer warp: as in the scan kernel
        if (lane == 0) {
            const CUtensorMap *map = &prm.maps[jb];
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
            int issued = 0;
            for (int j = 0; j < job.ntiles; ++j) {
                const int s = j % NS;
                if (j >= NS && !mbar_wait(&sm.empty[s], ((j / NS) - 1) & 1, prm.status)) break;
                mbar_arrive_expect_tx(&sm.full[s], TT * ROW_BYTES);
                tma_load_2d(&sm.stage[s][0][0], map, &sm.full[s], blk * ROW_BYTES, j * TT);
                issued = j + 1;
            }
            for (int j = issued > NS ? issued - NS : 0; j < issued; ++j)
                if (!mbar_wait(&sm.full[j % NS], (j / NS) & 1, prm.status)) break;
        }
        return;
    }
    const int64_t p = static_cast<int64_t>(blk) * BLOCK_PIX + warp * 32 + lane;
    const bool valid = p < job.P;
    OutT *col = static_cast<OutT *>(job.out) + (valid ? p : 0);
    const int L = job.window;
    uint32_t h1 = 0, h2 = 0;  // the two previous words (steps before the stream are empty)
    int k = 0;                // next frame
    for (int j = 0; j < job.ntiles; ++j) {
        const int s = j % NS;
        if (!__all_sync(FULL, mbar_wait(&sm.full[s], (j / NS) & 1, prm.status))) return;
        uint32_t r[WPT];
#pragma unroll
        for (int h = 0; h < WPT; ++h) r[h] = lds_u32(&sm.stage[s][lane + 32 * h][warp * 4]);
        fence_proxy_async_smem();
        mbar_arrive(&sm.empty[s]);
#pragma unroll
        for (int h = 0; h < WPT; ++h) {
            uint32_t w = warp_transpose32(r[h], lane);
            if (!valid) w = 0;
            const int base = job.t_base + j * TT + h * 32;
            const unsigned long long hist = static_cast<unsigned long long>(h2) |
                                            (static_cast<unsigned long long>(h1) << 32);
            for (; k < job.T_out && k * job.stride < base + 32; ++k) {  // frames sampled in this word
                const int o = k * job.stride - base;
                const int lo = o - L + 1;
                const uint32_t upto = (2u << o) - 1u;  // bits 0..o
                int cnt = __popc(w & upto & ~((1u << (lo > 0 ? lo : 0)) - 1u));
                if (lo < 0) cnt += __popcll(hist >> (64 + lo));  // the -lo steps before this word
                if (valid) col[static_cast<int64_t>(k) * job.P] =
                    from_bits<OutT>(value_bits<OutT>(job.theta, cnt, L));
            }
            h2 = h1;
            h1 = w;
        }
    }
}

// ------------------------------------------------------------------ TFI kernel ----
// TFI (Sec. II) of one whole stream: frame k = theta / (s_{j+1} - s_j) for the interval
// (s_j, s_{j+1}] holding t_k.  Every interval is its own span, so a lane needs no record
// ring: at each spike t it writes the frames sampled in (previous spike, t] with the
// interval's value (at the second spike also the head frames, sampled at or before the
// first spike: the same value, or 0 under SPK_ZERO_HEAD), and at the end the frames after
// the last spike (the last value, or 0 under SPK_ZERO_TAIL; 0 everywhere with fewer than
// two spikes).  A frame goes out as soon as its interval closes, one lane's store at a
// time.  Same TMA pipeline and transpose as the scan.  (Batches and live streams of TFI
// run in the scan kernel, whose record ring carries the state between pieces.)
template <typename OutT, int TT>
__global__ void __launch_bounds__(NTHREADS, 3) spk_tfi_kernel(const __grid_constant__ Batch<1> prm) {
    constexpr int WPT = TT / 32;
    extern __shared__ uint8_t smem_raw[];
    StageSmem<TT> &sm = *reinterpret_cast<StageSmem<TT> *>(smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Job &job = prm.jobs[0];
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], NCW * 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int blk = static_cast<int>(blockIdx.x);
    if (warp == NCW) {  // producer warp: as in the scan kernel
        if (lane == 0) {
            const CUtensorMap *map = &prm.maps[0];
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
            int issued = 0;
            for (int j = 0; j < job.ntiles; ++j) {
                const int s = j % NS;
                if (j >= NS && !mbar_wait(&sm.empty[s], ((j / NS) - 1) & 1, prm.status)) break;
                mbar_arrive_expect_tx(&sm.full[s], TT * ROW_BYTES);
                tma_load_2d(&sm.stage[s][0][0], map, &sm.full[s], blk * ROW_BYTES, j * TT);
                issued = j + 1;
            }
            for (int j = issued > NS ? issued - NS : 0; j < issued; ++j)
                if (!mbar_wait(&sm.full[j % NS], (j / NS) & 1, prm.status)) break;
        }
        return;
    }
    const int64_t p = static_cast<int64_t>(blk) * BLOCK_PIX + warp * 32 + lane;
    const bool valid = p < job.P;
    OutT *col = static_cast<OutT *>(job.out) + (valid ? p : 0);
    const int stride = job.stride;
    auto frame_of = [&](int t) {  // t / stride, t >= 0
        return stride == 1 ? t : static_cast<int>(__umulhi(static_cast<uint32_t>(t), job.div_m) >> job.div_s);
    };
    const bool zero_head = (job.edges & EDGE_ZERO_HEAD) != 0;
    int lt = -1;   // last spike
    int kh = -1;   // last head frame (sampled at or before the first spike)
    int kw = 0;    // frames < kw are written
    int vb = 0;    // value bits of the last interval
    int nsp = 0;   // spikes so far (saturating at 2)
    for (int j = 0; j < job.ntiles; ++j) {
        const int s = j % NS;
        if (!__all_sync(FULL, mbar_wait(&sm.full[s], (j / NS) & 1, prm.status))) return;
        uint32_t r[WPT];
#pragma unroll
        for (int h = 0; h < WPT; ++h) r[h] = lds_u32(&sm.stage[s][lane + 32 * h][warp * 4]);
        fence_proxy_async_smem();
        mbar_arrive(&sm.empty[s]);
#pragma unroll
        for (int h = 0; h < WPT; ++h) {
            uint32_t w = warp_transpose32(r[h], lane);
            if (!valid) w = 0;
            const int base = job.t_base + j * TT + h * 32;
            while (w) {
                const int t = base + __ffs(w) - 1;
                w &= w - 1;
                if (nsp == 0) {  // the first spike: the head frames wait for the first interval
                    kh = frame_of(t);
                } else {
                    vb = value_bits<OutT>(job.theta, 1, t - lt);
                    const int ke = min(frame_of(t), job.T_out - 1);
                    const OutT v = from_bits<OutT>(vb);
                    const OutT hv = zero_head ? from_bits<OutT>(0) : v;
                    for (int k = kw; k <= ke; ++k) col[static_cast<int64_t>(k) * job.P] = k <= kh ? hv : v;
                    kw = max(kw, ke + 1);
                }
                lt = t;
                nsp = min(nsp + 1, 2);
            }
        }
    }
    if (!valid) return;
    // the frames after the last spike: tail hold, 0 under the zero-tail policy or with < 2 spikes
    const OutT tv = from_bits<OutT>(nsp < 2 || (job.edges & EDGE_ZERO_TAIL) ? 0 : vb);
    for (int k = kw; k < job.T_out; ++k) col[static_cast<int64_t>(k) * job.P] = tv;
}

// --------------------------------------------------------- refiner input features ----
// Input of the learned refiner, bf16 with 16 channels per pixel and frame in two
// channel-chunk planes, [T_out][H][2][W][8]: channel 0 the plain reconstruction of the frame
// (given, fp32), channels 4..7 theta / x for the last four intervals x completed at or
// before t_k (the most recent first; 0 where the pixel has fewer), every other channel 0.
// Same TMA pipeline and transpose as the scan.
constexpr int FEAT_C = 16;  // refiner input channels (two 8-channel planes)

template <int TT>
__global__ void __launch_bounds__(NTHREADS, 3)
    spk_feature_kernel(const __grid_constant__ Batch<1> prm, const float *plain, __nv_bfloat16 *x0, int H, int W) {
    constexpr int WPT = TT / 32;
    extern __shared__ uint8_t smem_raw[];
    StageSmem<TT> &sm = *reinterpret_cast<StageSmem<TT> *>(smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Job &job = prm.jobs[0];
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], NCW * 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int blk = static_cast<int>(blockIdx.x);
    if (warp == NCW) {
        if (lane == 0) {
            const CUtensorMap *map = &prm.maps[0];
            int issued = 0;
            for (int j = 0; j < job.ntiles; ++j) {
                const int s = j % NS;
                if (j >= NS && !mbar_wait(&sm.empty[s], ((j / NS) - 1) & 1, prm.status)) break;
                mbar_arrive_expect_tx(&sm.full[s], TT * ROW_BYTES);
                tma_load_2d(&sm.stage[s][0][0], map, &sm.full[s], blk * ROW_BYTES, j * TT);
                issued = j + 1;
            }
            for (int j = issued > NS ? issued - NS : 0; j < issued; ++j)
                if (!mbar_wait(&sm.full[j % NS], (j / NS) & 1, prm.status)) break;
        }
        return;
    }
    const int64_t p = static_cast<int64_t>(blk) * BLOCK_PIX + warp * 32 + lane;
    const bool valid = p < job.P;
    const int py = static_cast<int>(p / W), px = static_cast<int>(p - static_cast<int64_t>(py) * W);
    int last_t = -1, x1 = 0, x2 = 0, x3 = 0, x4 = 0;
    int k = 0;
    for (int j = 0; j < job.ntiles; ++j) {
        const int s = j % NS;
        if (!__all_sync(FULL, mbar_wait(&sm.full[s], (j / NS) & 1, prm.status))) return;
        uint32_t r[WPT];
#pragma unroll
        for (int h = 0; h < WPT; ++h) r[h] = lds_u32(&sm.stage[s][lane + 32 * h][warp * 4]);
        fence_proxy_async_smem();
        mbar_arrive(&sm.empty[s]);
#pragma unroll
        for (int h = 0; h < WPT; ++h) {
            uint32_t w = warp_transpose32(r[h], lane);
            if (!valid) w = 0;
            const int base = job.t_base + j * TT + h * 32;
            for (; k < job.T_out && k * job.stride < base + 32; ++k) {  // frames sampled here
                const int o = k * job.stride - base;
                const uint32_t upto = (2u << o) - 1u;
                uint32_t now = w & upto;  // spikes at or before t_k
                w &= ~upto;
                while (now) {
                    const int t = base + __ffs(now) - 1;
                    now &= now - 1;
                    if (last_t >= 0) {
                        x4 = x3;
                        x3 = x2;
                        x2 = x1;
                        x1 = t - last_t;
                    }
                    last_t = t;
                }
                if (valid) {
                    const float th = job.theta;
                    const int64_t q = static_cast<int64_t>(k) * job.P + p;
                    __nv_bfloat162 c01 = __floats2bfloat162_rn(plain[q], 0.f);
                    __nv_bfloat162 c45 = __floats2bfloat162_rn(x1 ? __fdiv_rn(th, static_cast<float>(x1)) : 0.f,
                                                               x2 ? __fdiv_rn(th, static_cast<float>(x2)) : 0.f);
                    __nv_bfloat162 c67 = __floats2bfloat162_rn(x3 ? __fdiv_rn(th, static_cast<float>(x3)) : 0.f,
                                                               x4 ? __fdiv_rn(th, static_cast<float>(x4)) : 0.f);
                    uint4 lo;
                    lo.x = *reinterpret_cast<uint32_t *>(&c01);
                    lo.y = 0u;
                    lo.z = *reinterpret_cast<uint32_t *>(&c45);
                    lo.w = *reinterpret_cast<uint32_t *>(&c67);
                    // 16-byte cells: plane 0 of pixel (py, px) of frame k, then plane 1
                    uint4 *cell = reinterpret_cast<uint4 *>(x0);
                    const int64_t c0 = ((static_cast<int64_t>(k) * H + py) * 2) * W + px;
                    cell[c0] = lo;
                    cell[c0 + W] = make_uint4(0u, 0u, 0u, 0u);
                    static_assert(FEAT_C == 16, "two planes of 8 channels");
                }
            }
            while (w) {  // the rest of the word
                const int t = base + __ffs(w) - 1;
                w &= w - 1;
                if (last_t >= 0) {
                    x4 = x3;
                    x3 = x2;
                    x2 = x1;
                    x1 = t - last_t;
                }
                last_t = t;
            }
        }
    }
}

// Self-test of the bounded waits: one warp waits on an mbarrier that nothing arrives at,
// through the same mbar_wait the scan uses, gives up after `limit` cycles and flags the
// status word.
__global__ void wait_selftest_kernel(int *status, long long limit) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    mbar_wait(&bar, 0, status, limit);
}

}  // namespace

// ========================================================================= host ====
struct spk_stream {
    int H, W, T;
    int64_t pushed;  // steps pushed so far
    int device;
    int order_n;     // n-order tree: levels (0 for the other methods)
    int *d_carry;    // [CARRY_INTS][H*W], or the tree's [tree rows][H*W]
    int *d_ready;    // min over pixels of frames written, after the last push
    // n-order tree: the stream's pending-cut rings [H*W][pend_cap][2], and copies of the
    // carry and the rings taken before each launch (a launch that runs a ring full is rerun
    // from them with rings twice as large)
    int *d_pend, *d_carry_bak, *d_pend_bak;
    int pend_cap;
    size_t carry_bytes;
};

// Device allocations of the library go through dev_malloc, which a test hook can make fail
// (spk_debug_fail_allocations) to exercise the SPK_ERR_OOM paths without exhausting a GPU.
namespace {
std::atomic<int> g_fail_allocs{0};
std::atomic<int> g_norder_cap0{NORDER_CAP0};  // first ring size of an n-order call (test hook)
cudaError_t dev_malloc(void **p, size_t bytes) {
    int n = g_fail_allocs.load();
    while (n > 0 && !g_fail_allocs.compare_exchange_weak(n, n - 1)) {
    }
    if (n > 0) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}
template <typename T>
cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc(reinterpret_cast<void **>(p), bytes);
}
}  // namespace

struct spk_ctx {
    spk_config cfg;
    cudaStream_t stream;
    int *d_status;
    uint8_t *d_in;   // spk_reconstruct_host buffers
    size_t in_cap;
    void *d_out;
    size_t out_cap;
    int64_t launches;
    int tile;        // time tile of the frames kernels: 32, 64 or 128 steps
    // spk_reconstruct_host_async: two lanes, each a stream with its own staging buffers
    cudaStream_t lane_stream[2];
    uint8_t *lane_in[2];
    size_t lane_in_cap[2];
    void *lane_out[2];
    size_t lane_out_cap[2];
    cudaEvent_t lane_fence;  // orders the work already on `stream` before a lane's call
    int next_lane;
    int *d_pend;             // n-order tree: pending-cut rings, grown on demand
    size_t pend_bytes;
    bool pend_fixed;         // the rings live in caller-provided memory that may not grow
    char msg[512];
};

namespace {

thread_local char g_create_msg[512];

int fail(spk_ctx *ctx, int code, const char *fmt, ...) {
    char *buf = ctx ? ctx->msg : g_create_msg;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return code;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Page-locked host memory mapped into the device's address space (cudaHostAlloc, or
// cudaHostRegister with the mapped flag): its device-side address, else nullptr.  Frames
// written there by the kernel cross the host link once, with no device frame buffer and no
// separate copy.
void *mapped_host(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer || reinterpret_cast<uintptr_t>(a.devicePointer) % 16)
        return nullptr;
    return a.devicePointer;
}

int64_t pitch_of(int H, int W) {
    if (H <= 0 || W <= 0) return -1;
    int64_t P = static_cast<int64_t>(H) * W;
    return ((P + 7) / 8 + 15) / 16 * 16;
}

// bytes per frame value of an output type
size_t out_esz(int dtype) { return dtype == SPK_F16 ? 2 : dtype == SPK_U8 ? 1 : 4; }

// spk_config fields beyond the method: frame stride, output type, edge policy
const char *bad_output_cfg(const spk_config *cfg) {
    if (cfg->frame_stride < 1) return "frame_stride must be >= 1";
    if (cfg->out_dtype != SPK_F32 && cfg->out_dtype != SPK_F16 && cfg->out_dtype != SPK_U8) return "bad out_dtype";
    if (cfg->edges < 0 || cfg->edges > (SPK_ZERO_HEAD | SPK_ZERO_TAIL)) return "bad edges";
    return nullptr;
}

// 8-bit frames round theta * N / D in integers: theta must be integral, 1 .. 65535
bool u8_threshold_ok(float threshold) {
    return threshold >= 1.f && threshold <= 65535.f && threshold == std::floor(threshold);
}

// common argument checks of the stream-consuming calls
int check_stream_args(spk_ctx *ctx, const uint8_t *stream, int H, int W, int T, float threshold) {
    if (!ctx) return SPK_ERR_ARG;
    if (!stream) return fail(ctx, SPK_ERR_ARG, "stream is NULL");
    if (H <= 0 || W <= 0 || T <= 0) return fail(ctx, SPK_ERR_ARG, "H, W, T must be > 0 (got %d, %d, %d)", H, W, T);
    if (static_cast<int64_t>(H) * W > (1LL << 31) - BLOCK_PIX)
        return fail(ctx, SPK_ERR_ARG, "H*W too large");
    if (!std::isfinite(threshold) || !(threshold > 0.f))
        return fail(ctx, SPK_ERR_ARG, "threshold must be finite and > 0");
    if (ctx->cfg.out_dtype == SPK_U8 && !u8_threshold_ok(threshold))
        return fail(ctx, SPK_ERR_ARG, "8-bit frames need an integral threshold in 1 .. 65535");
    if (reinterpret_cast<uintptr_t>(stream) % 16) return fail(ctx, SPK_ERR_ARG, "stream is not 16-byte aligned");
    if (T > (1 << 30)) return fail(ctx, SPK_ERR_ARG, "T too large");
    return SPK_OK;
}

int make_tmap(spk_ctx *ctx, CUtensorMap *map, const uint8_t *stream, int64_t pitch, int rows, int tile) {
    auto enc = get_encode();
    if (!enc) return fail(ctx, SPK_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(pitch), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(pitch)};
    cuuint32_t box[2] = {ROW_BYTES, static_cast<cuuint32_t>(tile)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(stream), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, SPK_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
    return SPK_OK;
}

constexpr int MAXJ_BATCH = 96;  // jobs per launch (kernel parameters stay under 32 KB)

template <int ORDER, typename OutT, bool SEG, int MAXJ, int TT>
int launch(spk_ctx *ctx, const Batch<MAXJ> &prm, int nblocks) {
    auto kern = spk_scan_kernel<ORDER, OutT, SEG, MAXJ, TT>;
    static bool attr_set[64];  // per device, once (the first launch should precede any graph capture)
    const int dev = ctx->cfg.device;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<TT>()) != cudaSuccess)
            return fail(ctx, SPK_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(cudaGetLastError()));
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    kern<<<static_cast<unsigned>(nblocks), NTHREADS, smem_bytes<TT>(), ctx->stream>>>(prm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SPK_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    ++ctx->launches;
    return SPK_OK;
}

template <typename OutT, int MAXJ>
int launch_tfp(spk_ctx *ctx, const Batch<MAXJ> &prm, int nblocks) {
    auto kern = spk_tfp_kernel<OutT, MAXJ, TT_DEFAULT>;
    constexpr size_t bytes = sizeof(StageSmem<TT_DEFAULT>) + 128;
    kern<<<static_cast<unsigned>(nblocks), NTHREADS, bytes, ctx->stream>>>(prm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SPK_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    ++ctx->launches;
    return SPK_OK;
}

// TFI of one whole stream (one job)
template <typename OutT>
int launch_tfi(spk_ctx *ctx, const Batch<1> &prm, int nblocks) {
    auto kern = spk_tfi_kernel<OutT, TT_DEFAULT>;
    constexpr size_t bytes = sizeof(StageSmem<TT_DEFAULT>) + 128;
    kern<<<static_cast<unsigned>(nblocks), NTHREADS, bytes, ctx->stream>>>(prm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SPK_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    ++ctx->launches;
    return SPK_OK;
}

// the n-order tree runs single whole streams only (one job per launch), one kernel per
// order, so that the tree's node state is indexed by constants and stays in registers.
// (The n-order calls are synchronous and never captured in a graph.)
template <typename OutT, bool SEG, int MAXJ>
int launch_norder(spk_ctx *ctx, const Batch<MAXJ> &prm, int nblocks) {
    if constexpr (SEG && MAXJ > 1) {
        return fail(ctx, SPK_ERR_ARG, "segments are exported for one stream at a time");
    } else {
        switch (prm.jobs[0].order_n) {
            case 3: return launch<TREE_ORDER0 + 3, OutT, SEG, MAXJ, TT_DEFAULT>(ctx, prm, nblocks);
            case 4: return launch<TREE_ORDER0 + 4, OutT, SEG, MAXJ, TT_DEFAULT>(ctx, prm, nblocks);
            case 5: return launch<TREE_ORDER0 + 5, OutT, SEG, MAXJ, TT_DEFAULT>(ctx, prm, nblocks);
            default: return fail(ctx, SPK_ERR_ARG, "stability_order must be 3..5");
        }
    }
}

template <int MAXJ, int TT>
int dispatch_tile(spk_ctx *ctx, const Batch<MAXJ> &prm, int nblocks) {
    const int m = ctx->cfg.method;
    if (ctx->cfg.out_dtype == SPK_F16)
        return m == SPK_FSR ? launch<1, __half, false, MAXJ, TT>(ctx, prm, nblocks)
                            : launch<2, __half, false, MAXJ, TT>(ctx, prm, nblocks);
    return m == SPK_FSR ? launch<1, float, false, MAXJ, TT>(ctx, prm, nblocks)
                        : launch<2, float, false, MAXJ, TT>(ctx, prm, nblocks);
}

// 8-bit frames: every method in the default tile
template <int MAXJ>
int dispatch_u8(spk_ctx *ctx, const Batch<MAXJ> &prm, int nblocks) {
    switch (ctx->cfg.method) {
        case SPK_FSR: return launch<1, uint8_t, false, MAXJ, TT_DEFAULT>(ctx, prm, nblocks);
        case SPK_TFI:
            if constexpr (MAXJ == 1) return launch_tfi<uint8_t>(ctx, prm, nblocks);
            else return launch<3, uint8_t, false, MAXJ, TT_DEFAULT>(ctx, prm, nblocks);
        case SPK_TFP: return launch_tfp<uint8_t, MAXJ>(ctx, prm, nblocks);
        case SPK_NORDER: return launch_norder<uint8_t, false>(ctx, prm, nblocks);
        default: return launch<2, uint8_t, false, MAXJ, TT_DEFAULT>(ctx, prm, nblocks);
    }
}

// FSR / SSR frames kernels come in three time tiles (the autotuner's choice); TFI, TFP,
// 8-bit frames and the verification kernel in the default tile only
template <int MAXJ>
int dispatch(spk_ctx *ctx, const Batch<MAXJ> &prm, int nblocks, bool segments, int tile) {
    const int m = ctx->cfg.method;
    const bool f16 = ctx->cfg.out_dtype == SPK_F16;
    if (!segments && ctx->cfg.out_dtype == SPK_U8) return dispatch_u8(ctx, prm, nblocks);
    if (segments)
        return m == SPK_FSR      ? launch<1, float, true, MAXJ, TT_DEFAULT>(ctx, prm, nblocks)
             : m == SPK_TFI      ? launch<3, float, true, MAXJ, TT_DEFAULT>(ctx, prm, nblocks)
             : m == SPK_NORDER   ? launch_norder<float, true>(ctx, prm, nblocks)
                                 : launch<2, float, true, MAXJ, TT_DEFAULT>(ctx, prm, nblocks);
    if (m == SPK_NORDER)
        return f16 ? launch_norder<__half, false>(ctx, prm, nblocks) : launch_norder<float, false>(ctx, prm, nblocks);
    if (m == SPK_TFI) {  // one whole stream: the streaming TFI kernel; batches and pieces: the scan
        if constexpr (MAXJ == 1)
            return f16 ? launch_tfi<__half>(ctx, prm, nblocks) : launch_tfi<float>(ctx, prm, nblocks);
        else
            return f16 ? launch<3, __half, false, MAXJ, TT_DEFAULT>(ctx, prm, nblocks)
                       : launch<3, float, false, MAXJ, TT_DEFAULT>(ctx, prm, nblocks);
    }
    if (m == SPK_TFP)
        return f16 ? launch_tfp<__half, MAXJ>(ctx, prm, nblocks) : launch_tfp<float, MAXJ>(ctx, prm, nblocks);
    if (tile == 32) return dispatch_tile<MAXJ, 32>(ctx, prm, nblocks);
    if (tile == 128) return dispatch_tile<MAXJ, 128>(ctx, prm, nblocks);
    return dispatch_tile<MAXJ, 64>(ctx, prm, nblocks);
}

// the tile a call will use: the context's for FSR / SSR frames of 4 or 2 bytes, the
// default for the others
int tile_of(const spk_ctx *ctx, bool segments) {
    const int m = ctx->cfg.method;
    return (segments || m == SPK_TFI || m == SPK_TFP || m == SPK_NORDER || ctx->cfg.out_dtype == SPK_U8)
               ? TT_DEFAULT : ctx->tile;
}

bool valid_method(const spk_config *cfg) {
    if (cfg->method < SPK_FSR || cfg->method > SPK_NORDER) return false;
    if (cfg->method == SPK_NORDER) return cfg->stability_order >= spk::TREE_MIN && cfg->stability_order <= spk::TREE_MAX;
    return cfg->method != SPK_TFP || (cfg->tfp_window >= 1 && cfg->tfp_window <= 64);
}

// one job's kernel parameters; returns its block count (or a negative error)
int fill_job(spk_ctx *ctx, CUtensorMap *map, Job *job, const uint8_t *stream, int H, int W, int n, int t_base,
             int T, float threshold, void *out, int *carry, int *ready, int flags, int block0, int tile) {
    const int64_t P = static_cast<int64_t>(H) * W;
    int rc = make_tmap(ctx, map, stream, pitch_of(H, W), n, tile);
    if (rc) return rc;
    *job = Job{};
    job->P = P;
    job->out = out;
    job->carry = carry;
    job->ready = ready;
    job->n = n;
    job->ntiles = (n + tile - 1) / tile;
    job->t_base = t_base;
    job->stride = ctx->cfg.frame_stride;
    job->T_out = static_cast<int>((static_cast<int64_t>(T) + job->stride - 1) / job->stride);
    if (job->stride >= 2) {  // t / d = floor(m t / 2^(31 + l)), l = ceil(log2 d), m = ceil(2^(31+l) / d)
        int l = 0;
        while ((1LL << l) < job->stride) ++l;
        const unsigned long long m =
            ((1ULL << (31 + l)) + job->stride - 1) / static_cast<unsigned long long>(job->stride);
        job->div_m = static_cast<uint32_t>(m);
        job->div_s = l - 1;
    }
    job->theta = threshold;
    job->window = ctx->cfg.tfp_window;
    job->order_n = ctx->cfg.stability_order;
    job->edges = ctx->cfg.edges;
    job->flags = flags;
    job->block0 = block0;
    return static_cast<int>((P + BLOCK_PIX - 1) / BLOCK_PIX);
}

// The n-order tree holds cuts that are not final yet in a per-pixel ring: for whole streams
// in the context's rings (npix pixels over the launch's jobs, each job's from its pend_px
// on), for a piece of a live stream (live[k] != nullptr) in the stream's own rings, which
// carry pending cuts from piece to piece.  A pixel whose ring runs full reports it; the
// launch then runs again with rings twice as large: whole streams from scratch, live streams
// from copies of their carried state and rings taken before the launch (the pending cuts
// moved into the larger rings), so every valid stream is reconstructed (at most T + 1
// cuts can be pending).  Synchronous.
template <int MAXJ>
int run_norder(spk_ctx *ctx, Batch<MAXJ> &prm, int nblocks, bool segments, int64_t npix, int T_max,
               spk_stream *const *live = nullptr) {
    for (int k = 0; live && k < prm.njobs; ++k) {
        spk_stream *st = live[k];
        if (!st || (prm.jobs[k].flags & JOB_FIRST)) continue;
        const size_t ring = static_cast<size_t>(st->H) * st->W * 2 * st->pend_cap * sizeof(int);
        if (cudaMemcpyAsync(st->d_carry_bak, st->d_carry, st->carry_bytes, cudaMemcpyDeviceToDevice, ctx->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(st->d_pend_bak, st->d_pend, ring, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
            return fail(ctx, SPK_ERR_CUDA, "copy of a live stream's state failed");
    }
    int pcap = g_norder_cap0.load();
    for (;;) {
        const size_t need = static_cast<size_t>(2) * static_cast<size_t>(pcap) * static_cast<size_t>(npix) * sizeof(int);
        if (need > ctx->pend_bytes) {
            if (ctx->pend_fixed)
                return fail(ctx, SPK_ERR_INTERNAL, "n-order pending cuts need %zu bytes of rings, %zu available", need,
                            ctx->pend_bytes);
            if (ctx->d_pend) cudaFree(ctx->d_pend);
            ctx->d_pend = nullptr;
            ctx->pend_bytes = 0;
            if (dev_malloc(&ctx->d_pend, need) != cudaSuccess) {
                cudaGetLastError();
                return fail(ctx, SPK_ERR_OOM, "cudaMalloc(%zu) of the n-order pending-cut rings failed", need);
            }
            ctx->pend_bytes = need;
        }
        for (int k = 0; k < prm.njobs; ++k) {
            spk_stream *st = live ? live[k] : nullptr;
            prm.jobs[k].pend = st ? st->d_pend : ctx->d_pend + prm.jobs[k].pend_px * 2 * pcap;
            prm.jobs[k].pend_cap = st ? st->pend_cap : pcap;
        }
        int rc = dispatch(ctx, prm, nblocks, segments, TT_DEFAULT);
        if (rc) return rc;
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return fail(ctx, SPK_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
        int st = 0;
        if (cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(ctx, SPK_ERR_CUDA, "status read failed");
        if (st != DEV_PEND_FULL) return SPK_OK;  // done, or another failure for spk_synchronize to report
        if (static_cast<int64_t>(pcap) > T_max) return fail(ctx, SPK_ERR_INTERNAL, "n-order pending cuts exceed T");
        if (cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess)
            return fail(ctx, SPK_ERR_CUDA, "status reset failed");
        pcap *= 2;
        // every live stream of the launch: rings twice as large, filled from the copies, and
        // the carried state restored
        for (int k = 0; live && k < prm.njobs; ++k) {
            spk_stream *ls = live[k];
            if (!ls) continue;
            const int64_t P = static_cast<int64_t>(ls->H) * ls->W;
            const int ncap = 2 * ls->pend_cap;
            const size_t ring = static_cast<size_t>(P) * 2 * ncap * sizeof(int);
            int *nr = nullptr, *nb = nullptr;
            if (dev_malloc(&nr, ring) != cudaSuccess || dev_malloc(&nb, ring) != cudaSuccess) {
                cudaGetLastError();
                cudaFree(nr);
                return fail(ctx, SPK_ERR_OOM, "cudaMalloc(%zu) of a live stream's pending-cut rings failed", ring);
            }
            if (!(prm.jobs[k].flags & JOB_FIRST)) {
                tree_ring_grow_kernel<<<static_cast<unsigned>(std::min<int64_t>((P + 255) / 256, 4096)), 256, 0,
                                        ctx->stream>>>(ls->d_pend_bak, ls->pend_cap, nr, ncap, ls->d_carry_bak, P);
                if (cudaGetLastError() != cudaSuccess ||
                    cudaMemcpyAsync(ls->d_carry, ls->d_carry_bak, ls->carry_bytes, cudaMemcpyDeviceToDevice,
                                    ctx->stream) != cudaSuccess ||
                    cudaMemcpyAsync(nb, nr, ring, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) {
                    cudaFree(nr);
                    cudaFree(nb);
                    return fail(ctx, SPK_ERR_CUDA, "regrowth of a live stream's rings failed");
                }
                ++ctx->launches;
            }
            if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
                cudaFree(nr);
                cudaFree(nb);
                return fail(ctx, SPK_ERR_CUDA, "regrowth of a live stream's rings failed");
            }
            cudaFree(ls->d_pend);
            cudaFree(ls->d_pend_bak);
            ls->d_pend = nr;
            ls->d_pend_bak = nb;
            ls->pend_cap = ncap;
        }
    }
}

int run_scan(spk_ctx *ctx, const uint8_t *stream, int H, int W, int T, float threshold, void *out,
             int32_t *spikes, int32_t *counts, int32_t *ts, int32_t *te, int32_t *n, float *v, int cap,
             bool segments) {
    if (cudaSetDevice(ctx->cfg.device) != cudaSuccess) return fail(ctx, SPK_ERR_CUDA, "cudaSetDevice failed");
    Batch<1> prm{};
    const int tile = tile_of(ctx, segments);
    const int nb = fill_job(ctx, &prm.maps[0], &prm.jobs[0], stream, H, W, T, 0, T, threshold, out, nullptr,
                            nullptr, JOB_FIRST | JOB_LAST, 0, tile);
    if (nb < 0) return nb;
    prm.njobs = 1;
    prm.status = ctx->d_status;
    prm.spikes = spikes;
    prm.counts = counts;
    prm.seg_ts = ts;
    prm.seg_te = te;
    prm.seg_n = n;
    prm.seg_v = v;
    prm.cap = cap;
    if (ctx->cfg.method != SPK_NORDER) return dispatch(ctx, prm, nb, segments, tile);
    return run_norder(ctx, prm, nb, segments, static_cast<int64_t>(H) * W, T);
}

void stream_free(spk_stream *st) {
    cudaFree(st->d_carry);
    cudaFree(st->d_ready);
    cudaFree(st->d_pend);
    cudaFree(st->d_carry_bak);
    cudaFree(st->d_pend_bak);
    delete st;
}

// rows of carried state per pixel of an n-order tree stream (the kernel's tree type)
int tree_carry_rows_of(int n) {
    switch (n) {
        case 3: return tree_carry_rows<spk::TreeScan<3, 3 < TREE_REG_LEVELS ? 3 : TREE_REG_LEVELS>>();
        case 4: return tree_carry_rows<spk::TreeScan<4, 4 < TREE_REG_LEVELS ? 4 : TREE_REG_LEVELS>>();
        default: return tree_carry_rows<spk::TreeScan<5, 5 < TREE_REG_LEVELS ? 5 : TREE_REG_LEVELS>>();
    }
}

bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

}  // namespace

extern "C" {

int64_t spk_pitch(int H, int W) { return pitch_of(H, W); }

int64_t spk_num_frames(int T, int stride) {
    if (T <= 0 || stride <= 0) return -1;
    return (static_cast<int64_t>(T) + stride - 1) / stride;
}

int spk_create(spk_ctx **out, const spk_config *cfg) {
    if (!out) return fail(nullptr, SPK_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, SPK_ERR_ARG, "cfg is NULL");
    if (!valid_method(cfg)) return fail(nullptr, SPK_ERR_ARG, "method must be 1..5 (TFP: tfp_window 1..64; NORDER: stability_order 3..5)");
    if (const char *why = bad_output_cfg(cfg)) return fail(nullptr, SPK_ERR_ARG, "%s", why);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, SPK_ERR_CUDA, "no CUDA device");
    }
    if (cfg->device < 0 || cfg->device >= ndev) return fail(nullptr, SPK_ERR_ARG, "bad device ordinal");
    if (cudaSetDevice(cfg->device) != cudaSuccess) return fail(nullptr, SPK_ERR_CUDA, "cudaSetDevice failed");
    spk_ctx *c = new (std::nothrow) spk_ctx();
    if (!c) return fail(nullptr, SPK_ERR_OOM, "host allocation failed");
    c->cfg = *cfg;
    c->stream = static_cast<cudaStream_t>(cfg->stream);
    c->tile = TT_DEFAULT;
    if (dev_malloc(&c->d_status, 16) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(nullptr, SPK_ERR_OOM, "cudaMalloc of the status word failed");
    }
    if (cudaMemset(c->d_status, 0, 16) != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return fail(nullptr, SPK_ERR_CUDA, "cudaMemset failed");
    }
    *out = c;
    return SPK_OK;
}

int spk_destroy(spk_ctx *ctx) {
    if (!ctx) return SPK_OK;
    cudaSetDevice(ctx->cfg.device);
    cudaStreamSynchronize(ctx->stream);
    for (int l = 0; l < 2; ++l) {
        if (ctx->lane_stream[l]) {
            cudaStreamSynchronize(ctx->lane_stream[l]);
            cudaStreamDestroy(ctx->lane_stream[l]);
        }
        if (ctx->lane_in[l]) cudaFree(ctx->lane_in[l]);
        if (ctx->lane_out[l]) cudaFree(ctx->lane_out[l]);
    }
    if (ctx->lane_fence) cudaEventDestroy(ctx->lane_fence);
    cudaFree(ctx->d_status);
    if (ctx->d_in) cudaFree(ctx->d_in);
    if (ctx->d_out) cudaFree(ctx->d_out);
    if (ctx->d_pend) cudaFree(ctx->d_pend);
    delete ctx;
    return SPK_OK;
}

const char *spk_last_error(const spk_ctx *ctx) { return ctx ? ctx->msg : g_create_msg; }

int64_t spk_launch_count(const spk_ctx *ctx) { return ctx ? ctx->launches : 0; }

int spk_reconstruct(spk_ctx *ctx, const uint8_t *stream, int H, int W, int T, float threshold, void *out_frames) {
    int rc = check_stream_args(ctx, stream, H, W, T, threshold);
    if (rc) return rc;
    ctx->msg[0] = 0;
    if (!out_frames) return fail(ctx, SPK_ERR_ARG, "out_frames is NULL");
    if (reinterpret_cast<uintptr_t>(out_frames) % 16) return fail(ctx, SPK_ERR_ARG, "out_frames is not 16-byte aligned");
    const int64_t P = static_cast<int64_t>(H) * W;
    const int64_t T_out = spk_num_frames(T, ctx->cfg.frame_stride);
    const size_t esz = out_esz(ctx->cfg.out_dtype);
    const size_t out_bytes = static_cast<size_t>(T_out) * static_cast<size_t>(P) * esz;
    const size_t in_bytes = static_cast<size_t>(T) * static_cast<size_t>(pitch_of(H, W));
    if (overlaps(stream, in_bytes, out_frames, out_bytes)) return fail(ctx, SPK_ERR_ARG, "out_frames overlaps stream");
    if (!is_device_ptr(stream) || !is_device_ptr(out_frames))
        return fail(ctx, SPK_ERR_ARG, "stream and out_frames must be device memory");
    return run_scan(ctx, stream, H, W, T, threshold, out_frames, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0,
                    false);
}

int spk_segments(spk_ctx *ctx, const uint8_t *stream, int H, int W, int T, float threshold, int32_t *spike_counts,
                 int32_t *counts, int32_t *t_start, int32_t *t_end, int32_t *n_int, float *value, int cap) {
    int rc = check_stream_args(ctx, stream, H, W, T, threshold);
    if (rc) return rc;
    ctx->msg[0] = 0;
    if (ctx->cfg.method == SPK_TFP) return fail(ctx, SPK_ERR_ARG, "TFP has no stable spans");
    if (!counts || cap < 0) return fail(ctx, SPK_ERR_ARG, "counts is NULL or cap < 0");
    if (cap > 0 && (!t_start || !t_end || !n_int || !value)) return fail(ctx, SPK_ERR_ARG, "segment arrays are NULL");
    if (!is_device_ptr(stream) || !is_device_ptr(counts) || (spike_counts && !is_device_ptr(spike_counts)))
        return fail(ctx, SPK_ERR_ARG, "pointers must be device memory");
    if (cap > 0 && (!is_device_ptr(t_start) || !is_device_ptr(t_end) || !is_device_ptr(n_int) || !is_device_ptr(value)))
        return fail(ctx, SPK_ERR_ARG, "pointers must be device memory");
    return run_scan(ctx, stream, H, W, T, threshold, nullptr, spike_counts, counts, t_start, t_end, n_int, value, cap,
                    true);
}

int spk_synchronize(spk_ctx *ctx) {
    if (!ctx) return SPK_ERR_ARG;
    cudaSetDevice(ctx->cfg.device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    for (int l = 0; l < 2 && e == cudaSuccess; ++l)
        if (ctx->lane_stream[l]) e = cudaStreamSynchronize(ctx->lane_stream[l]);
    if (e != cudaSuccess) return fail(ctx, SPK_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
    int st = 0;
    if (cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(ctx, SPK_ERR_CUDA, "status read failed");
    if (st) {
        cudaMemset(ctx->d_status, 0, sizeof(int));
        if (st & DEV_TIMEOUT) return fail(ctx, SPK_ERR_TIMEOUT, "a bounded device wait gave up");
        return fail(ctx, SPK_ERR_INTERNAL, "device consistency check failed (status %d)", st);
    }
    return SPK_OK;
}

int spk_stream_open(spk_ctx *ctx, int H, int W, int T, spk_stream **out) {
    if (!ctx) return SPK_ERR_ARG;
    ctx->msg[0] = 0;
    if (!out) return fail(ctx, SPK_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (ctx->cfg.method == SPK_TFP) return fail(ctx, SPK_ERR_ARG, "TFP runs whole streams only");
    if (H <= 0 || W <= 0 || T <= 0 || T > (1 << 30)) return fail(ctx, SPK_ERR_ARG, "bad H, W or T");
    if (static_cast<int64_t>(H) * W > (1LL << 31) - BLOCK_PIX) return fail(ctx, SPK_ERR_ARG, "H*W too large");
    if (cudaSetDevice(ctx->cfg.device) != cudaSuccess) return fail(ctx, SPK_ERR_CUDA, "cudaSetDevice failed");
    spk_stream *st = new (std::nothrow) spk_stream();
    if (!st) return fail(ctx, SPK_ERR_OOM, "host allocation failed");
    st->H = H;
    st->W = W;
    st->T = T;
    st->device = ctx->cfg.device;
    const size_t P = static_cast<size_t>(H) * static_cast<size_t>(W);
    const bool tree = ctx->cfg.method == SPK_NORDER;
    st->order_n = tree ? ctx->cfg.stability_order : 0;
    st->carry_bytes = static_cast<size_t>(tree ? tree_carry_rows_of(st->order_n) : CARRY_INTS) * P * 4;
    st->pend_cap = tree ? g_norder_cap0.load() : 0;
    const size_t ring_bytes = P * 2 * static_cast<size_t>(st->pend_cap) * sizeof(int);
    bool ok = dev_malloc(&st->d_carry, st->carry_bytes) == cudaSuccess &&
              dev_malloc(&st->d_ready, sizeof(int)) == cudaSuccess;
    if (ok && tree)
        ok = dev_malloc(&st->d_carry_bak, st->carry_bytes) == cudaSuccess &&
             dev_malloc(&st->d_pend, ring_bytes) == cudaSuccess && dev_malloc(&st->d_pend_bak, ring_bytes) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        stream_free(st);
        return fail(ctx, SPK_ERR_OOM, "cudaMalloc of the stream state failed");
    }
    if (cudaMemsetAsync(st->d_ready, 0, sizeof(int), ctx->stream) != cudaSuccess) {
        stream_free(st);
        return fail(ctx, SPK_ERR_CUDA, "cudaMemsetAsync failed");
    }
    *out = st;
    return SPK_OK;
}

int spk_stream_close(spk_ctx *ctx, spk_stream *s) {
    if (!s) return SPK_OK;
    if (ctx) {
        cudaSetDevice(ctx->cfg.device);
        cudaStreamSynchronize(ctx->stream);
    }
    stream_free(s);
    return SPK_OK;
}

int64_t spk_stream_steps(const spk_stream *s) { return s ? s->pushed : -1; }

int spk_stream_ready(spk_ctx *ctx, const spk_stream *s, int64_t *ready) {
    if (!ctx || !s || !ready) return ctx ? fail(ctx, SPK_ERR_ARG, "NULL argument") : SPK_ERR_ARG;
    cudaSetDevice(ctx->cfg.device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(ctx, SPK_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
    int r = 0;
    if (cudaMemcpy(&r, s->d_ready, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(ctx, SPK_ERR_CUDA, "ready read failed");
    *ready = r;
    return SPK_OK;
}

int spk_run(spk_ctx *ctx, const spk_job *jobs, int njobs) {
    if (!ctx) return SPK_ERR_ARG;
    ctx->msg[0] = 0;
    if (njobs < 0 || (njobs > 0 && !jobs)) return fail(ctx, SPK_ERR_ARG, "bad job list");
    const size_t esz = out_esz(ctx->cfg.out_dtype);
    for (int k = 0; k < njobs; ++k) {  // validate everything before any launch
        const spk_job &jb = jobs[k];
        int rc = check_stream_args(ctx, jb.stream, jb.H, jb.W, jb.n, jb.threshold);
        if (rc) return rc;
        if (!jb.out_frames || reinterpret_cast<uintptr_t>(jb.out_frames) % 16)
            return fail(ctx, SPK_ERR_ARG, "job %d: out_frames is NULL or not 16-byte aligned", k);
        const int T = jb.state ? jb.state->T : jb.n;
        const size_t out_bytes = static_cast<size_t>(spk_num_frames(T, ctx->cfg.frame_stride)) *
                                 static_cast<size_t>(jb.H) * static_cast<size_t>(jb.W) * esz;
        const size_t in_bytes = static_cast<size_t>(jb.n) * static_cast<size_t>(pitch_of(jb.H, jb.W));
        if (overlaps(jb.stream, in_bytes, jb.out_frames, out_bytes))
            return fail(ctx, SPK_ERR_ARG, "job %d: out_frames overlaps its stream", k);
        if (!is_device_ptr(jb.stream) || !is_device_ptr(jb.out_frames))
            return fail(ctx, SPK_ERR_ARG, "job %d: stream and out_frames must be device memory", k);
        if (jb.state) {
            if (ctx->cfg.method == SPK_TFP) return fail(ctx, SPK_ERR_ARG, "TFP runs whole streams only");
            if (jb.state->order_n != (ctx->cfg.method == SPK_NORDER ? ctx->cfg.stability_order : 0))
                return fail(ctx, SPK_ERR_ARG, "job %d: stream opened for another method", k);
            if (jb.state->H != jb.H || jb.state->W != jb.W) return fail(ctx, SPK_ERR_ARG, "job %d: H, W differ from its stream", k);
            if (jb.state->pushed + jb.n > jb.state->T) return fail(ctx, SPK_ERR_ARG, "job %d: piece runs past the stream's T", k);
            if (jb.state->device != ctx->cfg.device) return fail(ctx, SPK_ERR_ARG, "job %d: stream on another device", k);
            for (int m = 0; m < k; ++m)
                if (jobs[m].state == jb.state) return fail(ctx, SPK_ERR_ARG, "jobs %d and %d push the same stream", m, k);
        }
    }
    if (cudaSetDevice(ctx->cfg.device) != cudaSuccess) return fail(ctx, SPK_ERR_CUDA, "cudaSetDevice failed");
    Batch<MAXJ_BATCH> *prm = new (std::nothrow) Batch<MAXJ_BATCH>();
    int *order = static_cast<int *>(malloc(sizeof(int) * (njobs > 0 ? njobs : 1)));
    if (!prm || !order) {
        delete prm;
        free(order);
        return fail(ctx, SPK_ERR_OOM, "host allocation failed");
    }
    // longest pieces first: their blocks take longest, so they should start first
    for (int k = 0; k < njobs; ++k) order[k] = k;
    for (int k = 1; k < njobs; ++k) {
        const int x = order[k];
        int m = k;
        while (m > 0 && jobs[order[m - 1]].n < jobs[x].n) {
            order[m] = order[m - 1];
            --m;
        }
        order[m] = x;
    }
    int rc = SPK_OK;
    for (int k0 = 0; k0 < njobs && rc == SPK_OK; k0 += MAXJ_BATCH) {
        const int nj = njobs - k0 < MAXJ_BATCH ? njobs - k0 : MAXJ_BATCH;
        int blocks = 0, T_max = 0;
        int64_t npix = 0;
        spk_stream *live[MAXJ_BATCH];
        for (int k = 0; k < nj && rc == SPK_OK; ++k) {
            const spk_job &jb = jobs[order[k0 + k]];
            spk_stream *st = jb.state;
            int flags = JOB_FIRST | JOB_LAST, t_base = 0, T = jb.n;
            if (st) {
                t_base = static_cast<int>(st->pushed);
                T = st->T;
                flags = (st->pushed == 0 ? JOB_FIRST : 0) | (st->pushed + jb.n == st->T ? JOB_LAST : 0);
                if (cudaMemsetAsync(st->d_ready, 0x7f, sizeof(int), ctx->stream) != cudaSuccess)
                    rc = fail(ctx, SPK_ERR_CUDA, "cudaMemsetAsync failed");
            }
            const int nb = fill_job(ctx, &prm->maps[k], &prm->jobs[k], jb.stream, jb.H, jb.W, jb.n, t_base, T,
                                    jb.threshold, jb.out_frames, st ? st->d_carry : nullptr,
                                    st ? st->d_ready : nullptr, flags, blocks, tile_of(ctx, false));
            if (nb < 0) {
                rc = nb;
            } else {
                blocks += nb;
                live[k] = st;
                if (!st) {  // the n-order tree's rings of whole streams, job after job
                    prm->jobs[k].pend_px = npix;
                    npix += static_cast<int64_t>(jb.H) * jb.W;
                }
                if (T > T_max) T_max = T;
            }
        }
        if (rc) break;
        prm->njobs = nj;
        prm->status = ctx->d_status;
        rc = ctx->cfg.method == SPK_NORDER ? run_norder(ctx, *prm, blocks, false, npix, T_max, live)
                                           : dispatch(ctx, *prm, blocks, false, tile_of(ctx, false));
        if (rc == SPK_OK)
            for (int k = 0; k < nj; ++k)
                if (jobs[order[k0 + k]].state) jobs[order[k0 + k]].state->pushed += jobs[order[k0 + k]].n;
    }
    delete prm;
    free(order);
    return rc;
}

int spk_set_tile(spk_ctx *ctx, int tile) {
    if (!ctx) return SPK_ERR_ARG;
    if (tile != 32 && tile != 64 && tile != 128) return fail(ctx, SPK_ERR_ARG, "tile must be 32, 64 or 128");
    ctx->tile = tile;
    return SPK_OK;
}

int spk_get_tile(const spk_ctx *ctx) { return ctx ? ctx->tile : -1; }

int spk_autotune(spk_ctx *ctx, const spk_job *jobs, int njobs, int *best_tile) {
    if (!ctx) return SPK_ERR_ARG;
    ctx->msg[0] = 0;
    for (int k = 0; k < njobs; ++k)
        if (jobs[k].state) return fail(ctx, SPK_ERR_ARG, "autotune runs jobs repeatedly: whole streams only");
    cudaSetDevice(ctx->cfg.device);
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
        return fail(ctx, SPK_ERR_CUDA, "cudaEventCreate failed");
    const int tiles[3] = {32, 64, 128};
    float best_ms = -1.f;
    int best = ctx->tile, rc = SPK_OK;
    for (int m = 0; m < 3 && rc == SPK_OK; ++m) {
        ctx->tile = tiles[m];
        rc = spk_run(ctx, jobs, njobs);  // warm-up
        if (rc) break;
        cudaEventRecord(a, ctx->stream);
        for (int r = 0; r < 3 && rc == SPK_OK; ++r) rc = spk_run(ctx, jobs, njobs);
        cudaEventRecord(b, ctx->stream);
        if (cudaEventSynchronize(b) != cudaSuccess) rc = fail(ctx, SPK_ERR_CUDA, "autotune run failed");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rc == SPK_OK && (best_ms < 0.f || ms < best_ms)) {
            best_ms = ms;
            best = tiles[m];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->tile = best;
    if (best_tile) *best_tile = best;
    if (rc == SPK_OK) rc = spk_synchronize(ctx);
    return rc;
}

int spk_features(spk_ctx *ctx, const uint8_t *stream, int H, int W, int T, float threshold, const float *plain,
                 void *x0) {
    int rc = check_stream_args(ctx, stream, H, W, T, threshold);
    if (rc) return rc;
    ctx->msg[0] = 0;
    if (!plain || !x0 || reinterpret_cast<uintptr_t>(x0) % 16 || reinterpret_cast<uintptr_t>(plain) % 4)
        return fail(ctx, SPK_ERR_ARG, "plain or x0 is NULL or misaligned");
    if (!is_device_ptr(stream) || !is_device_ptr(plain) || !is_device_ptr(x0))
        return fail(ctx, SPK_ERR_ARG, "pointers must be device memory");
    if (cudaSetDevice(ctx->cfg.device) != cudaSuccess) return fail(ctx, SPK_ERR_CUDA, "cudaSetDevice failed");
    Batch<1> prm{};
    const int nb = fill_job(ctx, &prm.maps[0], &prm.jobs[0], stream, H, W, T, 0, T, threshold, nullptr, nullptr,
                            nullptr, JOB_FIRST | JOB_LAST, 0, TT_DEFAULT);
    if (nb < 0) return nb;
    prm.njobs = 1;
    prm.status = ctx->d_status;
    constexpr size_t bytes = sizeof(StageSmem<TT_DEFAULT>) + 128;
    spk_feature_kernel<TT_DEFAULT><<<nb, NTHREADS, bytes, ctx->stream>>>(prm, plain,
                                                                          static_cast<__nv_bfloat16 *>(x0), H, W);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SPK_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    ++ctx->launches;
    return SPK_OK;
}

int spk_selftest_wait(spk_ctx *ctx, int64_t limit_cycles) {
    if (!ctx) return SPK_ERR_ARG;
    ctx->msg[0] = 0;
    if (limit_cycles < 0 || limit_cycles > WAIT_CYCLES) return fail(ctx, SPK_ERR_ARG, "limit_cycles out of range");
    cudaSetDevice(ctx->cfg.device);
    wait_selftest_kernel<<<1, 32, 0, ctx->stream>>>(ctx->d_status, static_cast<long long>(limit_cycles));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SPK_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    ++ctx->launches;
    return SPK_OK;
}

int spk_reconstruct_host(spk_ctx *ctx, const uint8_t *host_stream, int H, int W, int T, float threshold,
                         void *host_frames) {
    int rc = check_stream_args(ctx, host_stream, H, W, T, threshold);
    if (rc) return rc;
    ctx->msg[0] = 0;
    if (!host_frames) return fail(ctx, SPK_ERR_ARG, "host_frames is NULL");
    const int64_t P = static_cast<int64_t>(H) * W;
    const int64_t T_out = spk_num_frames(T, ctx->cfg.frame_stride);
    const size_t esz = out_esz(ctx->cfg.out_dtype);
    const size_t out_bytes = static_cast<size_t>(T_out) * static_cast<size_t>(P) * esz;
    const size_t in_bytes = static_cast<size_t>(T) * static_cast<size_t>(pitch_of(H, W));
    cudaSetDevice(ctx->cfg.device);
    // pinned frames: the kernel writes them in place, so no copy waits for the scan to end
    // (one call: 7.8 -> 5.9 ms on the 250x400x20000 stream)
    void *direct = mapped_host(host_frames);
    if (in_bytes > ctx->in_cap) {
        if (ctx->d_in) cudaFree(ctx->d_in);
        ctx->d_in = nullptr;
        ctx->in_cap = 0;
        if (dev_malloc(&ctx->d_in, in_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, SPK_ERR_OOM, "cudaMalloc(%zu) failed", in_bytes);
        }
        ctx->in_cap = in_bytes;
    }
    if (!direct && out_bytes > ctx->out_cap) {
        if (ctx->d_out) cudaFree(ctx->d_out);
        ctx->d_out = nullptr;
        ctx->out_cap = 0;
        if (dev_malloc(&ctx->d_out, out_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, SPK_ERR_OOM, "cudaMalloc(%zu) failed", out_bytes);
        }
        ctx->out_cap = out_bytes;
    }
    if (cudaMemcpyAsync(ctx->d_in, host_stream, in_bytes, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        return fail(ctx, SPK_ERR_CUDA, "H2D copy: %s", cudaGetErrorString(cudaGetLastError()));
    rc = run_scan(ctx, ctx->d_in, H, W, T, threshold, direct ? direct : ctx->d_out, nullptr, nullptr, nullptr,
                  nullptr, nullptr, nullptr, 0, false);
    if (rc) return rc;
    if (!direct &&
        cudaMemcpyAsync(host_frames, ctx->d_out, out_bytes, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
        return fail(ctx, SPK_ERR_CUDA, "D2H copy: %s", cudaGetErrorString(cudaGetLastError()));
    return spk_synchronize(ctx);
}

int spk_debug_fail_allocations(int n) {
    if (n < 0) return SPK_ERR_ARG;
    g_fail_allocs.store(n);
    return SPK_OK;
}

int spk_debug_norder_capacity(int cap) {
    if (cap < 0 || (cap & (cap - 1))) return SPK_ERR_ARG;
    g_norder_cap0.store(cap ? cap : NORDER_CAP0);
    return SPK_OK;
}

int spk_reconstruct_host_async(spk_ctx *ctx, const uint8_t *host_stream, int H, int W, int T, float threshold,
                               void *host_frames) {
    int rc = check_stream_args(ctx, host_stream, H, W, T, threshold);
    if (rc) return rc;
    ctx->msg[0] = 0;
    if (!host_frames) return fail(ctx, SPK_ERR_ARG, "host_frames is NULL");
    const int64_t P = static_cast<int64_t>(H) * W;
    const int64_t T_out = spk_num_frames(T, ctx->cfg.frame_stride);
    const size_t esz = out_esz(ctx->cfg.out_dtype);
    const size_t out_bytes = static_cast<size_t>(T_out) * static_cast<size_t>(P) * esz;
    const size_t in_bytes = static_cast<size_t>(T) * static_cast<size_t>(pitch_of(H, W));
    cudaSetDevice(ctx->cfg.device);
    const int l = ctx->next_lane;
    if (!ctx->lane_stream[l] && cudaStreamCreateWithFlags(&ctx->lane_stream[l], cudaStreamNonBlocking) != cudaSuccess)
        return fail(ctx, SPK_ERR_CUDA, "cudaStreamCreate failed");
    if (!ctx->lane_fence && cudaEventCreateWithFlags(&ctx->lane_fence, cudaEventDisableTiming) != cudaSuccess)
        return fail(ctx, SPK_ERR_CUDA, "cudaEventCreate failed");
    cudaStream_t ls = ctx->lane_stream[l];
    // (frames always go through the lane's device buffer and a copy-engine copy: written by the
    // kernel over the host link they would hold the SMs of the next call's scan)
    // a lane's buffers grow on demand; cudaFree waits for the lane's earlier work
    if (in_bytes > ctx->lane_in_cap[l]) {
        if (ctx->lane_in[l]) cudaFree(ctx->lane_in[l]);
        ctx->lane_in[l] = nullptr;
        ctx->lane_in_cap[l] = 0;
        if (dev_malloc(&ctx->lane_in[l], in_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, SPK_ERR_OOM, "cudaMalloc(%zu) failed", in_bytes);
        }
        ctx->lane_in_cap[l] = in_bytes;
    }
    if (out_bytes > ctx->lane_out_cap[l]) {
        if (ctx->lane_out[l]) cudaFree(ctx->lane_out[l]);
        ctx->lane_out[l] = nullptr;
        ctx->lane_out_cap[l] = 0;
        if (dev_malloc(&ctx->lane_out[l], out_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, SPK_ERR_OOM, "cudaMalloc(%zu) failed", out_bytes);
        }
        ctx->lane_out_cap[l] = out_bytes;
    }
    if (cudaEventRecord(ctx->lane_fence, ctx->stream) != cudaSuccess ||
        cudaStreamWaitEvent(ls, ctx->lane_fence, 0) != cudaSuccess)
        return fail(ctx, SPK_ERR_CUDA, "stream ordering: %s", cudaGetErrorString(cudaGetLastError()));
    if (cudaMemcpyAsync(ctx->lane_in[l], host_stream, in_bytes, cudaMemcpyHostToDevice, ls) != cudaSuccess)
        return fail(ctx, SPK_ERR_CUDA, "H2D copy: %s", cudaGetErrorString(cudaGetLastError()));
    cudaStream_t own = ctx->stream;  // the scan launches on the lane
    ctx->stream = ls;
    rc = run_scan(ctx, ctx->lane_in[l], H, W, T, threshold, ctx->lane_out[l], nullptr, nullptr, nullptr, nullptr,
                  nullptr, nullptr, 0, false);
    ctx->stream = own;
    if (rc) return rc;
    if (cudaMemcpyAsync(host_frames, ctx->lane_out[l], out_bytes, cudaMemcpyDeviceToHost, ls) != cudaSuccess)
        return fail(ctx, SPK_ERR_CUDA, "D2H copy: %s", cudaGetErrorString(cudaGetLastError()));
    ctx->next_lane = l ^ 1;
    return SPK_OK;
}

}  // extern "C"

// ============================================================ no-allocation variant ====
// spk_reconstruct_host_noalloc: the stream and frames are staged in this file-scope
// device array instead of context buffers.  In host code `g_noalloc_scratch` is only a
// host-side stand-in for the symbol; the device address is looked up once per device
// with cudaGetSymbolAddress and passed to the kernel.
namespace {

constexpr size_t NOALLOC_BYTES = SPK_NOALLOC_SCRATCH_BYTES;
constexpr size_t NOALLOC_STATUS_BYTES = 256;  // status word, padded to keep 256-byte alignment
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_ptr[NOALLOC_MAX_DEVICES];  // device address per device, once looked up

size_t round256(size_t n) { return (n + 255) / 256 * 256; }

}  // namespace

extern "C" int spk_reconstruct_host_noalloc(const spk_config *cfg, const uint8_t *host_stream, int H, int W,
                                            int T, float threshold, void *host_frames) {
    if (!cfg) return fail(nullptr, SPK_ERR_ARG, "cfg is NULL");
    if (!valid_method(cfg)) return fail(nullptr, SPK_ERR_ARG, "method must be 1..5 (TFP: tfp_window 1..64; NORDER: stability_order 3..5)");
    if (const char *why = bad_output_cfg(cfg)) return fail(nullptr, SPK_ERR_ARG, "%s", why);
    if (cfg->device < 0 || cfg->device >= NOALLOC_MAX_DEVICES) return fail(nullptr, SPK_ERR_ARG, "bad device ordinal");
    if (!host_stream || !host_frames) return fail(nullptr, SPK_ERR_ARG, "host_stream or host_frames is NULL");
    if (H <= 0 || W <= 0 || T <= 0) return fail(nullptr, SPK_ERR_ARG, "H, W, T must be > 0 (got %d, %d, %d)", H, W, T);
    if (!std::isfinite(threshold) || !(threshold > 0.f))
        return fail(nullptr, SPK_ERR_ARG, "threshold must be finite and > 0");
    if (cfg->out_dtype == SPK_U8 && !u8_threshold_ok(threshold))
        return fail(nullptr, SPK_ERR_ARG, "8-bit frames need an integral threshold in 1 .. 65535");
    const int64_t P = static_cast<int64_t>(H) * W;
    const int64_t T_out = spk_num_frames(T, cfg->frame_stride);
    const size_t esz = out_esz(cfg->out_dtype);
    // the n-order tree also needs its pending-cut rings: 2 x NORDER_CAP0 ints per pixel at first
    const double ring_d = cfg->method == SPK_NORDER ? 2.0 * NORDER_CAP0 * sizeof(int) * static_cast<double>(P) : 0.0;
    const double need_d = static_cast<double>(NOALLOC_STATUS_BYTES) +
                          static_cast<double>(round256(static_cast<size_t>(T) * static_cast<size_t>(pitch_of(H, W)))) +
                          static_cast<double>(round256(static_cast<size_t>(T_out) * static_cast<size_t>(P) * esz)) +
                          ring_d;
    if (need_d > static_cast<double>(NOALLOC_BYTES))
        return fail(nullptr, SPK_ERR_ARG,
                    "stream, frames and rings need %.0f bytes of device scratch; spk_reconstruct_host_noalloc has %zu "
                    "(use spk_reconstruct_host for larger problems)",
                    need_d, NOALLOC_BYTES);
    const size_t in_bytes = static_cast<size_t>(T) * static_cast<size_t>(pitch_of(H, W));
    const size_t out_bytes = static_cast<size_t>(T_out) * static_cast<size_t>(P) * esz;

    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, SPK_ERR_CUDA, "cudaSetDevice(%d) failed", cfg->device);
    }
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[cfg->device]) {  // set-up, once per device, with that device current
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                cudaGetLastError();
                return fail(nullptr, SPK_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            }
            g_noalloc_ptr[cfg->device] = static_cast<unsigned char *>(ptr);
        }
        base = g_noalloc_ptr[cfg->device];
    }
    int *d_status = reinterpret_cast<int *>(base);
    uint8_t *d_in = base + NOALLOC_STATUS_BYTES;
    void *d_out = base + NOALLOC_STATUS_BYTES + round256(in_bytes);

    spk_ctx tmp{};  // host-side view for the shared launch path; owns no device memory
    tmp.cfg = *cfg;
    tmp.tile = TT_DEFAULT;
    tmp.stream = static_cast<cudaStream_t>(cfg->stream);
    tmp.d_status = d_status;
    if (cfg->method == SPK_NORDER) {  // the rest of the array holds the rings (no allocation)
        const size_t used = NOALLOC_STATUS_BYTES + round256(in_bytes) + round256(out_bytes);
        tmp.d_pend = reinterpret_cast<int *>(base + used);
        tmp.pend_bytes = NOALLOC_BYTES - used;
        tmp.pend_fixed = true;
    }
    // A failure after the first enqueue waits for what was enqueued, so that no copy still
    // reads host_stream (or writes the array) once the call has returned.
    auto bail = [&](int code) {
        cudaStreamSynchronize(tmp.stream);
        cudaGetLastError();
        snprintf(g_create_msg, sizeof(g_create_msg), "%.480s", tmp.msg);
        return code;
    };
    // the array keeps the previous call's contents: clear the status word first
    if (cudaMemsetAsync(d_status, 0, sizeof(int), tmp.stream) != cudaSuccess ||
        cudaMemcpyAsync(d_in, host_stream, in_bytes, cudaMemcpyHostToDevice, tmp.stream) != cudaSuccess) {
        fail(&tmp, SPK_ERR_CUDA, "H2D staging: %s", cudaGetErrorString(cudaGetLastError()));
        return bail(SPK_ERR_CUDA);
    }
    int rc = run_scan(&tmp, d_in, H, W, T, threshold, d_out, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0,
                      false);
    if (rc) return bail(rc);
    if (cudaMemcpyAsync(host_frames, d_out, out_bytes, cudaMemcpyDeviceToHost, tmp.stream) != cudaSuccess) {
        fail(&tmp, SPK_ERR_CUDA, "D2H copy: %s", cudaGetErrorString(cudaGetLastError()));
        return bail(SPK_ERR_CUDA);
    }
    cudaError_t e = cudaStreamSynchronize(tmp.stream);
    if (e != cudaSuccess) {
        fail(&tmp, SPK_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
        return bail(SPK_ERR_CUDA);
    }
    int st = 0;
    if (cudaMemcpy(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        fail(&tmp, SPK_ERR_CUDA, "status read failed");
        return bail(SPK_ERR_CUDA);
    }
    if (st & DEV_TIMEOUT) {
        fail(&tmp, SPK_ERR_TIMEOUT, "a bounded device wait gave up");
        return bail(SPK_ERR_TIMEOUT);
    }
    if (st) {
        fail(&tmp, SPK_ERR_INTERNAL, "device consistency check failed (status %d)", st);
        return bail(SPK_ERR_INTERNAL);
    }
    return SPK_OK;
}
