// Learned refiner of the plain reconstruction -- kernels and the C ABI (spk.h, spk_refiner_*).
//
// The paper's method is parameter free (Sec. III-B); the refiner is this library's
// extension: a 5-layer 3x3 convolutional network that takes, per pixel and frame, the plain
// FSR/SSR value and the rates theta / x of the last four intervals (spk_features) and
// predicts a correction to the plain value.  Layers (bf16 activations in channel-chunk
// planes [N][H][C/8][W][8], fp32 accumulation on the tensor cores):
//   L0 16 -> 32 (ReLU), L1..L3 32 -> 32 (ReLU), L4 32 -> 16 (linear; channel 0 is used,
//   the other channels only pad K of the L4 gradient GEMM to the tensor-core k16)
//   out = plain + L4(...)[channel 0]
// Training minimises the mean squared error to the ground-truth intensity with Adam.
//
// Every convolution is an implicit GEMM on the 5th-generation tensor cores (tcgen05.mma,
// bf16 in, fp32 accumulate in tensor memory): a 128-pixel output row segment is M, the
// nine taps x input channels are K (conv3x3_kernel).  The weight gradient is a GEMM over
// pixels (K = pixels) with M = (tap, input channel) and N = output channel
// (wgrad_kernel), reduced over blocks in a fixed order.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <new>

#include "../../include/spk.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int NL = 5;                                 // layers
constexpr int CIN[NL] = {16, 32, 32, 32, 32};
constexpr int COUT[NL] = {32, 32, 32, 32, 16};  // L4: channel 0 is the output, 1..15 stay unused
constexpr int MT = 128;                               // pixels per block (one row segment)

// parameter block offsets (fp32 master copy): per layer W[9][COUT][CIN] then b[COUT]
constexpr int64_t layer_w(int l) { return 9LL * COUT[l] * CIN[l]; }
constexpr int64_t layer_off(int l) { return l == 0 ? 0 : layer_off(l - 1) + layer_w(l - 1) + COUT[l - 1]; }
constexpr int64_t NPARAM = layer_off(NL - 1) + layer_w(NL - 1) + COUT[NL - 1];



// Activations with C channels are stored as channel-chunk planes, [N][H][C/8][W][8]: the 8
// channels of a chunk are one 16-byte cell, and one image row of one chunk is W contiguous
// cells.  Element (n, y, x, c):
__host__ __device__ __forceinline__ int64_t act_idx(int n, int y, int x, int c, int H, int W, int C) {
    return ((static_cast<int64_t>(n) * H + y) * (C / 8) + c / 8) * W * 8 + static_cast<int64_t>(x) * 8 + (c & 7);
}



// ------------------------------------------------------------------- convolution ----
// Y[n][y][x][co] = act(sum_{tap, ci} X[n][y+ky-1][x+kx-1][ci] * Wt[tap][co][ci] + b[co])
// MODE 0: bf16 out, ReLU;  MODE 1: bf16 out, no bias, times (mask > 0) (the dgrad of a
// ReLU layer);  MODE 2: fp32 out of channel 0 plus resid (the last layer).
//
// Implicit GEMM on the 5th-generation tensor cores.  An output row segment of 128 pixels
// is one M = 128 tile; N = CO; K = 9 taps x CI, issued as 9 x CI/16 tcgen05.mma (bf16 in,
// fp32 accumulate in tensor memory) by one thread.  Both operands are K-major without
// swizzle: 8-row x 16-byte core matrices.  The input halo row (130 pixels) is stored as
// CI/8 planes of [pixel][8 channels], so the core-matrix row stride is 16 bytes and the
// 8-row group stride (SBO) 128 bytes: the A operand of tap (ky, kx) is the same planes
// seen from a start address kx * 16 bytes further.  Weights are stored per tap as
// [chunk][co][8 channels] (B operand, N = co rows).
//
// Persistent and warp-specialised: a block stages the weights once, then walks tasks of
// ry rows x 128 pixels of one image (a task reloads two halo rows, so tall tasks when there
// are enough of them for every block, 32 rows otherwise).  One thread loads halo rows with TMA (512-byte boxes of
// the channel-chunk planes) into a ring of
// RING row slots; one thread issues the MMAs of output row y as soon as rows y - 1 .. y + 1
// have landed and an accumulator is free, and releases a row slot (tcgen05.commit onto its
// mbarrier) after the last MMA that reads it; four warps read finished accumulators out of
// tensor memory and write the output rows.  Loads, MMAs and the write-out of different rows
// overlap.
constexpr int RY = 32;        // output rows per task, the short form
constexpr int RY_TALL = 125;  // ... and the tall one (two tasks per column of a 250-row image)
constexpr long long MMA_WAIT_CYCLES = 4000000000LL;  // ~2 s: bounded waits

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
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
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *status) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > MMA_WAIT_CYCLES) {
            atomicOr(status, 1);
            return false;
        }
    return true;
}

// shared-memory matrix descriptor: K-major, no swizzle; leading (K) and stride (M/N)
// byte offsets between core matrices
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
           (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);  // descriptor version 1
}
// instruction descriptor of kind::f16: bf16 A and B, fp32 D, both K-major, M x N
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16_tc(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// 32 lanes x 16 columns of fp32 accumulator: thread l of the warp gets lane (base + l)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 32 pixels x 8 channels of one chunk plane of one image row of a [N][H][C/8][W][8] tensor
// seen as (W*8 elements, C/8, H, N): the element coordinate e (a multiple of 8, so 16-byte
// aligned; negative or past the row for the halo: zero fill), chunk c, row y, image n
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, uint64_t *bar, int e, int c, int y,
                                            int n) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(e), "r"(c), "r"(y), "r"(n)
        : "memory");
}

constexpr int RING = 5;  // input-row slots
constexpr int TMA_PX = 32;                  // pixels per main TMA box (256 bf16: the largest box edge)
constexpr int TAIL_PX = 8;                  // pixels of the last box of a plane (pixels 128 .. 135)
constexpr int HALO_PX = 4 * TMA_PX + TAIL_PX;  // pixels loaded per halo row (>= 130), 136 x 16 B = 17 x 128 B
constexpr int NACC = 4;  // accumulators in tensor memory

template <int CI, int CO>
struct ConvSmem {
    static constexpr int CH = CI / 8;                        // 16-byte channel chunks
    static constexpr int PLANE = HALO_PX * 16;               // one chunk plane of a halo row: 160 x 16 B
    static constexpr int SLOT = CH * PLANE;                  // one halo row (all planes)
    static constexpr int WPLANE = CO * 16;                   // one chunk plane of a tap's weights
    static constexpr int W_OFF = RING * SLOT;
    static constexpr int BAR_OFF = W_OFF + 9 * CH * WPLANE;
    // full[RING], empty[RING], acc_full[NACC], acc_empty[NACC], done, then the TMEM address
    static constexpr int TMEM_OFF = BAR_OFF + 8 * (2 * RING + 2 * NACC + 1);
    static constexpr int BYTES = TMEM_OFF + 16 + 128;        // + 128 to align the base
    static constexpr int TCOLS = NACC * CO < 32 ? 32 : NACC * CO;
};

// Roles: warps 0-3 read accumulators out of tensor memory (warp w owns TMEM lanes 32w..)
// and write the output rows; warp 4 (one thread) loads halo rows with TMA into the ring;
// warp 5 (one thread) issues the MMAs, and allocates / frees the tensor memory.
template <int CI, int CO, int MODE>
__global__ void __launch_bounds__(192, 4) conv3x3_kernel(const __grid_constant__ CUtensorMap xmap,
                                                      const __grid_constant__ CUtensorMap xmap_tail,
                                                      const bf16 *__restrict__ Wt, const float *__restrict__ bias,
                                                      void *Y, const bf16 *__restrict__ mask,
                                                      const float *__restrict__ resid, int N, int H, int W,
                                                      int ry, int *status) {
    using L = ConvSmem<CI, CO>;
    constexpr int CH = L::CH;
    constexpr uint32_t IDESC = mma_idesc(MT, CO);
    constexpr uint32_t ROW_TX = CH * HALO_PX * 16;  // bytes of one halo row
    extern __shared__ unsigned char smraw_[];
    unsigned char *smraw = smraw_ + ((128 - (smem_u32(smraw_) & 127)) & 127);
    const uint32_t sbase = smem_u32(smraw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smraw + L::BAR_OFF);
    uint64_t *empty = full + RING;
    uint64_t *accf = empty + RING;
    uint64_t *acce = accf + NACC;
    uint64_t *done = acce + NACC;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smraw + L::TMEM_OFF);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < RING; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < NACC; ++i) {
            mbar_init(&accf[i], 1);
            mbar_init(&acce[i], 4);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(L::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // weights: Wt[tap][co][ci] -> [tap][chunk][co][8]
    for (int c = tid; c < 9 * CO * CH; c += 192) {
        const int tap = c / (CO * CH), rem = c % (CO * CH), co = rem / CH, ch = rem % CH;
        cp_async16(sbase + L::W_OFF + ((tap * CH + ch) * CO + co) * 16,
                   Wt + (static_cast<int64_t>(tap) * CO + co) * CI + ch * 8, true);
    }
    cp_async_commit();
    cp_async_wait0();
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int nxs = (W + MT - 1) / MT, nys = (H + ry - 1) / ry;
    const int64_t ntask = static_cast<int64_t>(N) * nxs * nys;
    auto geometry = [&](int64_t task, int &n, int &x0, int &y0, int &y1) {
        const int xs = static_cast<int>(task % nxs);
        const int ys = static_cast<int>((task / nxs) % nys);
        n = static_cast<int>(task / (static_cast<int64_t>(nxs) * nys));
        x0 = xs * MT;
        y0 = ys * ry;
        y1 = min(H, y0 + ry);
    };

    if (warp == 4) {  // ------------------------------------------------ TMA producer ----
        // lane 0 waits for the slot and arms its barrier; then CH x 5 lanes issue one box each
        constexpr int BOXES = CH * 5;  // four boxes of 32 pixels and one of 8 per chunk plane
        static_assert(BOXES <= 32, "one box per lane");
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&xmap)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&xmap_tail)) : "memory");
        }
        int sl = 0, ph = 0, issued = 0;  // ring slot, its phase, loads issued (the same in every lane)
        bool ok = true;
        for (int64_t task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
            int n, x0, y0, y1;
            geometry(task, n, x0, y0, y1);
            for (int r = y0 - 1; r <= y1; ++r) {
                // the slot's previous row must have been released (from the second pass over the ring on)
                bool go = true;
                if (lane == 0) {
                    if (issued >= RING) go = mbar_wait(&empty[sl], ph ^ 1, status);
                    if (go) mbar_expect_tx(&full[sl], ROW_TX);
                }
                if (!__shfl_sync(0xffffffffu, go, 0)) {
                    ok = false;
                    break;
                }
                if (lane < BOXES) {
                    const int ch = lane / 5, j = lane % 5;
                    tma_load_4d(sbase + sl * L::SLOT + ch * L::PLANE + j * TMA_PX * 16, j < 4 ? &xmap : &xmap_tail,
                                &full[sl], (x0 - 1 + j * TMA_PX) * 8, ch, r, n);
                }
                ++issued;
                if (++sl == RING) sl = 0, ph ^= 1;
            }
        }
        // let every issued copy land before this warp leaves: the last min(issued, RING) loads
        if (lane == 0)
            for (int k = 0; k < RING && k < issued; ++k) {
                if (--sl < 0) sl = RING - 1, ph ^= 1;
                if (!mbar_wait(&full[sl], ph, status)) break;
            }
    } else if (warp == 5) {  // ----------------------------------------- MMA issuer ----
        if (lane == 0) {
            // descriptors are linear in the start address (bits 0-13 hold address / 16), so every
            // operand is a base descriptor plus a compile-time or per-row offset
            const uint64_t a_base = smem_desc(sbase, L::PLANE, 128);
            const uint64_t b_base = smem_desc(sbase + L::W_OFF, L::WPLANE, 128);
            int sl = 0, ph = 0;   // slot and phase of the next load to wait for
            int a = 0, aph = 0;   // accumulator and its phase
            int rows_done = 0;    // MMA rows issued (accumulator uses)
            bool ok = true;
            auto wait_full = [&]() {  // the next load in order
                const bool r = mbar_wait(&full[sl], ph, status);
                if (++sl == RING) sl = 0, ph ^= 1;
                return r;
            };
            int s_first = 0;  // slot of input row y - 1 for the current output row
            for (int64_t task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
                int n, x0, y0, y1;
                geometry(task, n, x0, y0, y1);
                s_first = sl;
                if (!wait_full() || !wait_full()) {  // input rows y0 - 1 and y0
                    ok = false;
                    break;
                }
                for (int y = y0; y < y1; ++y) {
                    if (!wait_full() ||  // input row y + 1
                        (rows_done >= NACC && !mbar_wait(&acce[a], aph ^ 1, status))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + static_cast<uint32_t>(a * CO);
                    uint64_t arow[3];
                    for (int ky = 0, sk = s_first; ky < 3; ++ky, sk = (sk + 1 == RING ? 0 : sk + 1))
                        arow[ky] = a_base + static_cast<uint64_t>((sk * L::SLOT) >> 4);
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
                        for (int s = 0; s < CI / 16; ++s) {
                            const uint64_t ad = arow[tap / 3] + static_cast<uint64_t>(((tap % 3) * 16 + 2 * s * L::PLANE) >> 4);
                            const uint64_t bd = b_base + static_cast<uint64_t>(((tap * CH + 2 * s) * L::WPLANE) >> 4);
                            mma_bf16_tc(d, ad, bd, IDESC, (tap | s) ? 1u : 0u);
                        }
                    }
                    mma_commit(&accf[a]);
                    mma_commit(&empty[s_first]);  // input row y - 1 has no later reader
                    s_first = s_first + 1 == RING ? 0 : s_first + 1;
                    ++rows_done;
                    if (++a == NACC) a = 0, aph ^= 1;
                }
                if (!ok) break;
                // input rows y1 - 1 and y1 are released after the task's last MMAs
                mma_commit(&empty[s_first]);
                mma_commit(&empty[s_first + 1 == RING ? 0 : s_first + 1]);
            }
            mma_commit(done);  // every MMA of this block has completed once this arrives
            mbar_wait(done, 0, status);
        }
    } else {  // ------------------------------------------------------- epilogue warps ----
        constexpr int CPP = CO / 8;  // output chunks (planes)
        float bv[MODE == 0 ? CO : 1];  // the bias stays in registers (Y may alias it as far as the compiler knows)
        if constexpr (MODE == 0) {
#pragma unroll
            for (int c = 0; c < CO; ++c) bv[c] = bias[c];
        } else if constexpr (MODE == 2) {
            bv[0] = bias[0];
        }
        int a = 0, aph = 0;  // accumulator and its phase
        bool ok = true;
        for (int64_t task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
            int n, x0, y0, y1;
            geometry(task, n, x0, y0, y1);
            for (int y = y0; y < y1; ++y, a = (a + 1 == NACC ? 0 : a + 1), aph ^= (a == 0)) {
                const int x = x0 + warp * 32 + lane;
                // chunk q of pixel x of this row: cell (row * CPP + q) * W + x; loads that do not
                // depend on the MMAs go out before the wait
                const int64_t row = static_cast<int64_t>(n) * H + y;
                uint4 mk[MODE == 1 ? CPP : 1];
                float rs = 0.f;
                if (x < W) {
                    if constexpr (MODE == 1) {
#pragma unroll
                        for (int q = 0; q < CPP; ++q)
                            mk[q] = reinterpret_cast<const uint4 *>(mask)[(row * CPP + q) * W + x];
                    } else if constexpr (MODE == 2) {
                        rs = resid[row * W + x];
                    }
                }
                if (!__all_sync(0xffffffffu, mbar_wait(&accf[a], aph, status))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t ta = tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(a * CO);
                float v[CO];
#pragma unroll
                for (int c = 0; c < CO; c += 16) tmem_ld16(ta + c, v + c);
                tmem_wait_ld();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[a]);  // the accumulator may be overwritten
                if (x >= W) continue;
                if constexpr (MODE == 2) {
                    static_cast<float *>(Y)[row * W + x] = v[0] + bv[0] + rs;
                } else {
#pragma unroll
                    for (int q = 0; q < CPP; ++q) {  // lanes write consecutive 16-byte cells of a plane
                        float w8[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) w8[e] = v[q * 8 + e];
                        if constexpr (MODE == 0) {
#pragma unroll
                            for (int e = 0; e < 8; ++e) w8[e] = fmaxf(w8[e] + bv[q * 8 + e], 0.f);
                        } else {
                            const __nv_bfloat162 *m2 = reinterpret_cast<const __nv_bfloat162 *>(&mk[q]);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                if (!(__bfloat162float(m2[e].x) > 0.f)) w8[2 * e] = 0.f;
                                if (!(__bfloat162float(m2[e].y) > 0.f)) w8[2 * e + 1] = 0.f;
                            }
                        }
                        uint4 ov;
                        __nv_bfloat162 *o2 = reinterpret_cast<__nv_bfloat162 *>(&ov);
#pragma unroll
                        for (int e = 0; e < 4; ++e) o2[e] = __floats2bfloat162_rn(w8[2 * e], w8[2 * e + 1]);
                        reinterpret_cast<uint4 *>(Y)[(row * CPP + q) * W + x] = ov;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::TCOLS) : "memory");
    }
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

// halo-row loads of a [N][H][C/8][W][8] bf16 tensor viewed as (W*8, C/8, H, N): boxes of
// 256 elements (32 pixels) of one chunk plane, so every TMA request moves 512 contiguous bytes
bool make_xmap(CUtensorMap *map, const bf16 *X, int C, int N, int H, int W, int box_px) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[4] = {static_cast<cuuint64_t>(W) * 8, static_cast<cuuint64_t>(C / 8), static_cast<cuuint64_t>(H),
                          static_cast<cuuint64_t>(N)};
    cuuint64_t strides[3] = {static_cast<cuuint64_t>(W) * 16, static_cast<cuuint64_t>(W) * C * 2,
                             static_cast<cuuint64_t>(H) * W * C * 2};
    cuuint32_t box[4] = {static_cast<cuuint32_t>(box_px) * 8, 1, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(X), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int CI, int CO, int MODE>
bool conv(cudaStream_t s, int *status, int N, int H, int W, const bf16 *X, const bf16 *Wt, const float *bias,
          void *Y, const bf16 *mask, const float *resid) {
    constexpr int bytes = ConvSmem<CI, CO>::BYTES;
    static int blocks_per_sm = 0, sms = 0;  // attributes and occupancy: once
    if (!blocks_per_sm) {
        cudaFuncSetAttribute(conv3x3_kernel<CI, CO, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        int dev = 0, smem_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, conv3x3_kernel<CI, CO, MODE>);
        // resident blocks: shared memory (1 KB reserved per block), registers (allocated per
        // warp in units of 256), and the 512 tensor-memory columns, TCOLS per block
        const int by_smem = smem_sm / (bytes + 1024);
        const int regs_warp = ((std::max(fa.numRegs, 1) * 32 + 255) / 256) * 256;
        const int by_regs = 65536 / (regs_warp * 6);
        blocks_per_sm = std::max(1, std::min({by_smem, by_regs, 512 / ConvSmem<CI, CO>::TCOLS}));
    }
    CUtensorMap map, map_tail;
    if (!make_xmap(&map, X, CI, N, H, W, TMA_PX) || !make_xmap(&map_tail, X, CI, N, H, W, TAIL_PX)) return false;
    // tall tasks (fewer halo reloads) when every resident block gets about four of them
    const int64_t slots = static_cast<int64_t>(blocks_per_sm) * sms;
    const int nx = (W + MT - 1) / MT;
    const int ry = static_cast<int64_t>(N) * nx * ((H + RY_TALL - 1) / RY_TALL) >= 4 * slots ? RY_TALL : RY;
    const int64_t ntask = static_cast<int64_t>(N) * nx * ((H + ry - 1) / ry);
    const int64_t grid = std::min<int64_t>(ntask, slots);
    conv3x3_kernel<CI, CO, MODE><<<static_cast<unsigned>(grid), 192, bytes, s>>>(map, map_tail, Wt, bias, Y, mask,
                                                                                  resid, N, H, W, ry, status);
    return true;
}

// ------------------------------------------------------------------ weight gradient ----
// dW[tap][co][ci] = sum_p X[p + off(tap)][ci] * dZ[p][co],  dB[co] = sum_p dZ[p][co], with
// off(ky, kx) = (ky - 1, kx - 1) and p over every pixel of every image (K = pixels).
//
// On the tensor cores as D[(tap, ci)][co] = sum_k A[(tap, ci)][k] * B[co][k]: a block walks
// row segments of 128 pixels (one K tile each) and stages, per tap, the 128 input pixels that
// tap multiplies as CI/8 planes of [pixel][8 channels] -- the activation layout itself, so A
// is MN-major (8 channels contiguous in a 16-byte row, 8 pixels = 8 rows = one 128-byte core
// matrix), and the 9 taps' planes follow each other at one stride, so that M = 128 rows of
// (tap, ci) are one descriptor.  dZ is staged the same way as B (N = CO, MN-major).  Per
// 16-pixel K step one thread issues NT tcgen05.mma of M = 128 (taps 0-3, 4-7 and 5-8 for
// CI = 32, whose last tile contributes only tap 8; taps 0-7 and 1-8 for CI = 16), each
// accumulating into its own fp32 region of tensor memory for the whole block.  Stages are
// double-buffered: the next tile's cp.async loads are in flight while the tensor cores and
// the bias sums (all threads, pixel groups added in a fixed order) work on this one.  Each
// block writes its partial sums; wgrad_reduce_kernel adds the blocks' partials in block
// order, so the gradient is the same bit for bit on every run.
template <int CI, int CO>
struct WgSmem {
    static constexpr int CH = CI / 8, CHO = CO / 8;
    static constexpr int PLANE = MT * 16;                 // 128 pixels x 16 bytes
    static constexpr int A_BYTES = 9 * CH * PLANE;        // the taps' input planes
    static constexpr int B_BYTES = CHO * PLANE;           // dZ planes
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int RED_OFF = 2 * STAGE;             // bias partial sums, WG_THREADS floats
    static constexpr int BAR_OFF = RED_OFF + 256 * 4;     // mma_done[2], done
    static constexpr int TMEM_OFF = BAR_OFF + 8 * 3;
    static constexpr int BYTES = TMEM_OFF + 16 + 128;     // + 128 to align the base
    static constexpr int NT = CI == 32 ? 3 : 2;           // M = 128 tiles over (tap, ci)
    static constexpr int TPT = 128 / CI;                  // taps per tile
    static constexpr int COLS = NT * CO;
    static constexpr int TCOLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : 256;
    __host__ __device__ static constexpr int tap0(int a) { return a == 0 ? 0 : a == NT - 1 ? 9 - TPT : TPT * a; }
};
constexpr int WG_THREADS = 256;
constexpr int WG_MMA_TID = 128;   // warp 4, lane 0: issues the MMAs

// instruction descriptor of kind::f16 with both operands MN-major (transpose bits 15, 16)
__host__ __device__ constexpr uint32_t mma_idesc_mn(int M, int N) { return mma_idesc(M, N) | (1u << 15) | (1u << 16); }

template <int CI, int CO>
__global__ void __launch_bounds__(WG_THREADS, 1)
    wgrad_kernel(const bf16 *__restrict__ X, const bf16 *__restrict__ dZ, float *partial, int N, int H, int W,
                 int *status) {
    using L = WgSmem<CI, CO>;
    constexpr int CH = L::CH, CHO = L::CHO, NT = L::NT;
    constexpr uint32_t IDESC = mma_idesc_mn(128, CO);
    constexpr int NW = 9 * CO * CI;  // weights per block partial, then CO biases
    extern __shared__ unsigned char smraw_[];
    unsigned char *smraw = smraw_ + ((128 - (smem_u32(smraw_) & 127)) & 127);
    const uint32_t sbase = smem_u32(smraw);
    uint64_t *mma_done = reinterpret_cast<uint64_t *>(smraw + L::BAR_OFF);
    uint64_t *done = mma_done + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smraw + L::TMEM_OFF);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        mbar_init(&mma_done[0], 1);
        mbar_init(&mma_done[1], 1);
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(L::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int nxs = (W + MT - 1) / MT;
    const int64_t ntile = static_cast<int64_t>(N) * H * nxs;
    float bsum = 0.f;  // thread co < CO: its bias gradient over this block's pixels, in tile order
    float *red = reinterpret_cast<float *>(smraw + L::RED_OFF);  // [WG_THREADS / CO][CO] partial sums
    constexpr int PARTS = WG_THREADS / CO, PPX = MT / PARTS;     // pixel groups of the bias sum
    // cp.async of one tile into stage st: the 9 taps' input planes, then the dZ planes
    auto stage_tile = [&](int64_t tile, int st) {
        const int xs = static_cast<int>(tile % nxs), y = static_cast<int>((tile / nxs) % H);
        const int n = static_cast<int>(tile / (static_cast<int64_t>(nxs) * H));
        const int x0 = xs * MT;
        const uint32_t sa = sbase + st * L::STAGE, sb = sa + L::A_BYTES;
        for (int c = tid; c < 9 * CH * MT; c += WG_THREADS) {  // plane (tap, chunk), pixel j
            const int j = c % MT, rest = c / MT, ch = rest % CH, tap = rest / CH;
            const int yy = y + tap / 3 - 1, xx = x0 + tap % 3 - 1 + j;
            const bool v = yy >= 0 && yy < H && xx >= 0 && xx < W;
            cp_async16(sa + (tap * CH + ch) * L::PLANE + j * 16, v ? X + act_idx(n, yy, xx, ch * 8, H, W, CI) : X, v);
        }
        for (int c = tid; c < CHO * MT; c += WG_THREADS) {
            const int j = c % MT, ch = c / MT, xx = x0 + j;
            const bool v = xx < W;
            cp_async16(sb + ch * L::PLANE + j * 16, v ? dZ + act_idx(n, y, xx, ch * 8, H, W, CO) : dZ, v);
        }
    };
    bool ok = true;
    int it = 0;
    if (static_cast<int64_t>(blockIdx.x) < ntile) stage_tile(blockIdx.x, 0);
    cp_async_commit();
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x, ++it) {
        const int st = it & 1;
        const int64_t next = tile + gridDim.x;
        // the next tile goes to the other stage once the tile before this one has left the
        // tensor cores; its loads then overlap this tile's MMAs and bias sums
        if (next < ntile && it >= 1 && !mbar_wait(&mma_done[st ^ 1], ((it - 1) >> 1) & 1, status)) ok = false;
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        if (next < ntile) stage_tile(next, st ^ 1);
        cp_async_commit();
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // this tile's group has landed
        fence_proxy_async_smem();  // the staged planes become visible to the tensor cores
        __syncthreads();
        const uint32_t sa = sbase + st * L::STAGE, sb = sa + L::A_BYTES;
        if (tid == WG_MMA_TID) {
            tc_fence_after();
#pragma unroll
            for (int a = 0; a < NT; ++a) {
#pragma unroll
                for (int s = 0; s < MT / 16; ++s) {
                    // K step s: pixels 16 s .. 16 s + 15 = two 128-byte core matrices further
                    const uint64_t ad = smem_desc(sa + L::tap0(a) * CH * L::PLANE + s * 256, 128, L::PLANE);
                    const uint64_t bd = smem_desc(sb + s * 256, 128, L::PLANE);
                    mma_bf16_tc(tmem + static_cast<uint32_t>(a * CO), ad, bd, IDESC, (it > 0 || s > 0) ? 1u : 0u);
                }
            }
            mma_commit(&mma_done[st]);
        }
        {  // bias gradient: thread (part, co) sums pixels part*PPX .., then co adds the parts in order
            const int co = tid % CO, part = tid / CO;
            const bf16 *zp = reinterpret_cast<const bf16 *>(smraw + st * L::STAGE + L::A_BYTES) +
                             (co / 8) * (L::PLANE / 2) + (co & 7) + part * PPX * 8;
            float ps = 0.f;
#pragma unroll
            for (int j = 0; j < PPX; ++j) ps += __bfloat162float(zp[j * 8]);
            red[part * CO + co] = ps;
        }
        __syncthreads();
        if (tid < CO)
            for (int q = 0; q < PARTS; ++q) bsum += red[q * CO + tid];
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // nothing in flight when the block ends
    // every MMA this block issued has completed once `done` arrives
    if (tid == WG_MMA_TID) mma_commit(done);
    const bool fin = mbar_wait(done, 0, status);
    ok = __syncthreads_and(ok && fin);
    tc_fence_after();
    float *pw = partial + static_cast<int64_t>(blockIdx.x) * (NW + CO);
    if (warp < 4) {  // warp w reads tensor-memory lanes 32 w .. 32 w + 31: rows (tap, ci)
        const int m = warp * 32 + lane, tl = m / CI, ci = m % CI;
#pragma unroll
        for (int a = 0; a < NT; ++a) {
            float v[CO];
#pragma unroll
            for (int c = 0; c < CO; c += 16)
                tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(a * CO + c), v + c);
            tmem_wait_ld();
            // the last tile overlaps the one before it: it contributes its last tap only
            if (a == NT - 1 && NT > 1 && tl != L::TPT - 1) continue;
            const int tap = L::tap0(a) + tl;
#pragma unroll
            for (int co = 0; co < CO; ++co)
                pw[(static_cast<int64_t>(tap) * CO + co) * CI + ci] = (ok && it > 0) ? v[co] : 0.f;
        }
    }
    if (tid < CO) pw[NW + tid] = bsum;
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::TCOLS) : "memory");
    }
}

// g[i] = sum over blocks b = 0 .. nb-1, in that order, of partial[b][i]: a fixed order, so
// the weight and bias gradients do not depend on scheduling
__global__ void wgrad_reduce_kernel(const float *__restrict__ partial, int nb, int n, float *g) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nb; ++b) s += partial[static_cast<int64_t>(b) * n + i];
        g[i] = s;
    }
}

// out - gt -> loss sum and dZ of the last layer (bf16, 16 channels, channel 0 only)
__global__ void mse_grad_kernel(const float *out, const float *gt, int64_t n, int W, float scale, bf16 *dz,
                                float *loss) {
    __shared__ float red[8];
    float s = 0.f;
    for (int64_t i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x) {
        const float d = out[i] - gt[i];
        s += d * d;
        uint4 v = make_uint4(0, 0, 0, 0);
        __nv_bfloat162 h = __floats2bfloat162_rn(2.f * d * scale, 0.f);
        v.x = *reinterpret_cast<uint32_t *>(&h);
        const int64_t row = i / W, x = i - row * W;  // dz: [N][H][2][W][8], channel 0 in plane 0
        reinterpret_cast<uint4 *>(dz)[(row * 2) * W + x] = v;
        reinterpret_cast<uint4 *>(dz)[(row * 2 + 1) * W + x] = make_uint4(0, 0, 0, 0);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tsum = 0.f;
        for (int w = 0; w < 8; ++w) tsum += red[w];
        atomicAdd(loss, tsum);
    }
}

// Adam on the fp32 master parameters, then the bf16 forward weights Wt[tap][co][ci] and the
// dgrad weights Wd[8 - tap][ci][co] (the transposed, flipped kernel) of every layer.
struct LayerPtrs {
    int64_t off[NL];
    int ci[NL], co[NL];
    bf16 *wt[NL];
    bf16 *wd[NL];
};

__global__ void adam_kernel(float *w, float *m, float *v, const float *gr, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x) {
        const float gg = gr[i];
        const float mm = b1 * m[i] + (1.f - b1) * gg;
        const float vv = b2 * v[i] + (1.f - b2) * gg * gg;
        m[i] = mm;
        v[i] = vv;
        w[i] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

__global__ void weights_kernel(const float *w, LayerPtrs lp) {
    for (int l = 0; l < NL; ++l) {
        const int ci_n = lp.ci[l], co_n = lp.co[l];
        const int64_t nw = 9LL * ci_n * co_n;
        for (int64_t i = blockIdx.x * 256LL + threadIdx.x; i < nw; i += 256LL * gridDim.x) {
            const int tap = static_cast<int>(i / (co_n * ci_n)), co = static_cast<int>((i / ci_n) % co_n),
                      ci = static_cast<int>(i % ci_n);
            const bf16 v = __float2bfloat16(w[lp.off[l] + i]);
            lp.wt[l][i] = v;
            if (l > 0) lp.wd[l][(static_cast<int64_t>(8 - tap) * ci_n + ci) * co_n + co] = v;
        }
    }
}

}  // namespace

// ============================================================================ host ====
struct spk_refiner {
    int device;
    float *w, *m, *v, *g;      // fp32 parameters, Adam moments, gradient (NPARAM each)
    bf16 *wt[NL], *wd[NL];     // forward and dgrad weights
    float *loss;               // device scalar
    int *status;               // device word: bit 0 set if a kernel gave up a bounded wait
    bf16 *act[NL];             // activations of layers 0..3 (act[4] unused) [N][H][4][W][8]
    bf16 *grad[2];             // two ping-pong gradient buffers, same layout
    float *out;                // training forward output
    float *partial;            // weight-gradient partial sums, one row per block: [sms][9*32*32 + 32]
    int sms;                   // multiprocessors: the weight-gradient grid
    int64_t cap;               // pixels the buffers hold
    int64_t steps;             // Adam steps taken
    char msg[256];
};

namespace {

thread_local char g_ref_msg[256];

int rfail(spk_refiner *r, int code, const char *fmt, ...) {
    char *buf = r ? r->msg : g_ref_msg;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    return code;
}

bool dev_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

LayerPtrs layer_ptrs(spk_refiner *r) {
    LayerPtrs lp;
    for (int l = 0; l < NL; ++l) {
        lp.off[l] = layer_off(l);
        lp.ci[l] = CIN[l];
        lp.co[l] = COUT[l];
        lp.wt[l] = r->wt[l];
        lp.wd[l] = r->wd[l];
    }
    return lp;
}

// activation workspace for `pixels` pixel-frames: four activation buffers when training,
// two for inference; grown on demand, never shrunk
int ensure_buffers(spk_refiner *r, int64_t pixels, bool train) {
    if (pixels <= r->cap && (!train || r->grad[0])) return SPK_OK;
    pixels = pixels > r->cap ? pixels : r->cap;
    for (int l = 0; l < NL; ++l)
        if (r->act[l]) cudaFree(r->act[l]), r->act[l] = nullptr;
    for (int k = 0; k < 2; ++k)
        if (r->grad[k]) cudaFree(r->grad[k]), r->grad[k] = nullptr;
    if (r->out) cudaFree(r->out), r->out = nullptr;
    r->cap = 0;
    bool ok = true;
    for (int l = 0; l < (train ? NL - 1 : 2); ++l) ok &= cudaMalloc(&r->act[l], pixels * 32 * sizeof(bf16)) == cudaSuccess;
    if (train) {
        for (int k = 0; k < 2; ++k) ok &= cudaMalloc(&r->grad[k], pixels * 32 * sizeof(bf16)) == cudaSuccess;
        ok &= cudaMalloc(&r->out, pixels * sizeof(float)) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        return rfail(r, SPK_ERR_OOM, "refiner workspace allocation failed");
    }
    r->cap = pixels;
    return SPK_OK;
}

// weight and bias gradient of one layer into g (its W block, then its biases): one block per
// multiprocessor walks the row segments, then the partial sums are added in block order
template <int CI, int CO>
bool wgrad(spk_refiner *r, cudaStream_t s, const bf16 *X, const bf16 *dZ, int N, int H, int W, float *g) {
    constexpr int bytes = WgSmem<CI, CO>::BYTES;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(wgrad_kernel<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
            cudaSuccess)
            return false;
        attr = true;
    }
    const int64_t ntile = static_cast<int64_t>(N) * H * ((W + MT - 1) / MT);
    const int grid = static_cast<int>(std::min<int64_t>(ntile, r->sms));
    wgrad_kernel<CI, CO><<<grid, WG_THREADS, bytes, s>>>(X, dZ, r->partial, N, H, W, r->status);
    constexpr int n = 9 * CI * CO + CO;
    wgrad_reduce_kernel<<<(n + 255) / 256, 256, 0, s>>>(r->partial, grid, n, g);
    return true;
}

// forward through all layers; for training the activations of L0..L3 stay in r->act[0..3]
// (the backward pass reads them), for inference two of them are used in turn
int forward(spk_refiner *r, cudaStream_t s, const bf16 *x0, const float *plain, int N, int H, int W, float *out,
            bool keep) {
    auto act = [&](int l) { return r->act[keep ? l : (l & 1)]; };
    bool ok = conv<16, 32, 0>(s, r->status, N, H, W, x0, r->wt[0], r->w + layer_off(0) + layer_w(0), act(0), nullptr,
                              nullptr);
    for (int l = 1; l < NL - 1; ++l)
        ok = ok && conv<32, 32, 0>(s, r->status, N, H, W, act(l - 1), r->wt[l], r->w + layer_off(l) + layer_w(l),
                                   act(l), nullptr, nullptr);
    ok = ok && conv<32, 16, 2>(s, r->status, N, H, W, act(NL - 2), r->wt[NL - 1],
                               r->w + layer_off(NL - 1) + layer_w(NL - 1), out, nullptr, plain);
    if (!ok) return rfail(r, SPK_ERR_CUDA, "refiner forward: cuTensorMapEncodeTiled failed");
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPK_OK : rfail(r, SPK_ERR_CUDA, "refiner forward: %s", cudaGetErrorString(e));
}

uint64_t splitmix(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int64_t spk_refiner_num_params(void) { return NPARAM; }

int spk_refiner_create(int device, uint64_t seed, spk_refiner **out) {
    if (!out) return rfail(nullptr, SPK_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return rfail(nullptr, SPK_ERR_CUDA, "cudaSetDevice(%d) failed", device);
    }
    spk_refiner *r = new (std::nothrow) spk_refiner();
    if (!r) return rfail(nullptr, SPK_ERR_OOM, "host allocation failed");
    r->device = device;
    bool ok = true;
    for (float **p : {&r->w, &r->m, &r->v, &r->g}) ok &= cudaMalloc(p, NPARAM * sizeof(float)) == cudaSuccess;
    ok &= cudaMalloc(&r->loss, sizeof(float)) == cudaSuccess;
    ok &= cudaDeviceGetAttribute(&r->sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && r->sms > 0;
    ok &= ok && cudaMalloc(&r->partial, static_cast<size_t>(r->sms) * (9 * 32 * 32 + 32) * sizeof(float)) == cudaSuccess;
    ok &= cudaMalloc(&r->status, sizeof(int)) == cudaSuccess && cudaMemset(r->status, 0, sizeof(int)) == cudaSuccess;
    for (int l = 0; l < NL; ++l) {
        ok &= cudaMalloc(&r->wt[l], layer_w(l) * sizeof(bf16)) == cudaSuccess;
        ok &= cudaMalloc(&r->wd[l], layer_w(l) * sizeof(bf16)) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        spk_refiner_destroy(r);
        return rfail(nullptr, SPK_ERR_OOM, "refiner allocation failed");
    }
    // He-uniform weights from a counter hash of the seed; zero biases; the last layer is
    // scaled by 0.1 so that the untrained refiner returns about the plain value
    float *h = static_cast<float *>(malloc(NPARAM * sizeof(float)));
    if (!h) {
        spk_refiner_destroy(r);
        return rfail(nullptr, SPK_ERR_OOM, "host allocation failed");
    }
    uint64_t st = seed;
    for (int l = 0; l < NL; ++l) {
        const float bound = sqrtf(6.f / (9.f * CIN[l])) * (l == NL - 1 ? 0.1f : 1.f);
        for (int64_t i = 0; i < layer_w(l); ++i) {
            const double u = static_cast<double>(splitmix(st) >> 11) * 0x1.0p-53;
            h[layer_off(l) + i] = static_cast<float>((2.0 * u - 1.0) * bound);
        }
        for (int c = 0; c < COUT[l]; ++c) h[layer_off(l) + layer_w(l) + c] = 0.f;
    }
    int rc = spk_refiner_set_params(r, h, NPARAM);
    free(h);
    if (rc) {
        spk_refiner_destroy(r);
        return rc;
    }
    *out = r;
    return SPK_OK;
}

int spk_refiner_destroy(spk_refiner *r) {
    if (!r) return SPK_OK;
    cudaSetDevice(r->device);
    cudaDeviceSynchronize();
    for (float *p : {r->w, r->m, r->v, r->g, r->loss, r->out, r->partial})
        if (p) cudaFree(p);
    if (r->status) cudaFree(r->status);
    for (int l = 0; l < NL; ++l) {
        if (r->wt[l]) cudaFree(r->wt[l]);
        if (r->wd[l]) cudaFree(r->wd[l]);
        if (r->act[l]) cudaFree(r->act[l]);
    }
    for (int k = 0; k < 2; ++k)
        if (r->grad[k]) cudaFree(r->grad[k]);
    delete r;
    return SPK_OK;
}

const char *spk_refiner_last_error(const spk_refiner *r) { return r ? r->msg : g_ref_msg; }

int spk_refiner_synchronize(spk_refiner *r, void *stream) {
    if (!r) return SPK_ERR_ARG;
    cudaSetDevice(r->device);
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return rfail(r, SPK_ERR_CUDA, "refiner: %s", cudaGetErrorString(cudaGetLastError()));
    int st = 0;
    if (cudaMemcpy(&st, r->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return rfail(r, SPK_ERR_CUDA, "refiner status read failed");
    if (st) {
        cudaMemset(r->status, 0, sizeof(int));
        return rfail(r, SPK_ERR_TIMEOUT, "a refiner kernel gave up a bounded wait on the tensor cores");
    }
    return SPK_OK;
}

int spk_refiner_set_params(spk_refiner *r, const float *host, int64_t n) {
    if (!r || !host || n != NPARAM) return rfail(r, SPK_ERR_ARG, "need %lld parameters", (long long)NPARAM);
    cudaSetDevice(r->device);
    if (cudaMemcpy(r->w, host, NPARAM * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(r->m, 0, NPARAM * sizeof(float)) != cudaSuccess ||
        cudaMemset(r->v, 0, NPARAM * sizeof(float)) != cudaSuccess)
        return rfail(r, SPK_ERR_CUDA, "parameter upload failed");
    r->steps = 0;
    weights_kernel<<<64, 256>>>(r->w, layer_ptrs(r));
    if (cudaDeviceSynchronize() != cudaSuccess) return rfail(r, SPK_ERR_CUDA, "weight conversion failed");
    return SPK_OK;
}

int spk_refiner_get_params(spk_refiner *r, float *host, int64_t n, int which) {
    if (!r || !host || n != NPARAM || which < 0 || which > 1) return rfail(r, SPK_ERR_ARG, "bad arguments");
    cudaSetDevice(r->device);
    if (cudaMemcpy(host, which ? r->g : r->w, NPARAM * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return rfail(r, SPK_ERR_CUDA, "parameter download failed");
    return SPK_OK;
}

int spk_refiner_forward(spk_refiner *r, void *stream, const void *x0, const float *plain, int N, int H, int W,
                        float *out) {
    if (!r) return SPK_ERR_ARG;
    r->msg[0] = 0;
    if (!x0 || !plain || !out || N <= 0 || H <= 0 || W <= 0) return rfail(r, SPK_ERR_ARG, "bad arguments");
    if (reinterpret_cast<uintptr_t>(x0) % 16 || !dev_ptr(x0) || !dev_ptr(plain) || !dev_ptr(out))
        return rfail(r, SPK_ERR_ARG, "x0, plain, out must be device memory (x0 16-byte aligned)");
    if (N > 65535 || H > 65535) return rfail(r, SPK_ERR_ARG, "N and H must be < 65536");
    cudaSetDevice(r->device);
    int rc = ensure_buffers(r, static_cast<int64_t>(N) * H * W, false);
    if (rc) return rc;
    return forward(r, static_cast<cudaStream_t>(stream), static_cast<const bf16 *>(x0), plain, N, H, W, out, false);
}

int spk_refiner_train_step(spk_refiner *r, void *stream, const void *x0, const float *plain, const float *gt, int N,
                           int H, int W, float lr, float *loss_host) {
    if (!r) return SPK_ERR_ARG;
    r->msg[0] = 0;
    if (!x0 || !plain || !gt || N <= 0 || H <= 0 || W <= 0 || !(lr >= 0.f))
        return rfail(r, SPK_ERR_ARG, "bad arguments");
    if (reinterpret_cast<uintptr_t>(x0) % 16 || !dev_ptr(x0) || !dev_ptr(plain) || !dev_ptr(gt))
        return rfail(r, SPK_ERR_ARG, "x0, plain, gt must be device memory (x0 16-byte aligned)");
    if (N > 65535 || H > 65535) return rfail(r, SPK_ERR_ARG, "N and H must be < 65536");
    cudaSetDevice(r->device);
    const int64_t P = static_cast<int64_t>(N) * H * W;
    int rc = ensure_buffers(r, P, true);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bf16 *x = static_cast<const bf16 *>(x0);
    rc = forward(r, s, x, plain, N, H, W, r->out, true);
    if (rc) return rc;
    cudaMemsetAsync(r->loss, 0, sizeof(float), s);
    bf16 *dz = r->grad[0], *dz2 = r->grad[1];
    mse_grad_kernel<<<512, 256, 0, s>>>(r->out, gt, P, W, 1.f / static_cast<float>(P), dz, r->loss);
    // layer 4 (linear): weight gradient, then the gradient of act[3] through ReLU
    bool ok = wgrad<32, 16>(r, s, r->act[3], dz, N, H, W, r->g + layer_off(4));
    ok = ok && conv<16, 32, 1>(s, r->status, N, H, W, dz, r->wd[4], nullptr, dz2, r->act[3], nullptr);
    for (int l = 3; l >= 1; --l) {
        bf16 *tmp = dz;
        dz = dz2;
        dz2 = tmp;
        ok = ok && wgrad<32, 32>(r, s, r->act[l - 1], dz, N, H, W, r->g + layer_off(l));
        ok = ok && conv<32, 32, 1>(s, r->status, N, H, W, dz, r->wd[l], nullptr, dz2, r->act[l - 1], nullptr);
    }
    ok = ok && wgrad<16, 32>(r, s, x, dz2, N, H, W, r->g + layer_off(0));
    if (!ok) return rfail(r, SPK_ERR_CUDA, "refiner backward: kernel set-up failed");
    r->steps += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, static_cast<float>(r->steps)), c2 = 1.f - powf(b2, static_cast<float>(r->steps));
    adam_kernel<<<64, 256, 0, s>>>(r->w, r->m, r->v, r->g, NPARAM, lr, b1, b2, 1e-8f, c1, c2);
    weights_kernel<<<64, 256, 0, s>>>(r->w, layer_ptrs(r));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rfail(r, SPK_ERR_CUDA, "refiner train step: %s", cudaGetErrorString(e));
    if (loss_host) {
        if (cudaMemcpyAsync(loss_host, r->loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return rfail(r, SPK_ERR_CUDA, "loss read failed");
        *loss_host /= static_cast<float>(P);
        return spk_refiner_synchronize(r, stream);
    }
    return SPK_OK;
}

}  // extern "C"
