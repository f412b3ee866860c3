// Learned refiner of the plain reconstruction -- kernels and the C ABI (spk.h, spk_refiner_*).
//
// The paper's method is parameter free (Sec. III-B); the refiner is this library's
// extension: a 5-layer 3x3 convolutional network that takes, per pixel and frame, the plain
// FSR/SSR value and the rates theta / x of the last four intervals (spk_features) and
// predicts a correction to the plain value.  Layers (NHWC, bf16 activations, fp32
// accumulation on the tensor cores):
//   L0 16 -> 32 (ReLU), L1..L3 32 -> 32 (ReLU), L4 32 -> 16 (linear; channel 0 is used,
//   the other channels only pad K of the L4 gradient GEMM to the tensor-core k16)
//   out = plain + L4(...)[channel 0]
// Training minimises the mean squared error to the ground-truth intensity with Adam.
//
// Every convolution is an implicit GEMM: a block takes 128 pixels of one image row, stages
// the 3 x 130 pixel halo and the weights in shared memory, and each warp multiplies 32
// pixels by all output channels with mma.m16n8k16 (bf16 in, fp32 accumulate), the nine
// taps x input channels forming K.  The weight gradient is a GEMM over pixels (K = pixels),
// one warp per tap.
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

__device__ __forceinline__ void mma_bf16(float *d, const uint32_t *a, const uint32_t *b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// four 8x8 bf16 matrices from shared memory; lane l gives the address of row l % 8 of
// matrix l / 8 and receives, of each matrix, row l / 4, elements 2 (l % 4) and 2 (l % 4) + 1
__device__ __forceinline__ void ldsm_x4(uint32_t *r, const bf16 *p) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// ------------------------------------------------------------------- convolution ----
// Y[n][y][x][co] = act(sum_{tap, ci} X[n][y+ky-1][x+kx-1][ci] * Wt[tap][co][ci] + b[co])
// MODE 0: bf16 out, ReLU;  MODE 1: bf16 out, no bias, times (mask > 0) (the dgrad of a
// ReLU layer);  MODE 2: fp32 out of channel 0 plus resid (the last layer).
//
// Persistent: a block stages the weights once, then walks tasks of RY rows x 128 pixels
// of one image.  Within a task the three input rows an output row needs sit in a ring of
// four row buffers; while the 4 warps multiply row y, cp.async fills input row y + 2 (zero
// fill outside the image), so the loads overlap the tensor-core work.
constexpr int RY = 16;  // output rows per task

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int CI, int CO, int MODE>
__global__ void __launch_bounds__(128) conv3x3_kernel(const bf16 *__restrict__ X, const bf16 *__restrict__ Wt,
                                                      const float *__restrict__ bias, void *Y,
                                                      const bf16 *__restrict__ mask, const float *__restrict__ resid,
                                                      int N, int H, int W) {
    constexpr int CP = CI + 8;  // padded channel stride (conflict-free fragment loads)
    constexpr int CH = CI / 8;  // 16-byte chunks per pixel
    extern __shared__ __align__(16) unsigned char smraw[];
    bf16(*ring)[MT + 2][CP] = reinterpret_cast<bf16(*)[MT + 2][CP]>(smraw);  // [4][130][CP]
    bf16(*wsm)[CO][CP] = reinterpret_cast<bf16(*)[CO][CP]>(smraw + sizeof(bf16) * 4 * (MT + 2) * CP);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    for (int c = tid; c < 9 * CO * CH; c += 128) {
        const int tap = c / (CO * CH), rem = c % (CO * CH), co = rem / CH, ch = rem % CH;
        cp_async16(&wsm[tap][co][ch * 8], Wt + (static_cast<int64_t>(tap) * CO + co) * CI + ch * 8, true);
    }
    cp_async_commit();
    const int nxs = (W + MT - 1) / MT, nys = (H + RY - 1) / RY;
    const int64_t ntask = static_cast<int64_t>(N) * nxs * nys;
    constexpr int NT = CO / 8;
    const int m0 = warp * 32;
    for (int64_t task = blockIdx.x; task < ntask; task += gridDim.x) {
        const int xs = static_cast<int>(task % nxs);
        const int ys = static_cast<int>((task / nxs) % nys);
        const int n = static_cast<int>(task / (static_cast<int64_t>(nxs) * nys));
        const int x0 = xs * MT, y0 = ys * RY, y1 = min(H, y0 + RY);
        // input row r of this image into ring slot r & 3 (zeros outside the image)
        auto issue = [&](int r) {
            if (r > y1) return;  // past the last row this task reads
            for (int c = tid; c < (MT + 2) * CH; c += 128) {
                const int xx = c / CH, ch = c % CH, xg = x0 - 1 + xx;
                const bool ok = r >= 0 && r < H && xg >= 0 && xg < W;
                const bf16 *src = ok ? X + ((static_cast<int64_t>(n) * H + r) * W + xg) * CI + ch * 8 : X;
                cp_async16(&ring[r & 3][xx][ch * 8], src, ok);
            }
        };
        __syncthreads();  // the previous task's reads of the ring are done
        issue(y0 - 1);
        issue(y0);
        issue(y0 + 1);
        cp_async_commit();
        for (int y = y0; y < y1; ++y) {
            issue(y + 2);  // the next row's input, into the slot row y - 2 left
            cp_async_commit();
            cp_async_wait1();  // every group but the one just issued
            __syncthreads();   // rows y - 1 .. y + 1 (and the weights) have landed for every thread
            float acc[2][NT][4];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < NT; ++j)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int ky = tap / 3, kx = tap % 3;
                const int slot = (y + ky - 1) & 3;
#pragma unroll
                for (int kc = 0; kc < CI / 16; ++kc) {
                    uint32_t a[2][4], b[NT][2];
                    // A (pixels x channels): matrices (rows 0-7, k 0-7), (rows 8-15, k 0-7),
                    // (rows 0-7, k 8-15), (rows 8-15, k 8-15) = a0..a3 of m16n8k16
                    const int mr = (lane & 7) + ((lane >> 3) & 1) * 8, mk = (lane >> 4) * 8;
#pragma unroll
                    for (int i = 0; i < 2; ++i) ldsm_x4(a[i], &ring[slot][m0 + i * 16 + kx + mr][kc * 16 + mk]);
                    // B (channels x out channels, stored [co][ci]): matrices (co 0-7, k 0-7),
                    // (co 0-7, k 8-15), (co 8-15, k 0-7), (co 8-15, k 8-15) = b0, b1 of two n8 tiles
                    const int nr = (lane & 7) + (lane >> 4) * 8, nk = ((lane >> 3) & 1) * 8;
#pragma unroll
                    for (int j = 0; j < NT; j += 2) {
                        uint32_t q[4];
                        ldsm_x4(q, &wsm[tap][j * 8 + nr][kc * 16 + nk]);
                        b[j][0] = q[0];
                        b[j][1] = q[1];
                        b[j + 1][0] = q[2];
                        b[j + 1][1] = q[3];
                    }
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int j = 0; j < NT; ++j) mma_bf16(acc[i][j], a[i], b[j]);
                }
            }
            // epilogue: rows g and g+8 of each m16 tile, columns 2t and 2t+1 of each n8 tile
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int x = x0 + m0 + i * 16 + g + hh * 8;
                    if (x >= W) continue;
                    const int64_t pix = (static_cast<int64_t>(n) * H + y) * W + x;
                    if constexpr (MODE == 2) {
                        if (t == 0) static_cast<float *>(Y)[pix] = acc[i][0][hh * 2] + bias[0] + resid[pix];
                    } else {
#pragma unroll
                        for (int j = 0; j < NT; ++j) {
                            const int co = j * 8 + 2 * t;
                            float v0 = acc[i][j][hh * 2], v1 = acc[i][j][hh * 2 + 1];
                            if (MODE == 0) {
                                v0 = fmaxf(v0 + bias[co], 0.f);
                                v1 = fmaxf(v1 + bias[co + 1], 0.f);
                            } else {
                                const __nv_bfloat162 mk =
                                    *reinterpret_cast<const __nv_bfloat162 *>(mask + pix * CO + co);
                                if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
                                if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
                            }
                            *reinterpret_cast<__nv_bfloat162 *>(static_cast<bf16 *>(Y) + pix * CO + co) =
                                __floats2bfloat162_rn(v0, v1);
                        }
                    }
                }
            __syncthreads();  // every warp is done with slot (y - 1) & 3 before row y + 3 refills it
        }
    }
    cp_async_wait0();
}

template <int CI, int CO>
constexpr size_t conv_smem() { return sizeof(bf16) * (4 * (MT + 2) + 9 * CO) * (CI + 8); }

template <int CI, int CO, int MODE>
void conv(cudaStream_t s, int N, int H, int W, const bf16 *X, const bf16 *Wt, const float *bias, void *Y,
          const bf16 *mask, const float *resid) {
    static int blocks_per_sm = 0, sms = 0;  // dynamic shared memory above 48 KB: opt in once
    if (!blocks_per_sm) {
        cudaFuncSetAttribute(conv3x3_kernel<CI, CO, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(conv_smem<CI, CO>()));
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, conv3x3_kernel<CI, CO, MODE>, 128,
                                                      conv_smem<CI, CO>());
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    const int64_t ntask = static_cast<int64_t>(N) * ((W + MT - 1) / MT) * ((H + RY - 1) / RY);
    const int64_t grid = std::min<int64_t>(ntask, static_cast<int64_t>(blocks_per_sm) * sms);
    conv3x3_kernel<CI, CO, MODE><<<static_cast<unsigned>(grid), 128, conv_smem<CI, CO>(), s>>>(X, Wt, bias, Y, mask,
                                                                                                resid, N, H, W);
}

// dW[tap][co][ci] += sum_p X[p + tap][ci] * dZ[p][co],  dB[co] += sum_p dZ[p][co].
// One warp per tap (9 warps); a block walks `segs` row segments of 128 pixels.
template <int CI, int CO>
__global__ void __launch_bounds__(288) wgrad_kernel(const bf16 *__restrict__ X, const bf16 *__restrict__ dZ,
                                                    float *dW, float *dB, int N, int H, int W, int segs_per_block) {
    constexpr int PP = MT + 2 + 8;  // padded pixel stride of the transposed halo
    __shared__ __align__(16) bf16 xt[3][CI][PP];       // X transposed: [row][ci][pixel]
    __shared__ __align__(16) bf16 zt[CO][MT + 8];      // dZ transposed: [co][pixel]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const int tap = warp, ky = tap / 3, kx = tap % 3;
    constexpr int MTL = CO / 16;                       // m16 tiles over co
    constexpr int NTL = CI / 8;
    float acc[MTL][NTL][4];
#pragma unroll
    for (int i = 0; i < MTL; ++i)
#pragma unroll
        for (int j = 0; j < NTL; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    float bsum = 0.f;
    const int nseg_w = (W + MT - 1) / MT;
    const int64_t total = static_cast<int64_t>(N) * H * nseg_w;
    for (int s = 0; s < segs_per_block; ++s) {
        const int64_t seg = static_cast<int64_t>(blockIdx.x) * segs_per_block + s;
        if (seg >= total) break;
        const int xs = static_cast<int>(seg % nseg_w), y = static_cast<int>((seg / nseg_w) % H);
        const int n = static_cast<int>(seg / (static_cast<int64_t>(nseg_w) * H));
        const int x0 = xs * MT;
        __syncthreads();
        for (int c = tid; c < 3 * (MT + 2) * CI; c += 288) {
            const int r = c / ((MT + 2) * CI), rem = c % ((MT + 2) * CI), xx = rem / CI, ci = rem % CI;
            const int yy = y + r - 1, xg = x0 - 1 + xx;
            bf16 v = __float2bfloat16(0.f);
            if (yy >= 0 && yy < H && xg >= 0 && xg < W) v = X[((static_cast<int64_t>(n) * H + yy) * W + xg) * CI + ci];
            xt[r][ci][xx] = v;
        }
        for (int c = tid; c < MT * CO; c += 288) {
            const int xx = c / CO, co = c % CO, xg = x0 + xx;
            bf16 v = __float2bfloat16(0.f);
            if (xg < W) v = dZ[((static_cast<int64_t>(n) * H + y) * W + xg) * CO + co];
            zt[co][xx] = v;
        }
        __syncthreads();
        if (warp < 9) {
#pragma unroll 1
            for (int kc = 0; kc < MT / 16; ++kc) {
                uint32_t a[MTL][4], b[NTL][2];
#pragma unroll
                for (int i = 0; i < MTL; ++i) {
                    const int r0 = i * 16 + g, r1 = r0 + 8;
                    const int c0 = kc * 16 + 2 * t;
                    a[i][0] = r0 < CO ? ld32(&zt[r0][c0]) : 0u;
                    a[i][1] = r1 < CO ? ld32(&zt[r1][c0]) : 0u;
                    a[i][2] = r0 < CO ? ld32(&zt[r0][c0 + 8]) : 0u;
                    a[i][3] = r1 < CO ? ld32(&zt[r1][c0 + 8]) : 0u;
                }
#pragma unroll
                for (int j = 0; j < NTL; ++j) {  // B(k = pixel, n = ci): pixel + kx may be odd
                    const bf16 *col = &xt[ky][j * 8 + g][kc * 16 + 2 * t + kx];
                    __nv_bfloat162 p0, p1;
                    p0.x = col[0];
                    p0.y = col[1];
                    p1.x = col[8];
                    p1.y = col[9];
                    b[j][0] = *reinterpret_cast<uint32_t *>(&p0);
                    b[j][1] = *reinterpret_cast<uint32_t *>(&p1);
                }
#pragma unroll
                for (int i = 0; i < MTL; ++i)
#pragma unroll
                    for (int j = 0; j < NTL; ++j) mma_bf16(acc[i][j], a[i], b[j]);
            }
        }
        if (tid < CO)
            for (int xx = 0; xx < MT; ++xx) bsum += __bfloat162float(zt[tid][xx]);
    }
#pragma unroll
    for (int i = 0; i < MTL; ++i)
#pragma unroll
        for (int j = 0; j < NTL; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int co = i * 16 + g + (e >= 2 ? 8 : 0), ci = j * 8 + 2 * t + (e & 1);
                if (co < CO) atomicAdd(&dW[(static_cast<int64_t>(tap) * CO + co) * CI + ci], acc[i][j][e]);
            }
    if (tid < CO) atomicAdd(&dB[tid], bsum);
}

// out - gt -> loss sum and dZ of the last layer (bf16, 16 channels, channel 0 only)
__global__ void mse_grad_kernel(const float *out, const float *gt, int64_t n, float scale, bf16 *dz, float *loss) {
    __shared__ float red[8];
    float s = 0.f;
    for (int64_t i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x) {
        const float d = out[i] - gt[i];
        s += d * d;
        uint4 v = make_uint4(0, 0, 0, 0);
        __nv_bfloat162 h = __floats2bfloat162_rn(2.f * d * scale, 0.f);
        v.x = *reinterpret_cast<uint32_t *>(&h);
        reinterpret_cast<uint4 *>(dz + i * 16)[0] = v;
        reinterpret_cast<uint4 *>(dz + i * 16)[1] = make_uint4(0, 0, 0, 0);
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
    bf16 *act[NL];             // activations of layers 0..3 (act[4] unused) [N][H][W][32]
    bf16 *grad[2];             // two ping-pong gradient buffers [N][H][W][32]
    float *out;                // training forward output
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

// forward through all layers; for training the activations of L0..L3 stay in r->act[0..3]
// (the backward pass reads them), for inference two of them are used in turn
int forward(spk_refiner *r, cudaStream_t s, const bf16 *x0, const float *plain, int N, int H, int W, float *out,
            bool keep) {
    auto act = [&](int l) { return r->act[keep ? l : (l & 1)]; };
    conv<16, 32, 0>(s, N, H, W, x0, r->wt[0], r->w + layer_off(0) + layer_w(0), act(0), nullptr, nullptr);
    for (int l = 1; l < NL - 1; ++l)
        conv<32, 32, 0>(s, N, H, W, act(l - 1), r->wt[l], r->w + layer_off(l) + layer_w(l), act(l), nullptr, nullptr);
    conv<32, 16, 2>(s, N, H, W, act(NL - 2), r->wt[NL - 1], r->w + layer_off(NL - 1) + layer_w(NL - 1), out, nullptr,
                    plain);
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
    for (float *p : {r->w, r->m, r->v, r->g, r->loss, r->out})
        if (p) cudaFree(p);
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
    cudaMemsetAsync(r->g, 0, NPARAM * sizeof(float), s);
    cudaMemsetAsync(r->loss, 0, sizeof(float), s);
    bf16 *dz = r->grad[0], *dz2 = r->grad[1];
    mse_grad_kernel<<<512, 256, 0, s>>>(r->out, gt, P, 1.f / static_cast<float>(P), dz, r->loss);
    const int segs = 8;
    const int64_t nseg = static_cast<int64_t>(N) * H * ((W + MT - 1) / MT);
    const int wblocks = static_cast<int>((nseg + segs - 1) / segs);
    // layer 4 (linear): weight gradient, then the gradient of act[3] through ReLU
    wgrad_kernel<32, 16><<<wblocks, 288, 0, s>>>(r->act[3], dz, r->g + layer_off(4),
                                                 r->g + layer_off(4) + layer_w(4), N, H, W, segs);
    conv<16, 32, 1>(s, N, H, W, dz, r->wd[4], nullptr, dz2, r->act[3], nullptr);
    for (int l = 3; l >= 1; --l) {
        bf16 *tmp = dz;
        dz = dz2;
        dz2 = tmp;
        wgrad_kernel<32, 32><<<wblocks, 288, 0, s>>>(r->act[l - 1], dz, r->g + layer_off(l),
                                                     r->g + layer_off(l) + layer_w(l), N, H, W, segs);
        conv<32, 32, 1>(s, N, H, W, dz, r->wd[l], nullptr, dz2, r->act[l - 1], nullptr);
    }
    wgrad_kernel<16, 32><<<wblocks, 288, 0, s>>>(x, dz2, r->g + layer_off(0), r->g + layer_off(0) + layer_w(0), N, H,
                                                 W, segs);
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
    }
    return SPK_OK;
}

}  // extern "C"
