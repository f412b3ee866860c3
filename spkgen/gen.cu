// Seeded synthetic spike-stream generator on the GPU (input recipe only).
//
// The same discrete integrate-and-fire sensor (Eq. 2, Sec. II) and the same scene as
// gen.c, computed one thread per pixel so that many long clips can be made on the device
// (training data of the learned refiner, large benchmark streams).  It reads the texture
// table that the host renders for gen.c and repeats gen.c's fp64 arithmetic operation by
// operation; the file is compiled with -fmad=false so that no multiply-add is contracted,
// which makes every bit of the stream and of the ground truth equal to gen.c's output.
//
// Holds no part of the reconstruction method.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int MAX_EVENTS = 16;

struct Scene {
    const double *tex;
    int L;
    double x0, y0, vx, vy, ilo, ihi, theta, noise_p;
    uint64_t seed;
    int ne;
    double ev[MAX_EVENTS][6];  // (t, y_lo, x_lo, y_hi, x_hi, factor)
};

// SplitMix64 finaliser as a counter-based hash (Steele, Lea, Flood, OOPSLA 2014)
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) {
    const uint64_t h = mix64(mix64(mix64(seed ^ mix64(stream)) ^ a) ^ b);
    return static_cast<double>(h >> 11) * 0x1.0p-53;
}

__device__ __forceinline__ double sample_tex(const double *tex, int L, double u, double v) {
    const double fl = static_cast<double>(L);
    u = fmod(u, fl);
    if (u < 0.0) u += fl;
    v = fmod(v, fl);
    if (v < 0.0) v += fl;
    int iu = static_cast<int>(floor(u)), iv = static_cast<int>(floor(v));
    if (iu >= L) iu = L - 1;
    if (iv >= L) iv = L - 1;
    const double fu = u - static_cast<double>(iu), fv = v - static_cast<double>(iv);
    const int iu1 = (iu + 1 == L) ? 0 : iu + 1;
    const int iv1 = (iv + 1 == L) ? 0 : iv + 1;
    const double t00 = tex[static_cast<int64_t>(iv) * L + iu], t01 = tex[static_cast<int64_t>(iv) * L + iu1];
    const double t10 = tex[static_cast<int64_t>(iv1) * L + iu], t11 = tex[static_cast<int64_t>(iv1) * L + iu1];
    const double top = (1.0 - fu) * t00 + fu * t01;
    const double bot = (1.0 - fu) * t10 + fu * t11;
    return (1.0 - fv) * top + fv * bot;
}

// One thread per pixel, 32 consecutive pixels per warp: the warp's fire bits of a step are
// one ballot, written as one 32-bit word of the frame row.
__global__ void __launch_bounds__(256) simulate_kernel(const __grid_constant__ Scene sc, uint8_t *out,
                                                       int64_t pitch, int H, int W, int T, float *gt,
                                                       int gt_stride) {
    const int64_t P = static_cast<int64_t>(H) * W;
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t pw = p & ~static_cast<int64_t>(31);  // first pixel of the warp
    if (pw >= P) return;                                // whole warp out of range
    const bool valid = p < P;
    const int y = valid ? static_cast<int>(p / W) : 0, x = valid ? static_cast<int>(p % W) : 0;
    double V = sc.theta * uniform(sc.seed, 1, static_cast<uint64_t>(p), 0);
    double gain = 1.0;
    uint32_t *row = reinterpret_cast<uint32_t *>(out + (pw >> 3));
    for (int n = 0; n < T; ++n) {
        for (int e = 0; e < sc.ne; ++e) {
            const double *ev = sc.ev[e];
            if (static_cast<int>(ev[0]) != n) continue;
            if (y >= static_cast<int>(ev[1]) && y < static_cast<int>(ev[3]) && x >= static_cast<int>(ev[2]) &&
                x < static_cast<int>(ev[4]))
                gain *= ev[5];
        }
        const double tc = static_cast<double>(n) + 0.5;
        const double du = sc.x0 + sc.vx * tc, dv = sc.y0 + sc.vy * tc;
        double q = sample_tex(sc.tex, sc.L, static_cast<double>(x) + du, static_cast<double>(y) + dv) * gain;
        if (q < sc.ilo) q = sc.ilo;
        if (q > sc.ihi) q = sc.ihi;
        if (gt && valid && n % gt_stride == 0) gt[static_cast<int64_t>(n / gt_stride) * P + p] = static_cast<float>(q);
        double v = V + q;
        bool fire = v >= sc.theta;
        if (fire) v -= sc.theta;
        V = v;
        if (sc.noise_p > 0.0 && uniform(sc.seed, 2, static_cast<uint64_t>(p), static_cast<uint64_t>(n)) < sc.noise_p)
            fire = true;
        const uint32_t word = __ballot_sync(0xffffffffu, fire && valid);
        if ((threadIdx.x & 31) == 0) row[static_cast<int64_t>(n) * (pitch >> 2)] = word;
    }
}

}  // namespace

extern "C" {

// Writes the stream uint8 [T][pitch] (device, pitch a multiple of 16) of the scene gen.c's
// spkgen_simulate describes, and, if gt is not NULL, the clipped intensity at every
// gt_stride-th step (device fp32 [ceil(T / gt_stride)][H * W]).  tex: device fp64 [L][L]
// rendered by spkgen_render_texture; events: host fp64 [ne][6].  Asynchronous on
// `stream`.  Returns 0, -1 on bad arguments, -2 on a CUDA error.
int spkgen_cuda_simulate(uint8_t *out, int64_t pitch, int H, int W, int T, const double *tex, int L, double x0,
                         double y0, double vx, double vy, int ne, const double *events, double ilo, double ihi,
                         double theta, uint64_t seed, double noise_p, float *gt, int gt_stride, void *stream) {
    const int64_t P = static_cast<int64_t>(H) * W;
    if (!out || !tex || H <= 0 || W <= 0 || T <= 0 || pitch % 16 || pitch * 8 < P || L <= 0 || !(theta > 0.0) ||
        ne < 0 || ne > MAX_EVENTS || (ne && !events) || (gt && gt_stride <= 0) ||
        reinterpret_cast<uintptr_t>(out) % 16)
        return -1;
    Scene sc{};
    sc.tex = tex;
    sc.L = L;
    sc.x0 = x0, sc.y0 = y0, sc.vx = vx, sc.vy = vy, sc.ilo = ilo, sc.ihi = ihi, sc.theta = theta;
    sc.noise_p = noise_p;
    sc.seed = seed;
    sc.ne = ne;
    for (int e = 0; e < ne; ++e)
        for (int k = 0; k < 6; ++k) sc.ev[e][k] = events[6 * e + k];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(out, 0, static_cast<size_t>(pitch) * T, s) != cudaSuccess) return -2;
    const int64_t blocks = (P + 255) / 256;
    simulate_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(sc, out, pitch, H, W, T, gt, gt_stride);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // extern "C"
