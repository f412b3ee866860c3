/*
 * Seeded synthetic spike-stream generator (input recipe only).
 *
 * Simulates the discrete integrate-and-fire sensor of Eq. 2 (Sec. II): every pixel
 * accumulates V(n) = V_-(n-1) + Q(n); it fires P(n) = 1 when V(n) >= theta and then
 * subtracts theta (V_-(n) = V(n) - P(n) * theta).  Q(n) is the light intensity of the
 * pixel during step n, taken from a periodic texture table that may translate and that
 * may be multiplied by step events.  Dark-noise spikes are OR-ed into the output bit
 * without touching the accumulator.
 *
 * This file holds no part of the reconstruction method; both the CPU oracle and the
 * CUDA path consume the streams it writes.  All arithmetic is plain IEEE fp64, built
 * with -ffp-contract=off so that the same inputs give the same bits on every host.
 *
 * Output layout: uint8 [T][pitch]; pixel p = y * W + x is bit (p % 8), LSB first, of
 * byte p / 8 of its frame.  Padding bytes and bits are written as zero.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- RNG ---- */
/* SplitMix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), used as a counter-based hash of (seed, stream, a, b). */
static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t spkgen_hash(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) {
    return mix64(mix64(mix64(seed ^ mix64(stream)) ^ a) ^ b);
}

/* uniform double in [0, 1) with 53 random bits */
double spkgen_uniform(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) {
    return (double)(spkgen_hash(seed, stream, a, b) >> 11) * 0x1.0p-53;
}

enum { STREAM_R0 = 1, STREAM_NOISE = 2 };

/* ------------------------------------------------------------- texture ---- */
/*
 * Renders an L x L periodic intensity table (torus):
 *   tex(u, v) = base + sum_b amp_b * exp(-dist_torus^2 / (2 sigma_b^2))
 *                    + sum_g amp_g * sin(2 pi (u cos th_g + v sin th_g) / period_g + phase_g)
 * blobs: nb rows of (cu, cv, sigma, amp); gratings: ng rows of (amp, period, th, phase).
 * Gratings are not periodic on the torus in general; the seam is part of the texture.
 */
void spkgen_render_texture(double *tex, int L, double base,
                           int nb, const double *blobs, int ng, const double *grats) {
    const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
    for (int v = 0; v < L; ++v) {
        for (int u = 0; u < L; ++u) {
            double val = base;
            for (int b = 0; b < nb; ++b) {
                double du = fabs((double)u - blobs[4 * b + 0]);
                double dv = fabs((double)v - blobs[4 * b + 1]);
                if (du > 0.5 * L) du = L - du;
                if (dv > 0.5 * L) dv = L - dv;
                double s = blobs[4 * b + 2];
                val += blobs[4 * b + 3] * exp(-(du * du + dv * dv) / (2.0 * s * s));
            }
            for (int g = 0; g < ng; ++g) {
                double a = grats[4 * g + 0], per = grats[4 * g + 1];
                double th = grats[4 * g + 2], ph = grats[4 * g + 3];
                val += a * sin(two_pi * ((double)u * cos(th) + (double)v * sin(th)) / per + ph);
            }
            tex[(int64_t)v * L + u] = val;
        }
    }
}

/* bilinear sample of the periodic table at real coordinates (u, v) */
static inline double sample_tex(const double *tex, int L, double u, double v) {
    double fl = (double)L;
    u = fmod(u, fl);
    if (u < 0.0) u += fl;
    v = fmod(v, fl);
    if (v < 0.0) v += fl;
    int iu = (int)floor(u), iv = (int)floor(v);
    if (iu >= L) iu = L - 1;
    if (iv >= L) iv = L - 1;
    double fu = u - (double)iu, fv = v - (double)iv;
    int iu1 = (iu + 1 == L) ? 0 : iu + 1;
    int iv1 = (iv + 1 == L) ? 0 : iv + 1;
    double t00 = tex[(int64_t)iv * L + iu], t01 = tex[(int64_t)iv * L + iu1];
    double t10 = tex[(int64_t)iv1 * L + iu], t11 = tex[(int64_t)iv1 * L + iu1];
    double top = (1.0 - fu) * t00 + fu * t01;
    double bot = (1.0 - fu) * t10 + fu * t11;
    return (1.0 - fv) * top + fv * bot;
}

/* ---------------------------------------------------------- simulator ---- */
/*
 * Scene: pixel (y, x) at step n sees tex(x + x0 + vx (n + 0.5), y + y0 + vy (n + 0.5))
 * multiplied by the product of the factors of every event e with t_e <= n whose
 * rectangle [y_lo, y_hi) x [x_lo, x_hi) contains the pixel, clipped to [ilo, ihi].
 * events: ne rows of (t, y_lo, x_lo, y_hi, x_hi, factor).
 * The initial accumulator is r0 = theta * U[0,1) from the counter hash (seed, p);
 * dark noise fires with probability noise_p per pixel-step (hash of seed, p, n).
 * If gt != NULL it receives the clipped intensity of every pixel at every
 * gt_stride-th step: gt[(n / gt_stride) * P + p] (fp32).
 * Returns 0, or -1 on bad arguments.
 */
int spkgen_simulate(uint8_t *out, int64_t pitch, int H, int W, int T,
                    const double *tex, int L, double x0, double y0, double vx, double vy,
                    int ne, const double *events, double ilo, double ihi, double theta,
                    uint64_t seed, double noise_p, float *gt, int gt_stride) {
    int64_t P = (int64_t)H * W;
    if (H <= 0 || W <= 0 || T <= 0 || pitch * 8 < P || L <= 0 || !(theta > 0.0)) return -1;
    if (gt && gt_stride <= 0) return -1;
    memset(out, 0, (size_t)pitch * (size_t)T);
    const int64_t BLK = 2048; /* pixels per work item: whole bytes */
    int64_t nblk = (P + BLK - 1) / BLK;
#pragma omp parallel
    {
        double *V = (double *)malloc(sizeof(double) * BLK);
        double *gain = (double *)malloc(sizeof(double) * BLK);
#pragma omp for schedule(dynamic, 1)
        for (int64_t b = 0; b < nblk; ++b) {
            int64_t p0 = b * BLK, p1 = p0 + BLK < P ? p0 + BLK : P;
            for (int64_t p = p0; p < p1; ++p) {
                V[p - p0] = theta * spkgen_uniform(seed, STREAM_R0, (uint64_t)p, 0);
                gain[p - p0] = 1.0;
            }
            for (int n = 0; n < T; ++n) {
                for (int e = 0; e < ne; ++e) {
                    const double *ev = events + 6 * e;
                    if ((int)ev[0] != n) continue;
                    for (int64_t p = p0; p < p1; ++p) {
                        int y = (int)(p / W), x = (int)(p % W);
                        if (y >= (int)ev[1] && y < (int)ev[3] && x >= (int)ev[2] && x < (int)ev[4])
                            gain[p - p0] *= ev[5];
                    }
                }
                double tc = (double)n + 0.5;
                double du = x0 + vx * tc, dv = y0 + vy * tc;
                uint8_t *row = out + (int64_t)n * pitch;
                for (int64_t p = p0; p < p1; ++p) {
                    int y = (int)(p / W), x = (int)(p % W);
                    double q = sample_tex(tex, L, (double)x + du, (double)y + dv) * gain[p - p0];
                    if (q < ilo) q = ilo;
                    if (q > ihi) q = ihi;
                    if (gt && n % gt_stride == 0) gt[(int64_t)(n / gt_stride) * P + p] = (float)q;
                    double v = V[p - p0] + q;
                    int fire = v >= theta;
                    if (fire) v -= theta;
                    V[p - p0] = v;
                    if (noise_p > 0.0 && spkgen_uniform(seed, STREAM_NOISE, (uint64_t)p, (uint64_t)n) < noise_p)
                        fire = 1;
                    if (fire) row[p >> 3] |= (uint8_t)(1u << (p & 7));
                }
            }
        }
        free(V);
        free(gain);
    }
    return 0;
}

/*
 * Eq. 2 for explicitly given per-pixel intensities: q[n * P + p] (fp64) and initial
 * accumulators r0[p].  Used by the small hand-made cases and by the pins.
 */
int spkgen_simulate_table(uint8_t *out, int64_t pitch, int64_t P, int T,
                          const double *q, const double *r0, double theta) {
    if (P <= 0 || T <= 0 || pitch * 8 < P || !(theta > 0.0)) return -1;
    memset(out, 0, (size_t)pitch * (size_t)T);
    for (int64_t p = 0; p < P; ++p) {
        double v = r0[p];
        for (int n = 0; n < T; ++n) {
            v += q[(int64_t)n * P + p];
            if (v >= theta) {
                v -= theta;
                out[(int64_t)n * pitch + (p >> 3)] |= (uint8_t)(1u << (p & 7));
            }
        }
    }
    return 0;
}
