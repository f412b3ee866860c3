/*
 * The C ABI used from plain C (no Python): a stream whose pixel p spikes every (p % 7) + 1
 * steps has constant intervals, so every frame of every pixel is theta / interval (Eq. 4 of
 * one stable sequence).  Reconstructs it through spk_reconstruct_host and the asynchronous
 * variant, checks every frame, and checks the error codes of a few bad calls.  Then the
 * same stream as 8-bit frames (theta 255: round(255 / interval), halves up) with both edges
 * zeroed (frames at or before the first spike and after the last one read 0).
 * Prints "abi_demo ok" and returns 0 on success.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "spk.h"

#define H 3
#define W 50
#define T 700

static int check(const float *frames, int T_out, int stride, float theta) {
    int P = H * W;
    for (int k = 0; k < T_out; ++k)
        for (int p = 0; p < P; ++p) {
            float want = theta / (float)((p % 7) + 1);
            float got = frames[(size_t)k * P + p];
            if (fabsf(got - want) > 1e-6f * want) {
                fprintf(stderr, "frame %d pixel %d: %g != %g (stride %d)\n", k, p, got, want, stride);
                return 1;
            }
        }
    return 0;
}

int main(void) {
    int P = H * W;
    int pitch = spk_pitch(H, W);
    uint8_t *stream = calloc((size_t)T * pitch, 1);
    for (int t = 0; t < T; ++t)
        for (int p = 0; p < P; ++p)
            if (t % ((p % 7) + 1) == 0) stream[(size_t)t * pitch + p / 8] |= (uint8_t)(1u << (p % 8));

    spk_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.method = SPK_SSR;
    cfg.frame_stride = 5;
    cfg.out_dtype = SPK_F32;
    cfg.device = 0;
    cfg.stream = NULL;
    cfg.tfp_window = 32;
    cfg.stability_order = 3;
    spk_ctx *ctx = NULL;
    if (spk_create(&ctx, &cfg) != SPK_OK) {
        fprintf(stderr, "spk_create: %s\n", spk_last_error(NULL));
        return 1;
    }
    int T_out = spk_num_frames(T, cfg.frame_stride);
    float *frames = malloc(sizeof(float) * (size_t)T_out * P);
    float *frames2 = malloc(sizeof(float) * (size_t)T_out * P);
    if (spk_reconstruct_host(ctx, stream, H, W, T, 1.0f, frames) != SPK_OK) {
        fprintf(stderr, "spk_reconstruct_host: %s\n", spk_last_error(ctx));
        return 1;
    }
    if (check(frames, T_out, cfg.frame_stride, 1.0f)) return 1;
    if (spk_reconstruct_host_async(ctx, stream, H, W, T, 2.0f, frames) != SPK_OK ||
        spk_reconstruct_host_async(ctx, stream, H, W, T, 4.0f, frames2) != SPK_OK || spk_synchronize(ctx) != SPK_OK) {
        fprintf(stderr, "async: %s\n", spk_last_error(ctx));
        return 1;
    }
    if (check(frames, T_out, cfg.frame_stride, 2.0f) || check(frames2, T_out, cfg.frame_stride, 4.0f)) return 1;
    /* bad calls come back as error codes, the context stays usable */
    if (spk_reconstruct_host(ctx, stream, 0, W, T, 1.0f, frames) != SPK_ERR_ARG) return 1;
    if (spk_reconstruct_host(ctx, stream, H, W, T, -1.0f, frames) != SPK_ERR_ARG) return 1;
    if (spk_reconstruct_host(ctx, NULL, H, W, T, 1.0f, frames) != SPK_ERR_ARG) return 1;
    if (spk_reconstruct_host(ctx, stream, H, W, T, 1.0f, frames) != SPK_OK) return 1;
    if (check(frames, T_out, cfg.frame_stride, 1.0f)) return 1;
    spk_destroy(ctx);

    /* 8-bit frames with the zero-head and zero-tail policy */
    cfg.out_dtype = SPK_U8;
    cfg.edges = SPK_ZERO_HEAD | SPK_ZERO_TAIL;
    if (spk_create(&ctx, &cfg) != SPK_OK) {
        fprintf(stderr, "spk_create (u8): %s\n", spk_last_error(NULL));
        return 1;
    }
    uint8_t *f8 = malloc((size_t)T_out * P);
    if (spk_reconstruct_host(ctx, stream, H, W, T, 1.5f, f8) != SPK_ERR_ARG) return 1; /* integral theta */
    if (spk_reconstruct_host(ctx, stream, H, W, T, 255.0f, f8) != SPK_OK) {
        fprintf(stderr, "spk_reconstruct_host (u8): %s\n", spk_last_error(ctx));
        return 1;
    }
    for (int k = 0; k < T_out; ++k)
        for (int p = 0; p < P; ++p) {
            const int d = (p % 7) + 1, t = k * cfg.frame_stride, last = ((T - 1) / d) * d;
            int want = (2 * 255 + d) / (2 * d);
            if (want > 255) want = 255;
            if (t <= 0 || t > last) want = 0;
            if (f8[(size_t)k * P + p] != want) {
                fprintf(stderr, "u8 frame %d pixel %d: %d != %d\n", k, p, f8[(size_t)k * P + p], want);
                return 1;
            }
        }
    spk_destroy(ctx);
    free(f8);
    free(stream);
    free(frames);
    free(frames2);
    printf("abi_demo ok\n");
    return 0;
}
