/*
 * spk.h -- C ABI of the GB300 spike-camera reconstruction library (libspk.so).
 *
 * The library reconstructs intensity frames from the binary stream of a spike camera with
 * the two parameter-free methods of "High-speed and High-quality Vision Reconstruction of
 * Spike Camera with Spike Stability Theorem" (Zhang et al., arXiv 2412.11639):
 *   FSR (first-order stability reconstruction) and SSR (second-order), Sec. III-B.
 * For every pixel the stream S_0 (Eq. 2 output, one bit per step) gives the interval
 * stream S_1 (Def. 2, Eq. 5).  S_1 is cut greedily wherever the zero-order rule of Def. 2
 * (one value, or two values that differ by 1) would break; the breaking element opens the
 * next stable sequence (Sec. III-C).  SSR also cuts inside each FSR sequence wherever one
 * of the two second-order streams S_2 ('-': distances between occurrences of the smaller
 * value, '+': of the larger value, Fig. 1) breaks the same rule; such a break of S_2 cuts
 * S_1 after the element where the breaking distance starts.  A stable sequence of N
 * intervals spanning D steps has intensity threshold * N / D (Eq. 4, with the 8-bit scale
 * 255 generalised to `threshold`).
 *
 * Conventions shared by every entry point:
 *  - Time steps are 0-based, n = 0 .. T-1.  Interval i covers the steps (s_i, s_{i+1}].
 *  - Stream layout: uint8 [T][pitch], pitch = spk_pitch(H, W) = round_up(ceil(H*W/8), 16).
 *    Pixel p = y*W + x is bit (p % 8), least significant first, of byte p/8 of its frame.
 *    Padding bits and bytes are ignored.
 *  - Frame k (k = 0 .. T_out-1, T_out = spk_num_frames(T, stride)) samples t_k = k*stride
 *    and holds the value of the stable sequence covering t_k.  Steps up to the first spike
 *    take the first sequence's value, steps after the last spike the last one's (or 0
 *    under spk_config.edges), and a pixel with fewer than two spikes reads 0.  Frame
 *    layout: [T_out][H][W], row-major, 4, 2 or 1 bytes a value (spk_config.out_dtype).
 *  - Device pointers must be CUDA device (or managed) memory and 16-byte aligned.
 *  - Calls are asynchronous on the context's stream unless stated; spk_synchronize()
 *    waits and reports device-side failures.  A context is not thread-safe: use one per
 *    host thread.  No C++ exception crosses this boundary.
 *  - Return codes: SPK_OK (0) or one of the negative SPK_ERR_* codes; spk_last_error()
 *    then describes the failure.
 */
#ifndef SPK_H
#define SPK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum spk_status {
    SPK_OK = 0,
    SPK_ERR_ARG = -1,      /* bad argument: NULL, non-positive size, bad threshold,
                              misaligned or non-device pointer, size overflow, overlap */
    SPK_ERR_CUDA = -2,     /* a CUDA runtime or driver call failed */
    SPK_ERR_OOM = -3,      /* device or host allocation failed */
    SPK_ERR_TIMEOUT = -4,  /* a bounded device-side wait gave up (reported by spk_synchronize) */
    SPK_ERR_INTERNAL = -5  /* a device-side consistency check failed */
};

/* Frame value types.  SPK_U8 gives the 8-bit frames of a decoder (Sec. III-C with the 8-bit
 * scale of Eq. 4): threshold * N / D rounded half up and clamped to 255, computed exactly
 * in integers; it needs an integral threshold in 1 .. 65535. */
enum spk_dtype { SPK_F32 = 0, SPK_F16 = 1, SPK_U8 = 2 };

/* Frame edge policy bits (spk_config.edges).  The paper leaves the frames before the first
 * spike and after the last one open; by default they hold the first and the last stable
 * sequence's value.  SPK_ZERO_HEAD: frames at or before the first spike read 0.
 * SPK_ZERO_TAIL: frames after the last spike read 0.  TFP has no edges and ignores them;
 * spk_segments reports spans, not frames, and ignores them too. */
enum spk_edges { SPK_ZERO_HEAD = 1, SPK_ZERO_TAIL = 2 };

/* Reconstruction methods.  FSR and SSR are the paper's (Sec. III-B); TFI and TFP are the
 * physical-model baselines it compares them with (Sec. II, Tables II-III):
 *  SPK_TFI: theta / the interval (s_i, s_{i+1}] covering t_k (every interval is its own
 *           span, with the frame policy above);
 *  SPK_TFP: theta * (spikes in the tfp_window steps (t_k - L, t_k]) / L, steps before the
 *           stream counting as empty; whole streams only (no spk_stream, no spk_segments).
 *  SPK_NORDER: the general n-order stability tree of Sec. III-B (Fig. 1 caption) with
 *           n = stability_order levels (3..5; orders 1 and 2 are FSR and SSR): inside every
 *           stable sequence of a level-k stream the '-' and '+' streams of its two values
 *           (index distances between their occurrences) are segmented by the same rule,
 *           and each of their breaks cuts the level above after the element where the
 *           breaking distance ends.  Cuts of deep levels wait in a per-pixel ring (64 cuts,
 *           512 bytes, per pixel at first; owned by the context, or by a live stream, where
 *           they stay pending from piece to piece) until no earlier cut can appear; if a
 *           pixel needs more, the launch runs again with rings twice as large (a live
 *           stream's piece from a copy of its state taken before the launch), so every
 *           valid stream is reconstructed.  For this method spk_reconstruct, spk_segments
 *           and spk_run therefore wait for the device (synchronous; not for stream capture)
 *           and can also return SPK_ERR_OOM. */
enum spk_method { SPK_FSR = 1, SPK_SSR = 2, SPK_TFI = 3, SPK_TFP = 4, SPK_NORDER = 5 };

typedef struct spk_config {
    int method;         /* SPK_FSR, SPK_SSR, SPK_TFI, SPK_TFP or SPK_NORDER */
    int frame_stride;   /* >= 1: frame k samples step k * frame_stride */
    int out_dtype;      /* SPK_F32, SPK_F16 (the round-to-nearest-even of the fp32 value) or
                           SPK_U8 (integral threshold, see spk_dtype) */
    int device;         /* CUDA device ordinal */
    void *stream;       /* cudaStream_t to launch on; NULL = the legacy default stream */
    int tfp_window;     /* SPK_TFP only: window L in steps, 1..64 (the paper uses 32, 64) */
    int stability_order; /* SPK_NORDER only: levels n of the stability tree, 3..5 */
    int edges;          /* 0 or SPK_ZERO_HEAD | SPK_ZERO_TAIL (frame edge policy) */
} spk_config;

typedef struct spk_ctx spk_ctx;

/* Creates a context on cfg->device for one reconstruction method of the paper's problem
 * statement (Sec. II: a spike stream S_0 in, intensity images out; FSR and SSR of
 * Sec. III-B, the TFI and TFP baselines of Sec. II).  cfg fixes the method, the frame
 * stride and output type, the device and the CUDA stream every later call launches on.
 * Allocates a 16-byte device status word; scratch buffers are allocated lazily by the
 * calls that need them.  *out receives the handle (NULL on failure); spk_destroy frees it.
 * Errors: SPK_ERR_ARG (bad cfg), SPK_ERR_CUDA (no device), SPK_ERR_OOM. */
int spk_create(spk_ctx **out, const spk_config *cfg);

/* Frees every buffer owned by ctx.  NULL is a no-op returning SPK_OK. */
int spk_destroy(spk_ctx *ctx);

/* Bytes per frame of the stream layout: round_up(ceil(H*W/8), 16); -1 if H or W <= 0. */
int64_t spk_pitch(int H, int W);

/* Number of frames ceil(T / stride); -1 if T <= 0 or stride <= 0. */
int64_t spk_num_frames(int T, int stride);

/* Reconstructs every frame of one stream (Sec. III-B, Eq. 4).
 *   stream      device, uint8 [T][spk_pitch(H, W)], read only, owned by the caller
 *   H, W, T     sensor rows, columns, steps (> 0)
 *   threshold   finite, > 0: the scale of Eq. 4 (255 for 8-bit images, 1 for rates);
 *               integral, 1 .. 65535, for SPK_U8 frames
 *   out_frames  device, [T_out][H][W] of the context's out_dtype, written completely,
 *               owned by the caller; must not overlap `stream`
 * Asynchronous on the context's stream.  Errors: SPK_ERR_ARG, SPK_ERR_CUDA. */
int spk_reconstruct(spk_ctx *ctx, const uint8_t *stream, int H, int W, int T, float threshold,
                    void *out_frames);

/* Same reconstruction with HOST buffers: copies the stream to a device buffer owned by the
 * context (allocated on first use, grown as needed), reconstructs and waits.
 * host_stream: uint8 [T][pitch]; host_frames: [T_out][H][W] of out_dtype.  If host_frames
 * is page-locked memory mapped into the device's address space (cudaHostAlloc, pinned torch
 * tensors), the kernel writes the frames into it directly over the host link; otherwise
 * they go to a context-owned device buffer and are copied back.  Page-locked host_stream
 * makes its copy asynchronous DMA.  Synchronous.
 * Errors: SPK_ERR_ARG, SPK_ERR_CUDA, SPK_ERR_OOM, SPK_ERR_TIMEOUT, SPK_ERR_INTERNAL. */
int spk_reconstruct_host(spk_ctx *ctx, const uint8_t *host_stream, int H, int W, int T,
                         float threshold, void *host_frames);

/* Asynchronous spk_reconstruct_host: enqueues the host-to-device copy of the stream, the
 * reconstruction into a device buffer and the device-to-host copy of the frames (always by a
 * copy engine, which keeps the SMs free for the next call's scan), and returns.  Consecutive
 * calls alternate between two internal lanes (a stream and a pair of device buffers each,
 * grown on demand), so that one call's device-to-host copy overlaps the next call's input
 * copy and scan.  Work already enqueued on ctx's stream is ordered before the call.  host_stream and
 * host_frames must stay untouched until spk_synchronize(ctx) returns; it waits for every
 * call and reports device errors.  Pinned host memory keeps the copies asynchronous.
 * Errors: as spk_reconstruct_host. */
int spk_reconstruct_host_async(spk_ctx *ctx, const uint8_t *host_stream, int H, int W, int T,
                               float threshold, void *host_frames);

/* A live stream: pushed piece by piece (spk_run), with its per-pixel scan state resident
 * in device memory between pieces, so that pieces arriving over time give exactly the
 * frames of one spk_reconstruct over the whole stream.  The FPGA of Sec. III-C carries the
 * same state across its 32-frame chunks. */
typedef struct spk_stream spk_stream;

/* Opens a stream of H x W pixels and T steps on ctx (its method -- FSR, SSR, TFI or the
 * n-order tree --, frame stride and output type) and allocates its device state: 20 int32
 * per pixel (the stability scan, the frames already written, the cut that opens the
 * current span, up to two pending cut candidates) and one int32; for the n-order tree
 * 11 + 8 x (7 + max(1, 2^n - 8)) int32 per pixel of scan and node state (75, 131, 259 for
 * n = 3, 4, 5), its pending-cut rings (512 bytes per pixel at first), and a copy of both.
 * TFP has no live streams.  Errors: SPK_ERR_ARG, SPK_ERR_CUDA, SPK_ERR_OOM. */
int spk_stream_open(spk_ctx *ctx, int H, int W, int T, spk_stream **out);

/* Waits for ctx's stream and frees the stream's device state.  NULL is a no-op. */
int spk_stream_close(spk_ctx *ctx, spk_stream *s);

/* Steps pushed so far (the absolute step of the next piece's first row); -1 for NULL. */
int64_t spk_stream_steps(const spk_stream *s);

/* Waits for ctx's stream; *ready receives the number of leading frames that are final for
 * every pixel after the last piece pushed (a frame is final once the stable span covering
 * it has closed; all T_out frames after the last piece).  Errors: SPK_ERR_ARG, SPK_ERR_CUDA. */
int spk_stream_ready(spk_ctx *ctx, const spk_stream *s, int64_t *ready);

/* One unit of work for spk_run. */
typedef struct spk_job {
    const uint8_t *stream; /* device, uint8 [n][spk_pitch(H, W)], 16-byte aligned */
    int H, W;              /* sensor rows and columns (must match `state` if given) */
    int n;                 /* steps in this piece, > 0 */
    float threshold;       /* as for spk_reconstruct; the same for every piece of a stream */
    void *out_frames;      /* device, [T_out][H][W] of ctx's out_dtype, T_out frames of the whole
                              stream; each frame is written at its absolute index */
    spk_stream *state;     /* NULL: the piece is a whole stream of T = n steps.  Otherwise the
                              piece holds steps [spk_stream_steps(state), ... + n) of that
                              stream; the piece that reaches its T ends it (tail frames) */
} spk_job;

/* Runs every job in one kernel launch (at most 96 jobs per launch; larger calls are split
 * into consecutive launches): the blocks of all jobs share the GPU, so many streams of
 * uneven size and length -- and the next pieces of many live streams -- are processed
 * together.  Each job gives the frames of Sec. III-B exactly as spk_reconstruct would.
 * A stream may appear at most once per call; outputs of different jobs must not overlap.
 * Asynchronous on ctx's stream (synchronous for SPK_NORDER; see spk_method).  Errors:
 * SPK_ERR_ARG (bad job, piece past the stream's T, repeated stream, a live stream with TFP
 * or opened for another method), SPK_ERR_CUDA, and for SPK_NORDER SPK_ERR_OOM. */
int spk_run(spk_ctx *ctx, const spk_job *jobs, int njobs);

/* Time tile of the frames kernels: the steps one TMA box stages per block (32, 64 or 128;
 * 64 by default).  Results do not depend on it; speed does.  Errors: SPK_ERR_ARG. */
int spk_set_tile(spk_ctx *ctx, int tile);

/* The context's current time tile; -1 for NULL. */
int spk_get_tile(const spk_ctx *ctx);

/* Autotuner: runs the given whole-stream jobs (state == NULL; they are run repeatedly)
 * once to warm up and three times timed with each time tile, keeps the fastest in ctx and
 * returns it in *best_tile (may be NULL).  Synchronous.  Errors: as spk_run, and
 * SPK_ERR_ARG for stream jobs. */
int spk_autotune(spk_ctx *ctx, const spk_job *jobs, int njobs, int *best_tile);

/* Verification export: per pixel the spike count K and the stable sequences themselves
 * (the records the paper's FPGA encoder emits, Sec. III-C).  For pixel p:
 *   spike_counts[p]  K, the number of spikes of the pixel in the T steps: S_1 (Def. 2,
 *                    Eq. 5) has K - 1 intervals, so K < 2 leaves no sequence.  May be NULL.
 *   counts[p]        the number of stable sequences;
 *   sequence j < cap is written at index j*H*W + p of t_start (spike time opening it),
 *   t_end (spike time closing it), n_int (number of intervals N) and value
 *   (threshold * N / (t_end - t_start), fp32, Eq. 4).
 * cap may be 0 (counts only; the four sequence arrays may then be NULL).  All pointers
 * are int32 / fp32 device memory owned by the caller.  SPK_TFP has no sequences and is
 * rejected.  Asynchronous.  Errors: SPK_ERR_ARG, SPK_ERR_CUDA. */
int spk_segments(spk_ctx *ctx, const uint8_t *stream, int H, int W, int T, float threshold,
                 int32_t *spike_counts, int32_t *counts, int32_t *t_start, int32_t *t_end,
                 int32_t *n_int, float *value, int cap);

/* Waits for the context's stream, then reads and clears the device status word:
 * SPK_ERR_TIMEOUT if a bounded device wait gave up, SPK_ERR_INTERNAL if a consistency
 * check failed, SPK_ERR_CUDA if the stream reported an error, else SPK_OK. */
int spk_synchronize(spk_ctx *ctx);

/* Human-readable description of the last failure on ctx ("" if none).  Valid until the
 * next call on ctx.  A NULL ctx returns the message of the last failed spk_create. */
const char *spk_last_error(const spk_ctx *ctx);

/* Number of kernel launches this context has issued since it was created. */
int64_t spk_launch_count(const spk_ctx *ctx);

/* ------------------------------------------------------------- learned refiner ----
 * A learned extension of the plain method (no counterpart in the paper, which is
 * parameter free): a 5-layer 3x3 convolutional network (16 -> 32 -> 32 -> 32 -> 32 -> 1
 * channels, ReLU, bf16 weights and activations, fp32 accumulation on the tensor cores)
 * that reads, per pixel and frame, the plain reconstruction and the rates theta / x of the
 * last four intervals, and returns plain + a learned correction.  Trained with the mean
 * squared error to a ground-truth intensity (Adam).  The plain frames remain the
 * fallback and the reference its error is measured against. */

/* Refiner input for every frame of a stream: device bf16, 16 channels per pixel stored as
 * two channel-chunk planes, [T_out][H][2][W][8] (channel c of pixel (y, x) of frame k at
 * ((k*H + y)*2 + c/8)*W*8 + x*8 + c%8).
 * Channel 0 = plain[k][p] (device fp32 [T_out][H][W], e.g. the frames of spk_reconstruct
 * with SPK_F32); channels 4..7 = threshold / x for the last four intervals x completed at
 * or before t_k = k * stride (the most recent first, 0 where the pixel has fewer); the
 * other channels 0.  Uses ctx's frame_stride.  Asynchronous.
 * Errors: SPK_ERR_ARG (NULL, misaligned, not device memory), SPK_ERR_CUDA. */
int spk_features(spk_ctx *ctx, const uint8_t *stream, int H, int W, int T, float threshold,
                 const float *plain, void *x0);

typedef struct spk_refiner spk_refiner;

/* Number of fp32 parameters of the network (weights [9][Cout][Cin] and biases per layer). */
int64_t spk_refiner_num_params(void);

/* Creates a refiner on `device` with seeded He-uniform weights (the last layer scaled by
 * 0.1 so that an untrained refiner returns about the plain value).  Allocates its
 * parameters, Adam moments and (lazily) its activation workspace.
 * Errors: SPK_ERR_CUDA, SPK_ERR_OOM. */
int spk_refiner_create(int device, uint64_t seed, spk_refiner **out);

/* Waits for the device and frees the refiner.  NULL is a no-op. */
int spk_refiner_destroy(spk_refiner *r);

/* Description of the last refiner failure (NULL: of the last failed create). */
const char *spk_refiner_last_error(const spk_refiner *r);

/* Loads n == spk_refiner_num_params() fp32 parameters from host memory (a checkpoint)
 * and resets the Adam state.  Synchronous.  Errors: SPK_ERR_ARG, SPK_ERR_CUDA. */
int spk_refiner_set_params(spk_refiner *r, const float *host, int64_t n);

/* Copies the parameters (which = 0) or the gradient of the last train step (which = 1)
 * to host memory.  Synchronous.  Errors: SPK_ERR_ARG, SPK_ERR_CUDA. */
int spk_refiner_get_params(spk_refiner *r, float *host, int64_t n, int which);

/* out[n][y][x] = plain + network(x0) for N frames of H x W pixels.  x0: device bf16
 * [N][H][2][W][8] (spk_features' layout), plain and out: device fp32 [N][H][W].  Runs on `stream`
 * (a cudaStream_t, NULL = legacy default); asynchronous.  N, H < 65536.
 * Errors: SPK_ERR_ARG, SPK_ERR_CUDA, SPK_ERR_OOM. */
int spk_refiner_forward(spk_refiner *r, void *stream, const void *x0, const float *plain, int N,
                        int H, int W, float *out);

/* One Adam step (lr, beta1 0.9, beta2 0.999) on the mean squared error between the
 * refined frames and gt (device fp32 [N][H][W]).  If loss_host is not NULL it receives
 * the batch's mean squared error before the step (this synchronises `stream`).
 * Errors: SPK_ERR_ARG, SPK_ERR_CUDA, SPK_ERR_OOM. */
int spk_refiner_train_step(spk_refiner *r, void *stream, const void *x0, const float *plain,
                           const float *gt, int N, int H, int W, float lr, float *loss_host);

/* Waits for `stream` (a cudaStream_t) and reports the refiner kernels' status: SPK_OK, or
 * SPK_ERR_TIMEOUT if a convolution gave up its bounded wait for the tensor cores (the
 * status is then cleared), SPK_ERR_CUDA on a CUDA error.  spk_refiner_train_step with a
 * loss_host performs the same check. */
int spk_refiner_synchronize(spk_refiner *r, void *stream);

/* Test hook of the failure paths (no counterpart in the paper): the library's next n device
 * allocations (contexts, stream states, host-call staging buffers) fail as if the device
 * were out of memory, so that the SPK_ERR_OOM paths can be exercised without exhausting a
 * shared GPU.  n = 0 clears it.  Errors: SPK_ERR_ARG for n < 0. */
int spk_debug_fail_allocations(int n);

/* Test hook of the n-order rings (no counterpart in the paper): later SPK_NORDER calls
 * start with rings of `cap` cuts per pixel (a power of two; 0 restores the default 64), so
 * that the regrowth path can be exercised on small streams.  Errors: SPK_ERR_ARG. */
int spk_debug_norder_capacity(int cap);

/* Diagnostic of the bounded device waits (no counterpart in the paper).  Every wait of
 * the kernels (the mbarrier waits of the stream pipeline) gives up after a bounded time
 * (about 2 s) instead of hanging, sets the timeout bit of the context's status word and
 * returns.  This call launches one warp that waits, through the same code, on a barrier
 * nothing will complete, with the limit limit_cycles (0 .. 4e9 SM clock cycles).  The
 * following spk_synchronize(ctx) must return SPK_ERR_TIMEOUT, after which the context is
 * usable again.  Asynchronous.  Errors: SPK_ERR_ARG, SPK_ERR_CUDA. */
int spk_selftest_wait(spk_ctx *ctx, int64_t limit_cycles);

/* Device scratch of spk_reconstruct_host_noalloc, in bytes (16 MiB). */
#define SPK_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Host-buffer reconstruction that allocates nothing (the paper has no counterpart: this
 * is a deployment variant of spk_reconstruct_host).
 *
 * Some callers cannot call cudaMalloc: processes whose device memory is owned entirely
 * by another allocator or held to a fixed budget (an allocation outside it fails or is
 * forbidden), and latency-critical camera loops that must not pay for an allocation or
 * for the device-wide synchronisation a cudaFree implies.  This entry point needs no
 * context (spk_create allocates) and stages the stream and the frames in one file-scope
 * device array of SPK_NOALLOC_SCRATCH_BYTES that the library's module holds on every
 * device it is loaded on, until the process exits.  It calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *
 *   cfg           method, frame_stride, out_dtype, device, stream, tfp_window,
 *                 stability_order, as for
 *                 spk_create
 *                 (the stream must belong to cfg->device)
 *   host_stream   host, uint8 [T][spk_pitch(H, W)]
 *   host_frames   host, [T_out][H][W] of cfg->out_dtype, written completely
 * The scratch holds a 256-byte status block, the stream and the frames, each rounded up
 * to 256 bytes, and for SPK_NORDER the pending-cut rings (512 bytes per pixel at first):
 * 256 + round_up(T*pitch, 256) + round_up(T_out*H*W*sizeof(out), 256) (+ 512*H*W) must not
 * exceed SPK_NOALLOC_SCRATCH_BYTES, else the call returns SPK_ERR_ARG before any device
 * work.  An n-order stream whose rings must grow beyond the rest of the array returns
 * SPK_ERR_INTERNAL (spk_reconstruct_host grows them instead).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture begins.
 * Every call shares the one array: a call clears the status word it needs, but two calls
 * whose device work overlaps (other host threads, or other streams) race on the array
 * and corrupt each other's results -- serialise them.  Synchronous: returns after the
 * frames are in host_frames.  spk_last_error(NULL) describes a failure.
 * Errors: SPK_ERR_ARG, SPK_ERR_CUDA, SPK_ERR_TIMEOUT, SPK_ERR_INTERNAL. */
int spk_reconstruct_host_noalloc(const spk_config *cfg, const uint8_t *host_stream, int H, int W,
                                 int T, float threshold, void *host_frames);

#ifdef __cplusplus
}
#endif

#endif /* SPK_H */
