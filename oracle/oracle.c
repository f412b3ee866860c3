/*
 * ORACLE -- test infrastructure only.  Plain, slow, fp64 CPU restatement of the
 * paper's two parameter-free reconstructions (FSR and SSR, Sec. III-B) and of the
 * segment intensity of Eq. 4.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may call it; the product path never does.  It shares no code with
 * the CUDA path.
 *
 * Steps, per pixel, in the paper's order:
 *   1. spike times s_1 < ... < s_K of the binary stream S_0 (Eq. 2 output);
 *   2. interval stream S_1 = {T_0(i)}, T_0(i) = s_{i+1} - s_i (Def. 2, Eq. 5);
 *   3. FSR: break S_1 greedily wherever the next element would violate the
 *      zero-order rule (Def. 2: one value, or two values differing by 1); the
 *      violating element opens the next stable sequence (Sec. III-C, Fig. 4 text);
 *   4. SSR (order 2): inside each FSR sequence with values {a, a+1}, form S_2 for the
 *      '-' choice (firing value a) and the '+' choice (firing value a+1): the index
 *      distances between consecutive occurrences of that value in S_1 (Def. 2 applied
 *      to S_1, Fig. 1).  Break each S_2 greedily by the same zero-order rule; a break
 *      before distance d_j = q_{j+1} - q_j cuts S_1 after element q_j.  The cuts of
 *      both choices are united and split the FSR sequence (Sec. III-B);
 *   (order n > 2: the general n-order tree, oracle_segments_n);
 *   5. intensity of a stable sequence of N intervals: theta / ((1/N) sum T_0(i)) (Eq. 4,
 *      with 255 generalised to the threshold argument theta);
 *   6. frames: frame k samples t_k = k * stride and takes the value of the sequence
 *      covering t_k, a sequence of intervals i0..i1 covering the steps
 *      (s_{i0}, s_{i1+1}].  Steps up to s_1 take the first sequence's value, steps
 *      after s_K the last one's (or 0 under the zero edge policies), and a pixel with
 *      fewer than two spikes reads 0; 8-bit frames round theta * N / D half up (oracle_u8).
 *
 * Readings where the paper is silent (frame policy, cut position, hierarchy of the
 * two orders) are the ones listed in the design notes of this repository.
 *
 * Time indices are 0-based steps n = 0 .. T-1.  Values are fp64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the OpenMP loops over pixels (the CPU-baseline timing runs both 1 and all). */
void oracle_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

/* bit of pixel p in frame n of a [T][pitch] LSB-first packed stream */
static int spike_bit(const uint8_t *stream, int64_t pitch, int n, int64_t p) {
    return (stream[(int64_t)n * pitch + (p >> 3)] >> (p & 7)) & 1;
}

/* Step 1: spike times of pixel p; returns K. */
int oracle_spike_times(const uint8_t *stream, int64_t pitch, int T, int64_t p, int32_t *times) {
    int K = 0;
    for (int n = 0; n < T; ++n)
        if (spike_bit(stream, pitch, n, p)) times[K++] = n;
    return K;
}

/* zero-order rule of Def. 2 for a running range [lo, hi] of integers */
static int zero_order_ok(int lo, int hi) { return hi - lo <= 1; }

/*
 * Steps 2-5 for one pixel.  s[0..K-1] are spike times.  Writes up to K-1 segments:
 * t_start[j], t_end[j] (spike times bounding the segment), n_int[j] (number of
 * intervals N) and val[j] = theta * N / (t_end - t_start).  Returns the count.
 * work must hold 3 * K ints.
 */
int oracle_segments(const int32_t *s, int K, int order, double theta, int32_t *t_start,
                    int32_t *t_end, int32_t *n_int, double *val, int32_t *work) {
    if (K < 2) return 0;
    int n = K - 1;                    /* number of intervals */
    int32_t *x = work;                /* S_1 */
    int32_t *cut_after = work + n;    /* 1 if a stable sequence ends at this interval */
    int32_t *pos = work + 2 * n;      /* positions of one value inside a segment */
    for (int i = 0; i < n; ++i) {
        x[i] = s[i + 1] - s[i];
        cut_after[i] = 0;
    }
    cut_after[n - 1] = 1;

    /* Step 3: FSR, greedy zero-order segmentation of S_1. */
    int lo = x[0], hi = x[0];
    for (int i = 1; i < n; ++i) {
        int nlo = x[i] < lo ? x[i] : lo;
        int nhi = x[i] > hi ? x[i] : hi;
        if (zero_order_ok(nlo, nhi)) {
            lo = nlo;
            hi = nhi;
        } else {
            cut_after[i - 1] = 1;     /* the violating element opens the next sequence */
            lo = hi = x[i];
        }
    }

    /* Step 4: SSR, second-order test inside every FSR sequence. */
    if (order >= 2) {
        int i0 = 0;
        while (i0 < n) {
            int i1 = i0;
            while (!cut_after[i1]) ++i1;          /* FSR sequence [i0, i1] */
            int a = x[i0];
            for (int i = i0; i <= i1; ++i)
                if (x[i] < a) a = x[i];
            int fsr_end = i1;
            for (int v = a; v <= a + 1; ++v) {     /* '-' then '+' */
                int m = 0;
                for (int i = i0; i <= fsr_end; ++i)
                    if (x[i] == v) pos[m++] = i;
                if (m < 3) continue;              /* fewer than two distances: no break */
                int dlo = pos[1] - pos[0], dhi = dlo;
                for (int j = 1; j + 1 < m; ++j) {
                    int d = pos[j + 1] - pos[j];
                    int nlo = d < dlo ? d : dlo;
                    int nhi = d > dhi ? d : dhi;
                    if (zero_order_ok(nlo, nhi)) {
                        dlo = nlo;
                        dhi = nhi;
                    } else {
                        cut_after[pos[j]] = 1;   /* d_j spans S_1 elements pos[j]+1 .. pos[j+1] */
                        dlo = dhi = d;
                    }
                }
            }
            i0 = fsr_end + 1;
        }
    }

    /* Step 5: one value per stable sequence (Eq. 4). */
    int nseg = 0, i0 = 0;
    for (int i = 0; i < n; ++i) {
        if (!cut_after[i]) continue;
        int N = i - i0 + 1;
        int ts = s[i0], te = s[i + 1];
        t_start[nseg] = ts;
        t_end[nseg] = te;
        n_int[nseg] = N;
        double mean_interval = (double)(te - ts) / (double)N;   /* (1/N) sum T_0(i) */
        val[nseg] = theta / mean_interval;
        ++nseg;
        i0 = i + 1;
    }
    return nseg;
}

/*
 * General n-order stability (Sec. III-B and the caption of Fig. 1): the interval streams
 * S_1, S_2^1, S_2^2, S_3^1, ... are each broken greedily by the zero-order rule of Def. 2.
 * Inside every stable sequence of a level-k stream, whose values are {a, a+1}, the two
 * level-(k+1) streams are the index distances between consecutive occurrences of a (the
 * '-' choice) and of a+1 (the '+' choice).  A level-(k+1) stable sequence that ends at its
 * distance j (not the stream's last) cuts the level-k stream after the element at which
 * distance j ends, so that every cut lands, level by level, on S_1.  The tree stops at
 * level n, or where a stream has fewer than two elements (the empty S_n^m of Fig. 1).
 * Orders 1 and 2 are FSR and SSR.
 *
 * cut[i] = 1 marks a cut after element i of v[0 .. L-1]; the caller clears cut.
 */
static void norder_cuts(const int32_t *v, int L, int depth, int n, int32_t *cut) {
    int i0 = 0;
    while (i0 < L) {
        int lo = v[i0], hi = v[i0], i1 = i0;          /* greedy stable sequence [i0, i1] */
        while (i1 + 1 < L) {
            int nlo = v[i1 + 1] < lo ? v[i1 + 1] : lo;
            int nhi = v[i1 + 1] > hi ? v[i1 + 1] : hi;
            if (!zero_order_ok(nlo, nhi)) break;
            lo = nlo;
            hi = nhi;
            ++i1;
        }
        if (i1 < L - 1) cut[i1] = 1;
        if (depth < n) {
            for (int val = lo; val <= lo + 1; ++val) {  /* '-' then '+' */
                int m = 0;
                for (int i = i0; i <= i1; ++i)
                    if (v[i] == val) ++m;
                if (m < 3) continue;                  /* fewer than two distances: nothing to break */
                int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
                int32_t *d = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m - 1));
                int32_t *sub = (int32_t *)calloc((size_t)(m - 1), sizeof(int32_t));
                m = 0;
                for (int i = i0; i <= i1; ++i)
                    if (v[i] == val) pos[m++] = i;
                for (int j = 0; j + 1 < m; ++j) d[j] = pos[j + 1] - pos[j];
                norder_cuts(d, m - 1, depth + 1, n, sub);
                for (int j = 0; j + 2 < m; ++j)
                    if (sub[j]) cut[pos[j + 1]] = 1;  /* distance j ends at element pos[j+1] */
                free(pos);
                free(d);
                free(sub);
            }
        }
        i0 = i1 + 1;
    }
}

/* Steps 2-5 with the n-order tree in place of steps 3-4 (same outputs as oracle_segments). */
int oracle_segments_n(const int32_t *s, int K, int n, double theta, int32_t *t_start, int32_t *t_end,
                      int32_t *n_int, double *val) {
    if (K < 2 || n < 1) return 0;
    int L = K - 1;
    int32_t *x = (int32_t *)malloc(sizeof(int32_t) * (size_t)L);
    int32_t *cut = (int32_t *)calloc((size_t)L, sizeof(int32_t));
    for (int i = 0; i < L; ++i) x[i] = s[i + 1] - s[i];
    norder_cuts(x, L, 1, n, cut);
    cut[L - 1] = 1;                                  /* the last sequence ends at the last spike */
    int nseg = 0, i0 = 0;
    for (int i = 0; i < L; ++i) {
        if (!cut[i]) continue;
        int N = i - i0 + 1;
        int ts = s[i0], te = s[i + 1];
        t_start[nseg] = ts;
        t_end[nseg] = te;
        n_int[nseg] = N;
        val[nseg] = theta / ((double)(te - ts) / (double)N);   /* Eq. 4 */
        ++nseg;
        i0 = i + 1;
    }
    free(x);
    free(cut);
    return nseg;
}

/*
 * 8-bit output (the paper's decoder writes 8-bit frames, Sec. III-C, and Eq. 4 carries the
 * 8-bit scale 255): the value theta * N / D of a sequence of N intervals over D steps,
 * rounded half up and clamped to 255, in exact integer arithmetic for an integral theta:
 * floor((2 theta N + D) / (2 D)).
 */
int oracle_u8(int64_t theta, int64_t N, int64_t D) {
    int64_t v = (2 * theta * N + D) / (2 * D);
    return v > 255 ? 255 : (int)v;
}

/* Frame edge policy bits: frames up to the first spike read 0 instead of the first
 * sequence's value, frames after the last spike read 0 instead of the last one's. */
enum { ORACLE_ZERO_HEAD = 1, ORACLE_ZERO_TAIL = 2 };

/* Step 6 for one pixel: frames[k * fstride] for k = 0 .. ceil(T/stride)-1, under the edge
 * policy `edges`. */
void oracle_frames_edges(int K, int nseg, const int32_t *t_start, const int32_t *t_end,
                         const double *val, int T, int stride, int edges, double *frames, int64_t fstride) {
    int T_out = (T + stride - 1) / stride;
    int j = 0;
    for (int k = 0; k < T_out; ++k) {
        int64_t t = (int64_t)k * stride;
        double v;
        if (K < 2 || nseg == 0) {
            v = 0.0;
        } else if (t <= t_start[0]) {
            v = (edges & ORACLE_ZERO_HEAD) ? 0.0 : val[0];          /* up to the first spike */
        } else if (t > t_end[nseg - 1]) {
            v = (edges & ORACLE_ZERO_TAIL) ? 0.0 : val[nseg - 1];   /* after the last spike */
        } else {
            while (!(t_start[j] < t && t <= t_end[j])) ++j;   /* covering sequence */
            v = val[j];
        }
        frames[(int64_t)k * fstride] = v;
    }
}

/* Step 6 with head fill and tail hold. */
void oracle_frames(int K, int nseg, const int32_t *t_start, const int32_t *t_end,
                   const double *val, int T, int stride, double *frames, int64_t fstride) {
    oracle_frames_edges(K, nseg, t_start, t_end, val, T, stride, 0, frames, fstride);
}

/*
 * Whole-stream driver over a list of pixels (all pixels when pix == NULL), OpenMP over
 * pixels.  Any output pointer may be NULL.
 *   frames  [T_out][npix] fp64
 *   K       [npix] spike counts
 *   nseg    [npix] segment counts
 *   seg_off [npix+1] (input): if given together with seg_* buffers, pixel i's segments
 *           are written at seg_off[i] .. seg_off[i+1]-1; a pixel whose count differs
 *           from its slot size makes the call return -2.
 * Returns 0, -1 on bad arguments, -2 on a segment-slot mismatch.
 */
int oracle_reconstruct2(const uint8_t *stream, int64_t pitch, int64_t P, int T, double theta,
                        int order, int stride, const int64_t *pix, int64_t npix, double *frames,
                        int32_t *K_out, int32_t *nseg_out, const int64_t *seg_off,
                        int32_t *seg_ts, int32_t *seg_te, int32_t *seg_n, double *seg_val,
                        int edges, int u8);

int oracle_reconstruct(const uint8_t *stream, int64_t pitch, int64_t P, int T, double theta,
                       int order, int stride, const int64_t *pix, int64_t npix, double *frames,
                       int32_t *K_out, int32_t *nseg_out, const int64_t *seg_off,
                       int32_t *seg_ts, int32_t *seg_te, int32_t *seg_n, double *seg_val) {
    return oracle_reconstruct2(stream, pitch, P, T, theta, order, stride, pix, npix, frames, K_out, nseg_out,
                               seg_off, seg_ts, seg_te, seg_n, seg_val, 0, 0);
}

/* The same with a frame edge policy and, if u8, 8-bit frame values (oracle_u8 of each
 * sequence, theta integral) instead of fp64 ones. */
int oracle_reconstruct2(const uint8_t *stream, int64_t pitch, int64_t P, int T, double theta,
                        int order, int stride, const int64_t *pix, int64_t npix, double *frames,
                        int32_t *K_out, int32_t *nseg_out, const int64_t *seg_off,
                        int32_t *seg_ts, int32_t *seg_te, int32_t *seg_n, double *seg_val,
                        int edges, int u8) {
    if (u8 && (theta != (double)(int64_t)theta || theta < 1)) return -1;
    if (P <= 0 || T <= 0 || pitch * 8 < P || stride <= 0 || order < 1 || order > 32) return -1;
    if (pix == NULL) npix = P;
    int err = 0;
#pragma omp parallel
    {
        int32_t *s = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
        int32_t *ts = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
        int32_t *te = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
        int32_t *nn = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
        double *vv = (double *)malloc(sizeof(double) * (size_t)T);
        int32_t *work = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)T);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < npix; ++i) {
            int64_t p = pix ? pix[i] : i;
            if (p < 0 || p >= P) {
#pragma omp atomic write
                err = -1;
                continue;
            }
            int K = oracle_spike_times(stream, pitch, T, p, s);
            int ns = order <= 2 ? oracle_segments(s, K, order, theta, ts, te, nn, vv, work)
                                : oracle_segments_n(s, K, order, theta, ts, te, nn, vv);
            if (K_out) K_out[i] = K;
            if (nseg_out) nseg_out[i] = ns;
            if (seg_off && seg_ts) {
                if (seg_off[i + 1] - seg_off[i] != ns) {
#pragma omp atomic write
                    err = -2;
                } else {
                    int64_t o = seg_off[i];
                    memcpy(seg_ts + o, ts, sizeof(int32_t) * (size_t)ns);
                    memcpy(seg_te + o, te, sizeof(int32_t) * (size_t)ns);
                    memcpy(seg_n + o, nn, sizeof(int32_t) * (size_t)ns);
                    memcpy(seg_val + o, vv, sizeof(double) * (size_t)ns);
                }
            }
            if (frames) {
                if (u8)  /* the frame values become the 8-bit ones of the same sequences */
                    for (int q = 0; q < ns; ++q) vv[q] = (double)oracle_u8((int64_t)theta, nn[q], te[q] - ts[q]);
                oracle_frames_edges(K, ns, ts, te, vv, T, stride, edges, frames + i, npix);
            }
        }
        free(s);
        free(ts);
        free(te);
        free(nn);
        free(vv);
        free(work);
    }
    return err;
}

/*
 * Baselines of Sec. II (the paper compares FSR/SSR with them, Tables II-III).
 *
 * TFI (texture from inter-spike interval): the intensity is theta divided by the interval
 * between two adjacent spikes.  Frame k takes the interval (s_i, s_{i+1}] covering
 * t_k = k * stride; before the first spike the first interval, after the last spike the
 * last interval, fewer than two spikes 0 (the frame policy of the FSR/SSR frames).
 *
 * TFP (texture from playback): a virtual exposure window of L steps; the intensity is
 * theta * N_spk / L, N_spk the spikes in the window.  Frame k's window is the L steps
 * ending at t_k, (t_k - L, t_k]; steps before the stream count as empty.
 *
 * frames [T_out][npix] fp64 as in oracle_reconstruct; pix == NULL means all pixels.
 */
int oracle_tfi2(const uint8_t *stream, int64_t pitch, int64_t P, int T, double theta, int stride,
                const int64_t *pix, int64_t npix, double *frames, int edges, int u8);

int oracle_tfi(const uint8_t *stream, int64_t pitch, int64_t P, int T, double theta, int stride,
               const int64_t *pix, int64_t npix, double *frames) {
    return oracle_tfi2(stream, pitch, P, T, theta, stride, pix, npix, frames, 0, 0);
}

/* TFI under a frame edge policy, fp64 or 8-bit (oracle_u8 with N = 1) values. */
int oracle_tfi2(const uint8_t *stream, int64_t pitch, int64_t P, int T, double theta, int stride,
                const int64_t *pix, int64_t npix, double *frames, int edges, int u8) {
    if (P <= 0 || T <= 0 || pitch * 8 < P || stride <= 0) return -1;
    if (u8 && (theta != (double)(int64_t)theta || theta < 1)) return -1;
    if (pix == NULL) npix = P;
    int T_out = (T + stride - 1) / stride;
    int err = 0;
#pragma omp parallel
    {
        int32_t *s = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < npix; ++i) {
            int64_t p = pix ? pix[i] : i;
            if (p < 0 || p >= P) {
#pragma omp atomic write
                err = -1;
                continue;
            }
            int K = oracle_spike_times(stream, pitch, T, p, s);
            int j = 0;  /* interval j = (s_j, s_{j+1}] */
            for (int k = 0; k < T_out; ++k) {
                int64_t t = (int64_t)k * stride;
                double v = 0.0;
                if (K >= 2) {
                    while (j < K - 2 && t > s[j + 1]) ++j;
                    const int x = s[j + 1] - s[j];
                    v = u8 ? (double)oracle_u8((int64_t)theta, 1, x) : theta / (double)x;
                    if ((edges & ORACLE_ZERO_HEAD) && t <= s[0]) v = 0.0;
                    if ((edges & ORACLE_ZERO_TAIL) && t > s[K - 1]) v = 0.0;
                }
                frames[(int64_t)k * npix + i] = v;
            }
        }
        free(s);
    }
    return err;
}

int oracle_tfp2(const uint8_t *stream, int64_t pitch, int64_t P, int T, double theta, int stride, int L,
                const int64_t *pix, int64_t npix, double *frames, int u8);

int oracle_tfp(const uint8_t *stream, int64_t pitch, int64_t P, int T, double theta, int stride, int L,
               const int64_t *pix, int64_t npix, double *frames) {
    return oracle_tfp2(stream, pitch, P, T, theta, stride, L, pix, npix, frames, 0);
}

/* TFP with fp64 or 8-bit values (oracle_u8 of the count over the window). */
int oracle_tfp2(const uint8_t *stream, int64_t pitch, int64_t P, int T, double theta, int stride, int L,
                const int64_t *pix, int64_t npix, double *frames, int u8) {
    if (P <= 0 || T <= 0 || pitch * 8 < P || stride <= 0 || L <= 0) return -1;
    if (u8 && (theta != (double)(int64_t)theta || theta < 1)) return -1;
    if (pix == NULL) npix = P;
    int T_out = (T + stride - 1) / stride;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < npix; ++i) {
        int64_t p = pix ? pix[i] : i;
        if (p < 0 || p >= P) {
#pragma omp atomic write
            err = -1;
            continue;
        }
        for (int k = 0; k < T_out; ++k) {
            int64_t t = (int64_t)k * stride;
            int n = 0;
            for (int64_t u = t - L + 1; u <= t; ++u)
                if (u >= 0 && u < T && spike_bit(stream, pitch, (int)u, p)) ++n;
            frames[(int64_t)k * npix + i] = u8 ? (double)oracle_u8((int64_t)theta, n, L) : theta * (double)n / (double)L;
        }
    }
    return err;
}
