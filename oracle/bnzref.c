/*
 * bnzref.c -- plain, slow, obviously correct CPU oracle for exact locally
 * adaptive binarization (Sauvola and Niblack rules).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * bench's CPU-baseline / reference arm may load it.  It shares no code,
 * header, table or constant with the GPU library, and it never calls it.
 *
 * What it computes (the paper's definitions, with the readings this project
 * fixes where the paper is silent):
 *   - Gray conversion, Eq. 1 (Sec. 1): f = 0.299 r + 0.587 g + 0.114 b.  The
 *     paper states the weights but no rounding; the reading used here is the
 *     integer rule f = (299 r + 587 g + 114 b + 500) / 1000 (round half up).
 *   - Window set S, Sec. 2: the W x W window around (x, y).  W odd: centred.
 *     W even: r_lo = W/2 rows/cols before the pixel, r_hi = W/2 - 1 after.
 *     At the borders the window is clipped to the image and n = |S| varies.
 *   - Local mean m and standard deviation s over S, Sec. 1 and Sec. 2
 *     (population standard deviation, via the exact integer variance
 *     numerator V = n*S2 - S1^2).
 *   - Sauvola threshold, Eq. 4: t = m * (1 + k * (s / R - 1)).
 *   - Niblack threshold (cited in Sec. 1, formula not printed): t = m + k*s.
 *   - Decision, Eq. 3: g = 0 if f < t, else 255.
 *   All sums are exact 64-bit integers.  m, s, t are evaluated in IEEE fp64 in
 *   exactly this order, with no FMA contraction (build with
 *   -ffp-contract=off):
 *       m = (double)S1 / (double)n
 *       s = sqrt((double)V) / (double)n
 *       Sauvola: t = m * (1.0 + k * (s / R - 1.0))
 *       Niblack: t = m + k * s
 *   A "tie" is a pixel with |f - t| < 1e-9; ties are counted.
 *   - Global rule, Eq. 2 (g = 0 if f < T, else 255) with Otsu's T (cited in
 *     Sec. 1 as the best global method, formula not printed): see
 *     bnzref_otsu_threshold below.
 *
 * Two independent window-sum paths are provided:
 *   A. naive: sum over the clipped window for every pixel, O(W^2) per pixel
 *      (the direct evaluation the paper measures against, O(W^2 N^2) overall).
 *   B. sliding: along each row, the window sum of pixel x+1 is that of pixel
 *      x plus the entering column minus the leaving column, each a sum over
 *      the window's rows -- O(W) per pixel and no extra image-sized memory,
 *      the complexity and memory bound of Sec. 3 (O(W N^2), 2 S_z + c).
 *   A and B must agree bit-exactly.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "bnzref.h"

/* Window extent before / after the centre pixel (Sec. 2, reading for even W). */
static void bnzref_radii(int W, int *r_lo, int *r_hi)
{
    *r_lo = W / 2;
    *r_hi = W - 1 - *r_lo;
}

static int imax(int a, int b) { return a > b ? a : b; }
static int imin(int a, int b) { return a < b ? a : b; }

/* Eq. 1 with the integer round-half-up reading. */
static uint8_t bnzref_gray_px(const uint8_t *rgb)
{
    int r = rgb[0], g = rgb[1], b = rgb[2];
    return (uint8_t)((299 * r + 587 * g + 114 * b + 500) / 1000);
}

int bnzref_gray(const uint8_t *src, int h, int w, int ch, long long pitch, uint8_t *gray)
{
    if (!src || !gray || h < 0 || w < 0 || (ch != 1 && ch != 3) || pitch < (long long)w * ch)
        return BNZREF_EINVAL;
    for (int y = 0; y < h; ++y) {
        const uint8_t *row = src + (long long)y * pitch;
        uint8_t *out = gray + (long long)y * w;
        for (int x = 0; x < w; ++x)
            out[x] = (ch == 1) ? row[x] : bnzref_gray_px(row + 3 * x);
    }
    return BNZREF_OK;
}

/* Path A: direct sums over the clipped window of one pixel. */
static void naive_pixel(const uint8_t *f, int h, int w, int W, int y, int x,
                        int64_t *n, int64_t *s1, int64_t *s2)
{
    int r_lo, r_hi;
    bnzref_radii(W, &r_lo, &r_hi);
    int y0 = imax(0, y - r_lo), y1 = imin(h - 1, y + r_hi);
    int x0 = imax(0, x - r_lo), x1 = imin(w - 1, x + r_hi);
    int64_t a = 0, b = 0, c = 0;
    for (int yy = y0; yy <= y1; ++yy)
        for (int xx = x0; xx <= x1; ++xx) {
            int64_t v = f[(long long)yy * w + xx];
            a += 1;
            b += v;
            c += v * v;
        }
    *n = a;
    *s1 = b;
    *s2 = c;
}

int bnzref_window_sums_naive(const uint8_t *f, int h, int w, int W,
                             int64_t *n, int64_t *s1, int64_t *s2)
{
    if (!f || !n || !s1 || !s2 || h < 1 || w < 1 || W < 1)
        return BNZREF_EINVAL;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            long long i = (long long)y * w + x;
            naive_pixel(f, h, w, W, y, x, &n[i], &s1[i], &s2[i]);
        }
    return BNZREF_OK;
}

/* Sum of f and f^2 over rows [y0, y1] of one column x (0 if x is outside). */
static void column_sum(const uint8_t *f, int w, int y0, int y1, int x, int64_t *a, int64_t *b)
{
    int64_t p = 0, q = 0;
    for (int yy = y0; yy <= y1; ++yy) {
        int64_t v = f[(long long)yy * w + x];
        p += v;
        q += v * v;
    }
    *a = p;
    *b = q;
}

/* Path B for one row: O(W) per pixel, entering minus leaving column. */
static void sliding_row(const uint8_t *f, int h, int w, int W, int y,
                        int64_t *n, int64_t *s1, int64_t *s2)
{
    int r_lo, r_hi;
    bnzref_radii(W, &r_lo, &r_hi);
    int y0 = imax(0, y - r_lo), y1 = imin(h - 1, y + r_hi);
    int64_t rows = y1 - y0 + 1;
    int64_t a = 0, b = 0;
    /* window of pixel x = 0: columns [0, min(w-1, r_hi)] */
    for (int xx = 0; xx <= imin(w - 1, r_hi); ++xx) {
        int64_t p, q;
        column_sum(f, w, y0, y1, xx, &p, &q);
        a += p;
        b += q;
    }
    for (int x = 0; x < w; ++x) {
        if (x > 0) {
            int xin = x + r_hi, xout = x - r_lo - 1;
            int64_t p, q;
            if (xin < w) {
                column_sum(f, w, y0, y1, xin, &p, &q);
                a += p;
                b += q;
            }
            if (xout >= 0) {
                column_sum(f, w, y0, y1, xout, &p, &q);
                a -= p;
                b -= q;
            }
        }
        int cols = imin(w - 1, x + r_hi) - imax(0, x - r_lo) + 1;
        n[x] = rows * cols;
        s1[x] = a;
        s2[x] = b;
    }
}

int bnzref_window_sums_sliding(const uint8_t *f, int h, int w, int W,
                               int64_t *n, int64_t *s1, int64_t *s2)
{
    if (!f || !n || !s1 || !s2 || h < 1 || w < 1 || W < 1)
        return BNZREF_EINVAL;
    for (int y = 0; y < h; ++y) {
        long long o = (long long)y * w;
        sliding_row(f, h, w, W, y, n + o, s1 + o, s2 + o);
    }
    return BNZREF_OK;
}

/* Eq. 4 / Niblack threshold in the fixed fp64 order stated at the top. */
double bnzref_threshold_value(int64_t n, int64_t s1, int64_t s2, int rule, double k, double R)
{
    int64_t V = n * s2 - s1 * s1;
    double m = (double)s1 / (double)n;
    double s = sqrt((double)V) / (double)n;
    if (rule == BNZREF_SAUVOLA)
        return m * (1.0 + k * (s / R - 1.0));
    return m + k * s;
}

/* Eq. 3 decision; returns 0 or 255 and flags a tie (|f - t| < 1e-9). */
int bnzref_decide(int f, int64_t n, int64_t s1, int64_t s2, int rule, double k, double R,
                  int *tie, double *t_out)
{
    double t = bnzref_threshold_value(n, s1, s2, rule, k, R);
    double d = (double)f - t;
    if (tie)
        *tie = fabs(d) < 1e-9;
    if (t_out)
        *t_out = t;
    return ((double)f < t) ? 0 : 255;
}

int bnzref_threshold(const uint8_t *f, const int64_t *n, const int64_t *s1, const int64_t *s2,
                     int h, int w, int rule, double k, double R, uint8_t *out, int64_t *ties)
{
    if (!f || !n || !s1 || !s2 || !out || h < 1 || w < 1)
        return BNZREF_EINVAL;
    int64_t nt = 0;
    for (long long i = 0; i < (long long)h * w; ++i) {
        int tie = 0;
        out[i] = (uint8_t)bnzref_decide(f[i], n[i], s1[i], s2[i], rule, k, R, &tie, NULL);
        nt += tie;
    }
    if (ties)
        *ties = nt;
    return BNZREF_OK;
}

/* ---- full pipeline, row bands on threads ---------------------------------- */

typedef struct {
    const uint8_t *f;
    int h, w, W, rule, method, y_begin, y_end;
    double k, R;
    uint8_t *dst;
    long long dst_pitch;
    int64_t ties;
} band_job;

static void *band_worker(void *arg)
{
    band_job *j = (band_job *)arg;
    int w = j->w;
    int64_t *n = (int64_t *)malloc(sizeof(int64_t) * (size_t)w);
    int64_t *a = (int64_t *)malloc(sizeof(int64_t) * (size_t)w);
    int64_t *b = (int64_t *)malloc(sizeof(int64_t) * (size_t)w);
    j->ties = 0;
    if (!n || !a || !b) {
        j->ties = -1;
        free(n);
        free(a);
        free(b);
        return NULL;
    }
    for (int y = j->y_begin; y < j->y_end; ++y) {
        if (j->method == BNZREF_NAIVE) {
            for (int x = 0; x < w; ++x)
                naive_pixel(j->f, j->h, w, j->W, y, x, &n[x], &a[x], &b[x]);
        } else {
            sliding_row(j->f, j->h, w, j->W, y, n, a, b);
        }
        const uint8_t *frow = j->f + (long long)y * w;
        uint8_t *out = j->dst + (long long)y * j->dst_pitch;
        for (int x = 0; x < w; ++x) {
            int tie = 0;
            out[x] = (uint8_t)bnzref_decide(frow[x], n[x], a[x], b[x], j->rule, j->k, j->R, &tie, NULL);
            j->ties += tie;
        }
    }
    free(n);
    free(a);
    free(b);
    return NULL;
}

int bnzref_binarize(const uint8_t *src, int h, int w, int ch, long long src_pitch, int W,
                    int rule, double k, double R, int method, uint8_t *dst, long long dst_pitch,
                    int64_t *ties, int nthreads)
{
    if (!src || !dst || h < 1 || w < 1 || (ch != 1 && ch != 3) || W < 1 ||
        src_pitch < (long long)w * ch || dst_pitch < w ||
        (rule != BNZREF_SAUVOLA && rule != BNZREF_NIBLACK) ||
        (method != BNZREF_NAIVE && method != BNZREF_SLIDING))
        return BNZREF_EINVAL;
    if (rule == BNZREF_SAUVOLA && !(R > 0.0))
        return BNZREF_EINVAL;
    uint8_t *f = (uint8_t *)malloc((size_t)h * (size_t)w);
    if (!f)
        return BNZREF_ENOMEM;
    bnzref_gray(src, h, w, ch, src_pitch, f);
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > h)
        nthreads = h;
    band_job *jobs = (band_job *)calloc((size_t)nthreads, sizeof(band_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tids) {
        free(f);
        free(jobs);
        free(tids);
        return BNZREF_ENOMEM;
    }
    for (int t = 0; t < nthreads; ++t) {
        band_job *j = &jobs[t];
        j->f = f;
        j->h = h;
        j->w = w;
        j->W = W;
        j->rule = rule;
        j->method = method;
        j->k = k;
        j->R = R;
        j->dst = dst;
        j->dst_pitch = dst_pitch;
        j->y_begin = (int)((long long)h * t / nthreads);
        j->y_end = (int)((long long)h * (t + 1) / nthreads);
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&tids[t], NULL, band_worker, &jobs[t]) != 0)
            break;
        started = t;
    }
    band_worker(&jobs[0]);
    for (int t = started + 1; t < nthreads; ++t)
        band_worker(&jobs[t]); /* threads that could not start run inline */
    for (int t = 1; t <= started; ++t)
        pthread_join(tids[t], NULL);
    int64_t total = 0;
    int rc = BNZREF_OK;
    for (int t = 0; t < nthreads; ++t) {
        if (jobs[t].ties < 0)
            rc = BNZREF_ENOMEM;
        else
            total += jobs[t].ties;
    }
    if (ties)
        *ties = total;
    free(f);
    free(jobs);
    free(tids);
    return rc;
}

int bnzref_pixel(const uint8_t *src, int h, int w, int ch, long long src_pitch, int W,
                 int rule, double k, double R, int y, int x, int *tie, double *t_out)
{
    if (!src || h < 1 || w < 1 || (ch != 1 && ch != 3) || W < 1 || y < 0 || y >= h ||
        x < 0 || x >= w || src_pitch < (long long)w * ch)
        return -1;
    int r_lo, r_hi;
    bnzref_radii(W, &r_lo, &r_hi);
    int y0 = imax(0, y - r_lo), y1 = imin(h - 1, y + r_hi);
    int x0 = imax(0, x - r_lo), x1 = imin(w - 1, x + r_hi);
    int64_t n = 0, a = 0, b = 0;
    for (int yy = y0; yy <= y1; ++yy) {
        const uint8_t *row = src + (long long)yy * src_pitch;
        for (int xx = x0; xx <= x1; ++xx) {
            int64_t v = (ch == 1) ? row[xx] : bnzref_gray_px(row + 3 * xx);
            n += 1;
            a += v;
            b += v * v;
        }
    }
    const uint8_t *crow = src + (long long)y * src_pitch;
    int f = (ch == 1) ? crow[x] : bnzref_gray_px(crow + 3 * x);
    return bnzref_decide(f, n, a, b, rule, k, R, tie, t_out);
}

/* Summed-area tables as defined for the integral-image method (Sec. 1):
 * I1[y][x] = sum of f over rows < y and cols < x, I2 likewise for f^2,
 * both (h+1) x (w+1), first row and column zero, int64. */
int bnzref_integral(const uint8_t *f, int h, int w, int64_t *I1, int64_t *I2)
{
    if (!f || !I1 || !I2 || h < 0 || w < 0)
        return BNZREF_EINVAL;
    long long W1 = (long long)w + 1;
    for (long long x = 0; x < W1; ++x) {
        I1[x] = 0;
        I2[x] = 0;
    }
    for (int y = 0; y < h; ++y) {
        I1[(y + 1) * W1] = 0;
        I2[(y + 1) * W1] = 0;
        int64_t ra = 0, rb = 0;
        for (int x = 0; x < w; ++x) {
            int64_t v = f[(long long)y * w + x];
            ra += v;
            rb += v * v;
            I1[(y + 1) * W1 + x + 1] = I1[y * W1 + x + 1] + ra;
            I2[(y + 1) * W1 + x + 1] = I2[y * W1 + x + 1] + rb;
        }
    }
    return BNZREF_OK;
}

/* 1 bit per pixel, row-major, LSB of each byte = leftmost pixel,
 * bit 1 <=> output value 255; trailing bits of the last byte are 0. */
int bnzref_pack(const uint8_t *mask, int h, int w, long long mask_pitch, uint8_t *packed,
                long long packed_pitch)
{
    long long pb = ((long long)w + 7) / 8;
    if (!mask || !packed || h < 0 || w < 0 || mask_pitch < w || packed_pitch < pb)
        return BNZREF_EINVAL;
    for (int y = 0; y < h; ++y) {
        const uint8_t *m = mask + (long long)y * mask_pitch;
        uint8_t *p = packed + (long long)y * packed_pitch;
        memset(p, 0, (size_t)pb);
        for (int x = 0; x < w; ++x)
            if (m[x] == 255)
                p[x >> 3] |= (uint8_t)(1u << (x & 7));
    }
    return BNZREF_OK;
}

/* ---- Otsu's global threshold ------------------------------------------------
 * Sec. 1 names Otsu's method as the best global technique; Eq. 2 applies one
 * threshold T to every pixel: g = 0 if f < T, else 255.  The paper gives no
 * formula for T; Otsu's published definition is used: over the histogram of f
 * (Eq. 1 gray), T in [1, 255] splits the levels into [0, T-1] and [T, 255] with
 * counts n0, n1 and level sums s0, s1 (N = n0 + n1, S = s0 + s1), and T
 * maximises the between-class variance
 *     w0 w1 (mu0 - mu1)^2 = (N s0 - S n0)^2 / (N^2 n0 n1).
 * D = N s0 - S n0 is formed exactly in 128-bit integers; the criterion, an
 * argmax decided in floating point, is q(T) = (d * d) / (a * b) in fp64 with
 * d = (double)D, a = (double)n0, b = (double)n1.  The smallest T with the
 * largest q wins; T = 0 (every pixel 255) when no T leaves both classes
 * non-empty (a page of one gray level). */

int bnzref_histogram(const uint8_t *src, int h, int w, int ch, long long pitch, uint64_t *hist)
{
    if (!src || !hist || h < 0 || w < 0 || (ch != 1 && ch != 3) || pitch < (long long)w * ch)
        return BNZREF_EINVAL;
    for (int i = 0; i < 256; ++i)
        hist[i] = 0;
    for (int y = 0; y < h; ++y) {
        const uint8_t *row = src + (long long)y * pitch;
        for (int x = 0; x < w; ++x)
            hist[ch == 1 ? row[x] : bnzref_gray_px(row + 3 * x)]++;
    }
    return BNZREF_OK;
}

int bnzref_otsu_threshold(const uint64_t *hist, double *q_out)
{
    __int128 N = 0, S = 0;
    for (int i = 0; i < 256; ++i) {
        N += (__int128)hist[i];
        S += (__int128)hist[i] * i;
    }
    __int128 n0 = 0, s0 = 0;
    int best_t = 0;
    double best_q = -1.0;
    for (int t = 1; t < 256; ++t) {
        n0 += (__int128)hist[t - 1];
        s0 += (__int128)hist[t - 1] * (t - 1);
        const __int128 n1 = N - n0;
        double q = -1.0; /* no split */
        if (n0 > 0 && n1 > 0) {
            const __int128 D = N * s0 - S * n0;
            const double d = (double)D, a = (double)n0, b = (double)n1;
            q = (d * d) / (a * b);
        }
        if (q_out)
            q_out[t] = q;
        if (q > best_q) {
            best_q = q;
            best_t = t;
        }
    }
    if (q_out)
        q_out[0] = -1.0;
    return best_q < 0.0 ? 0 : best_t;
}

int bnzref_otsu(const uint8_t *src, int h, int w, int ch, long long pitch, uint8_t *dst, long long dst_pitch,
                int *T_out)
{
    uint64_t hist[256];
    int rc = bnzref_histogram(src, h, w, ch, pitch, hist);
    if (rc != BNZREF_OK)
        return rc;
    if (!dst || dst_pitch < w)
        return BNZREF_EINVAL;
    const int T = bnzref_otsu_threshold(hist, NULL);
    for (int y = 0; y < h; ++y) {
        const uint8_t *row = src + (long long)y * pitch;
        uint8_t *out = dst + (long long)y * dst_pitch;
        for (int x = 0; x < w; ++x) {
            const int f = ch == 1 ? row[x] : bnzref_gray_px(row + 3 * x);
            out[x] = f < T ? 0 : 255; /* Eq. 2 */
        }
    }
    if (T_out)
        *T_out = T;
    return BNZREF_OK;
}

/* ---- reduced sets S' (Sec. 2, Eq. 5) ----------------------------------------
 *
 * Sec. 2 replaces the window set S by a reduced set S' of pixels sampled from
 * the window in a geometric order, and Eq. 5 evaluates Sauvola's rule on the
 * mean m' and standard deviation s' of S' with a dynamic range R'.  The
 * structures themselves are drawn in Fig. 1, which is not available, so the
 * six below are proposed here (they are not the paper's drawings).  Each has
 * O(W) samples, as the O(W N^2) bound of Sec. 3.2 requires.  Offsets (dy, dx)
 * run over the window [-r_lo, r_hi]^2 (bnzref_radii); with lo = -r_lo and
 * hi = r_hi:
 *   0  the whole window (S' = S: Eq. 5 is Eq. 4)
 *   1  cross        dy == 0 or dx == 0
 *   2  diagonals    dy == dx or dy == -dx
 *   3  star         cross or diagonals
 *   4  frame        dy in {lo, hi} or dx in {lo, hi}
 *   5  frame or cross
 *   6  frame or diagonals
 * As for S, samples outside the image are dropped and n' counts the others;
 * m' = S1'/n' and s' = sqrt(n' S2' - S1'^2)/n' (population deviation), and the
 * decision is Eq. 3 on t' with the fp64 order of bnzref_threshold_value
 * (Niblack's rule on m', s' likewise).  Every sum is exact. */
int bnzref_gs_member(int gs, int W, int dy, int dx)
{
    int r_lo, r_hi;
    bnzref_radii(W, &r_lo, &r_hi);
    if (dy < -r_lo || dy > r_hi || dx < -r_lo || dx > r_hi)
        return 0;
    const int cross = dy == 0 || dx == 0;
    const int diag = dy == dx || dy == -dx;
    const int frame = dy == -r_lo || dy == r_hi || dx == -r_lo || dx == r_hi;
    switch (gs) {
    case 0: return 1;
    case 1: return cross;
    case 2: return diag;
    case 3: return cross || diag;
    case 4: return frame;
    case 5: return frame || cross;
    case 6: return frame || diag;
    default: return 0;
    }
}

/* The offsets of S' in row-major order; returns their number (-1: bad args).
 * dy, dx may be NULL to count only; otherwise they hold at least cap entries. */
int bnzref_gs_offsets(int gs, int W, int *dy, int *dx, int cap)
{
    if (W < 1 || gs < 0 || gs > 6)
        return -1;
    int r_lo, r_hi, n = 0;
    bnzref_radii(W, &r_lo, &r_hi);
    for (int a = -r_lo; a <= r_hi; ++a)
        for (int b = -r_lo; b <= r_hi; ++b) {
            if (!bnzref_gs_member(gs, W, a, b))
                continue;
            if (dy && dx) {
                if (n >= cap)
                    return -1;
                dy[n] = a;
                dx[n] = b;
            }
            ++n;
        }
    return n;
}

/* n', S1', S2' of every pixel: the in-image samples of S' summed one by one
 * (O(|S'|) = O(W) per pixel, the evaluation Sec. 3.2 counts). */
int bnzref_gs_sums(const uint8_t *f, int h, int w, int W, int gs, int64_t *n, int64_t *s1, int64_t *s2)
{
    if (!f || !n || !s1 || !s2 || h < 1 || w < 1)
        return BNZREF_EINVAL;
    const int cnt = bnzref_gs_offsets(gs, W, NULL, NULL, 0);
    if (cnt < 1)
        return BNZREF_EINVAL;
    int *dy = (int *)malloc(sizeof(int) * (size_t)cnt);
    int *dx = (int *)malloc(sizeof(int) * (size_t)cnt);
    if (!dy || !dx) {
        free(dy);
        free(dx);
        return BNZREF_ENOMEM;
    }
    bnzref_gs_offsets(gs, W, dy, dx, cnt);
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            int64_t c = 0, a = 0, b = 0;
            for (int i = 0; i < cnt; ++i) {
                const int yy = y + dy[i], xx = x + dx[i];
                if (yy < 0 || yy >= h || xx < 0 || xx >= w)
                    continue;
                const int64_t v = f[(long long)yy * w + xx];
                ++c;
                a += v;
                b += v * v;
            }
            const long long i = (long long)y * w + x;
            n[i] = c;
            s1[i] = a;
            s2[i] = b;
        }
    free(dy);
    free(dx);
    return BNZREF_OK;
}

/* Eq. 1 gray, the reduced-set sums and the Eq. 3 decision on t' (Eq. 5 for
 * Sauvola with R' = R); ties |f - t'| < 1e-9 counted. */
int bnzref_gs_binarize(const uint8_t *src, int h, int w, int ch, long long src_pitch, int W, int gs, int rule,
                       double k, double R, uint8_t *dst, long long dst_pitch, int64_t *ties)
{
    if (!src || !dst || h < 1 || w < 1 || (ch != 1 && ch != 3) || W < 1 || gs < 0 || gs > 6 ||
        src_pitch < (long long)w * ch || dst_pitch < w || (rule != BNZREF_SAUVOLA && rule != BNZREF_NIBLACK))
        return BNZREF_EINVAL;
    if (rule == BNZREF_SAUVOLA && !(R > 0.0))
        return BNZREF_EINVAL;
    const size_t np = (size_t)h * (size_t)w;
    uint8_t *f = (uint8_t *)malloc(np);
    int64_t *n = (int64_t *)malloc(np * sizeof(int64_t));
    int64_t *a = (int64_t *)malloc(np * sizeof(int64_t));
    int64_t *b = (int64_t *)malloc(np * sizeof(int64_t));
    uint8_t *out = (uint8_t *)malloc(np);
    int rc = BNZREF_ENOMEM;
    if (f && n && a && b && out) {
        bnzref_gray(src, h, w, ch, src_pitch, f);
        rc = bnzref_gs_sums(f, h, w, W, gs, n, a, b);
        if (rc == BNZREF_OK)
            rc = bnzref_threshold(f, n, a, b, h, w, rule, k, R, out, ties);
        if (rc == BNZREF_OK)
            for (int y = 0; y < h; ++y)
                memcpy(dst + (long long)y * dst_pitch, out + (long long)y * w, (size_t)w);
    }
    free(f);
    free(n);
    free(a);
    free(b);
    free(out);
    return rc;
}

/* ---- F-measure, Eq. 6 ---------------------------------------------------------
 * Confusion counts of a binarized mask against a reference mask, the text
 * (foreground) of each being the pixels equal to its ink value: counts[0] =
 * TP (ink in both), [1] = FP (ink in the mask only), [2] = FN (ink in the
 * reference only), [3] = TN.  Eq. 6 then needs R = TP/(TP+FN), P = TP/(TP+FP). */
int bnzref_confusion(const uint8_t *mask, long long mask_pitch, int mask_ink, const uint8_t *ref, long long ref_pitch,
                     int ref_ink, int h, int w, int64_t *counts)
{
    if (!mask || !ref || !counts || h < 0 || w < 0 || mask_pitch < w || ref_pitch < w)
        return BNZREF_EINVAL;
    int64_t c[4] = {0, 0, 0, 0};
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            const int a = mask[(long long)y * mask_pitch + x] == mask_ink;
            const int b = ref[(long long)y * ref_pitch + x] == ref_ink;
            c[a ? (b ? 0 : 1) : (b ? 2 : 3)]++;
        }
    memcpy(counts, c, sizeof c);
    return BNZREF_OK;
}
