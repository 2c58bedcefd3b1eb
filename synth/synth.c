/*
 * synth.c -- seeded synthetic document pages (uint8 gray or interleaved RGB).
 *
 * The pages imitate the degradations of the document images the method is
 * evaluated on (uneven illumination, stains, camera noise): a linear
 * illumination gradient, dark 1-3 px strokes grouped in text-like glyph
 * boxes, optional coloured stains and low-frequency blotches, optional
 * vignetting, and Gaussian noise.  Every random draw comes from a
 * counter-based generator (SplitMix64 finaliser applied to a key built from
 * the seed, a stream id and an index), so the output does not depend on the
 * number of threads.
 *
 * This module holds no part of the binarization method: it never converts
 * colour to gray, never sums windows and never thresholds.  Both the oracle
 * tests and the GPU tests/bench draw their inputs from it.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYNTH_PI 3.14159265358979323846

enum { PROF_DOC = 0, PROF_STAINS = 1, PROF_VIGNETTE = 2 };
enum { FLAG_RANDOM_DIR = 1 };

static uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t key3(uint64_t seed, uint64_t stream, uint64_t idx)
{
    return mix64(mix64(seed ^ (stream * 0xD1B54A32D192ED03ull)) ^ idx);
}

/* uniform in [0, 1) */
static double u01(uint64_t seed, uint64_t stream, uint64_t idx)
{
    return (double)(key3(seed, stream, idx) >> 11) * (1.0 / 9007199254740992.0);
}

/* standard normal by Box-Muller from two counter draws */
static double gauss(uint64_t seed, uint64_t stream, uint64_t idx)
{
    double a = u01(seed, stream, 2 * idx);
    double b = u01(seed, stream, 2 * idx + 1);
    if (a < 1e-300)
        a = 1e-300;
    return sqrt(-2.0 * log(a)) * cos(2.0 * SYNTH_PI * b);
}

typedef struct {
    double cx, cy, ax, ay, cs, sn, tint[3], strength;
} stain_t;

typedef struct {
    double cx, cy, sig, amp;
} blotch_t;

typedef struct {
    uint8_t *out;
    int h, w, ch, profile;
    long long pitch;
    uint64_t seed;
    uint8_t *gt; /* ink mask, h*w, always allocated internally */
    double g0, g1, dirx, diry, noise_sigma;
    double paper[3];
    int nst, nbl;
    stain_t st[8];
    blotch_t bl[6];
    /* text layout */
    int fs, line_pitch, margin_x, margin_y, nlines;
    int y_begin, y_end, line_begin, line_end;
} job_t;

/* distance-to-segment rasterisation of one stroke into the ink mask */
static void draw_segment(uint8_t *gt, int h, int w, double ax, double ay, double bx, double by,
                         double half)
{
    int x0 = (int)floor(fmin(ax, bx) - half - 1), x1 = (int)ceil(fmax(ax, bx) + half + 1);
    int y0 = (int)floor(fmin(ay, by) - half - 1), y1 = (int)ceil(fmax(ay, by) + half + 1);
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > w - 1) x1 = w - 1;
    if (y1 > h - 1) y1 = h - 1;
    double dx = bx - ax, dy = by - ay, L2 = dx * dx + dy * dy;
    for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x) {
            double px = x + 0.5 - ax, py = y + 0.5 - ay;
            double t = L2 > 0 ? (px * dx + py * dy) / L2 : 0.0;
            if (t < 0) t = 0;
            if (t > 1) t = 1;
            double ex = px - t * dx, ey = py - t * dy;
            if (ex * ex + ey * ey <= half * half)
                gt[(long long)y * w + x] = 1;
        }
}

/* text lines [line_begin, line_end): glyph boxes made of random strokes */
static void draw_lines(job_t *j)
{
    int w = j->w, h = j->h;
    for (int li = j->line_begin; li < j->line_end; ++li) {
        int top = j->margin_y + li * j->line_pitch;
        if (top + j->fs >= h - j->margin_y)
            break;
        double x = j->margin_x;
        uint64_t gi = 0;
        while (1) {
            uint64_t base = ((uint64_t)li << 24) + gi * 16;
            double gw = j->fs * (0.45 + 0.45 * u01(j->seed, 11, base));
            if (x + gw >= w - j->margin_x)
                break;
            int thick = 1 + (int)(3.0 * u01(j->seed, 11, base + 1)); /* 1..3 px */
            double half = 0.5 * thick;
            int nseg = 2 + (int)(3.0 * u01(j->seed, 11, base + 2));
            for (int s = 0; s < nseg; ++s) {
                double ax = x + gw * u01(j->seed, 12, base * 8 + 4 * s);
                double ay = top + j->fs * u01(j->seed, 12, base * 8 + 4 * s + 1);
                double bx = x + gw * u01(j->seed, 12, base * 8 + 4 * s + 2);
                double by = top + j->fs * u01(j->seed, 12, base * 8 + 4 * s + 3);
                draw_segment(j->gt, h, w, ax, ay, bx, by, half);
            }
            x += gw + j->fs * 0.18;
            if (u01(j->seed, 11, base + 3) < 0.18) /* word gap */
                x += j->fs * 0.6;
            ++gi;
        }
    }
}

static void *lines_worker(void *arg)
{
    draw_lines((job_t *)arg);
    return NULL;
}

static void compose_rows(job_t *j)
{
    int w = j->w, h = j->h;
    double cxv = 0.5 * (w - 1), cyv = 0.5 * (h - 1);
    double rmax2 = cxv * cxv + cyv * cyv + 1e-9;
    double ink_base = 40.0;
    for (int y = j->y_begin; y < j->y_end; ++y) {
        uint8_t *row = j->out + (long long)y * j->pitch;
        for (int x = 0; x < w; ++x) {
            long long idx = (long long)y * w + x;
            /* illumination gradient along (dirx, diry), 0..1 across the page */
            double u = (j->dirx >= 0 ? x : (w - 1 - x)) * fabs(j->dirx) / (w > 1 ? w - 1 : 1) +
                       (j->diry >= 0 ? y : (h - 1 - y)) * fabs(j->diry) / (h > 1 ? h - 1 : 1);
            double bg = j->g0 + (j->g1 - j->g0) * u;
            if (j->profile == PROF_VIGNETTE) {
                double dx = x - cxv, dy = y - cyv;
                bg *= 1.0 - 0.55 * (dx * dx + dy * dy) / rmax2;
            }
            double blot = 0.0;
            for (int b = 0; b < j->nbl; ++b) {
                double dx = x - j->bl[b].cx, dy = y - j->bl[b].cy;
                blot += j->bl[b].amp * exp(-(dx * dx + dy * dy) / (2 * j->bl[b].sig * j->bl[b].sig));
            }
            double tint[3] = {1.0, 1.0, 1.0};
            for (int s = 0; s < j->nst; ++s) {
                const stain_t *st = &j->st[s];
                double dx = x - st->cx, dy = y - st->cy;
                double p = (dx * st->cs + dy * st->sn) / st->ax, q = (-dx * st->sn + dy * st->cs) / st->ay;
                double r2 = p * p + q * q;
                if (r2 < 1.0) {
                    double a = st->strength * (1.0 - r2 * r2);
                    for (int c = 0; c < 3; ++c)
                        tint[c] *= 1.0 - a * (1.0 - st->tint[c]);
                }
            }
            int ink = j->gt[idx];
            double v = ink ? ink_base * (0.8 + 0.4 * bg / 220.0) : bg + blot;
            if (j->ch == 1) {
                double g = v * tint[0] + j->noise_sigma * gauss(j->seed, 21, (uint64_t)idx);
                g = floor(g + 0.5);
                row[x] = (uint8_t)(g < 0 ? 0 : g > 255 ? 255 : g);
            } else {
                for (int c = 0; c < 3; ++c) {
                    double g = v * (ink ? 1.0 : j->paper[c]) * tint[c] +
                               j->noise_sigma * gauss(j->seed, 22 + c, (uint64_t)idx);
                    g = floor(g + 0.5);
                    row[3 * x + c] = (uint8_t)(g < 0 ? 0 : g > 255 ? 255 : g);
                }
            }
        }
    }
}

static void *rows_worker(void *arg)
{
    compose_rows((job_t *)arg);
    return NULL;
}

static void run_parallel(job_t *base, int nthreads, int nitems, int lines_mode)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nitems) nthreads = nitems > 0 ? nitems : 1;
    job_t *jobs = (job_t *)malloc(sizeof(job_t) * (size_t)nthreads);
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    int *ok = (int *)calloc((size_t)nthreads, sizeof(int));
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *base;
        int b = (int)((long long)nitems * t / nthreads), e = (int)((long long)nitems * (t + 1) / nthreads);
        if (lines_mode) {
            jobs[t].line_begin = b;
            jobs[t].line_end = e;
        } else {
            jobs[t].y_begin = b;
            jobs[t].y_end = e;
        }
    }
    for (int t = 1; t < nthreads; ++t)
        ok[t] = pthread_create(&tid[t], NULL, lines_mode ? lines_worker : rows_worker, &jobs[t]) == 0;
    for (int t = 0; t < nthreads; ++t)
        if (t == 0 || !ok[t]) {
            if (lines_mode) draw_lines(&jobs[t]);
            else compose_rows(&jobs[t]);
        }
    for (int t = 1; t < nthreads; ++t)
        if (ok[t]) pthread_join(tid[t], NULL);
    free(jobs);
    free(tid);
    free(ok);
}

/*
 * out: h rows of `pitch` bytes, ch = 1 (gray) or 3 (r,g,b interleaved).
 * profile: 0 = plain page (sigma 8), 1 = page with stains and blotches (sigma 8),
 *          2 = strong vignetting (sigma 15).
 * flags & 1: draw the illumination direction from the seed (else left to right).
 * gt (nullable): h*w bytes, 1 where a stroke was drawn.
 */
int synth_page(uint8_t *out, int h, int w, int ch, long long pitch, uint64_t seed, int profile,
               int flags, uint8_t *gt_out, int nthreads)
{
    if (!out || h < 1 || w < 1 || (ch != 1 && ch != 3) || pitch < (long long)w * ch ||
        profile < 0 || profile > 2)
        return 1;
    job_t j;
    memset(&j, 0, sizeof(j));
    j.out = out;
    j.h = h;
    j.w = w;
    j.ch = ch;
    j.pitch = pitch;
    j.seed = seed;
    j.profile = profile;
    j.gt = gt_out ? gt_out : (uint8_t *)malloc((size_t)h * (size_t)w);
    if (!j.gt)
        return 2;
    memset(j.gt, 0, (size_t)h * (size_t)w);
    j.g0 = 90.0;
    j.g1 = 220.0;
    j.dirx = 1.0;
    j.diry = 0.0;
    if (flags & FLAG_RANDOM_DIR) {
        double a = 2 * SYNTH_PI * u01(seed, 1, 0);
        double cx = cos(a), sy = sin(a), s = fabs(cx) + fabs(sy);
        j.dirx = cx / s;
        j.diry = sy / s;
    }
    j.noise_sigma = profile == PROF_VIGNETTE ? 15.0 : 8.0;
    j.paper[0] = 1.0;
    j.paper[1] = 0.97;
    j.paper[2] = 0.90;
    if (profile == PROF_STAINS) {
        j.nst = 3 + (int)(4 * u01(seed, 2, 0));
        for (int s = 0; s < j.nst; ++s) {
            stain_t *st = &j.st[s];
            st->cx = w * u01(seed, 3, 8 * s);
            st->cy = h * u01(seed, 3, 8 * s + 1);
            double size = (w < h ? w : h);
            st->ax = size * (0.05 + 0.2 * u01(seed, 3, 8 * s + 2));
            st->ay = size * (0.05 + 0.2 * u01(seed, 3, 8 * s + 3));
            double ang = SYNTH_PI * u01(seed, 3, 8 * s + 4);
            st->cs = cos(ang);
            st->sn = sin(ang);
            double hue = u01(seed, 3, 8 * s + 5);
            st->tint[0] = 0.75 + 0.25 * hue;
            st->tint[1] = 0.60 + 0.3 * u01(seed, 3, 8 * s + 6);
            st->tint[2] = 0.45 + 0.4 * (1.0 - hue);
            st->strength = 0.3 + 0.5 * u01(seed, 3, 8 * s + 7);
        }
        j.nbl = 3 + (int)(3 * u01(seed, 4, 0));
        for (int b = 0; b < j.nbl; ++b) {
            j.bl[b].cx = w * u01(seed, 5, 4 * b);
            j.bl[b].cy = h * u01(seed, 5, 4 * b + 1);
            j.bl[b].sig = (w + h) * (0.04 + 0.1 * u01(seed, 5, 4 * b + 2));
            j.bl[b].amp = -35.0 + 55.0 * u01(seed, 5, 4 * b + 3);
        }
    }
    /* text layout: font size scales mildly with the page, 14..40 px */
    int smin = w < h ? w : h;
    double fs = smin / 60.0;
    if (fs < 14) fs = 14;
    if (fs > 40) fs = 40;
    j.fs = (int)(fs * (0.85 + 0.3 * u01(seed, 6, 0)));
    if (j.fs < 6) j.fs = 6;
    j.line_pitch = (int)(j.fs * 1.7) + 4;
    j.margin_x = w / 20;
    j.margin_y = h / 20;
    int avail = h - 2 * j.margin_y;
    j.nlines = avail > 0 ? avail / j.line_pitch : 0;
    run_parallel(&j, nthreads, j.nlines, 1);
    run_parallel(&j, nthreads, h, 0);
    if (!gt_out)
        free(j.gt);
    return 0;
}
