/*
 * bnzref.h -- interface of the CPU oracle (test infrastructure only).
 * This header belongs to the oracle alone; the GPU library never includes it.
 */
#ifndef BNZREF_H
#define BNZREF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { BNZREF_OK = 0, BNZREF_EINVAL = 1, BNZREF_ENOMEM = 2 };
enum { BNZREF_SAUVOLA = 0, BNZREF_NIBLACK = 1 };
enum { BNZREF_NAIVE = 0, BNZREF_SLIDING = 1 };

int bnzref_gray(const uint8_t *src, int h, int w, int ch, long long pitch, uint8_t *gray);
int bnzref_window_sums_naive(const uint8_t *f, int h, int w, int W, int64_t *n, int64_t *s1, int64_t *s2);
int bnzref_window_sums_sliding(const uint8_t *f, int h, int w, int W, int64_t *n, int64_t *s1, int64_t *s2);
double bnzref_threshold_value(int64_t n, int64_t s1, int64_t s2, int rule, double k, double R);
int bnzref_decide(int f, int64_t n, int64_t s1, int64_t s2, int rule, double k, double R, int *tie, double *t_out);
int bnzref_threshold(const uint8_t *f, const int64_t *n, const int64_t *s1, const int64_t *s2, int h, int w,
                     int rule, double k, double R, uint8_t *out, int64_t *ties);
int bnzref_binarize(const uint8_t *src, int h, int w, int ch, long long src_pitch, int W, int rule, double k,
                    double R, int method, uint8_t *dst, long long dst_pitch, int64_t *ties, int nthreads);
int bnzref_pixel(const uint8_t *src, int h, int w, int ch, long long src_pitch, int W, int rule, double k,
                 double R, int y, int x, int *tie, double *t_out);
int bnzref_integral(const uint8_t *f, int h, int w, int64_t *I1, int64_t *I2);
int bnzref_pack(const uint8_t *mask, int h, int w, long long mask_pitch, uint8_t *packed, long long packed_pitch);
/* Otsu's global threshold and the Eq. 2 mask (see bnzref.c for the definition and the readings). */
int bnzref_histogram(const uint8_t *src, int h, int w, int ch, long long pitch, uint64_t *hist);
int bnzref_otsu_threshold(const uint64_t *hist, double *q_out);
int bnzref_otsu(const uint8_t *src, int h, int w, int ch, long long pitch, uint8_t *dst, long long dst_pitch,
                int *T_out);

/* Reduced sets S' of Sec. 2 (Eq. 5; structures proposed here, see bnzref.c) and Eq. 6 confusion counts. */
int bnzref_gs_member(int gs, int W, int dy, int dx);
int bnzref_gs_offsets(int gs, int W, int *dy, int *dx, int cap);
int bnzref_gs_sums(const uint8_t *f, int h, int w, int W, int gs, int64_t *n, int64_t *s1, int64_t *s2);
int bnzref_gs_binarize(const uint8_t *src, int h, int w, int ch, long long src_pitch, int W, int gs, int rule,
                       double k, double R, uint8_t *dst, long long dst_pitch, int64_t *ties);
int bnzref_confusion(const uint8_t *mask, long long mask_pitch, int mask_ink, const uint8_t *ref, long long ref_pitch,
                     int ref_ink, int h, int w, int64_t *counts);

#ifdef __cplusplus
}
#endif
#endif
