/*
 * bnz.h -- C ABI of the GB300 (sm_103a) locally adaptive binarization library.
 *
 * The library computes, for every pixel (x, y) of a uint8 page, the exact
 * integer sums S1 = sum f and S2 = sum f^2 over the W x W window around the
 * pixel (Sec. 2 of the paper: the window set S, "the most time consuming
 * operation"), the local mean m = S1/n and standard deviation
 * s = sqrt(n*S2 - S1^2)/n, the threshold t, and the binary value of Eq. 3:
 *     g(x, y) = 0 if f(x, y) < t(x, y), else 255.
 * Threshold rules:
 *     Sauvola, Eq. 4:  t = m * (1 + k * (s / R - 1))
 *     Niblack (cited in Sec. 1; formula not printed there): t = m + k * s
 * Colour input is converted with Eq. 1 (f = 0.299 r + 0.587 g + 0.114 b)
 * using the integer round-half-up rule f = (299 r + 587 g + 114 b + 500) / 1000.
 *
 * Conventions shared by every entry point:
 *   - Images are row-major.  `channels` is 1 (gray) or 3 (interleaved r,g,b).
 *     `height` = number of rows (M in the paper), `width` = columns (N).
 *   - W >= 1 is the full window side.  Odd W is centred; even W spans W/2
 *     pixels before the centre and W/2 - 1 after it (rows and columns).
 *     W <= BNZ_MAX_W.
 *   - Borders: the window is clipped to the image and n counts the pixels
 *     actually inside (no padding, no reflection).
 *   - m, s and t are decided exactly as an IEEE fp64 evaluation in the order
 *     m = S1/n, s = sqrt(V)/n, then the rule's formula left to right, would
 *     decide them.  The kernels filter with fp32 and a proven error margin and
 *     re-evaluate that fp64 sequence for the few pixels inside the margin, so
 *     every output byte equals that fp64 decision.
 *   - Output: a byte mask with values {0, 255} (dst_pitch >= width), or, with
 *     packed = 1, one bit per pixel: byte x/8 of a row holds pixel x in bit
 *     x%8 (LSB = leftmost), bit set <=> 255, unused trailing bits are 0
 *     (dst_pitch >= (width + 7) / 8).
 *   - Ownership: the caller owns every buffer.  The library keeps no pointer
 *     after a synchronous call returns, or after the stream passes an
 *     asynchronous call.
 *   - Errors: every call returns a bnz_status and never aborts the process.
 *     bnz_last_error() returns a message for the calling thread's last
 *     failure.  There is no CPU fallback: without a CUDA device the calls
 *     return BNZ_ENODEV.
 *   - Statistics (optional, `d_stats`): device pointer to 4 unsigned 64-bit
 *     counters that the kernels add to (the caller zeroes them):
 *       [0] pixels re-evaluated past the fp32 filter (inside its proven
 *           margin: for Niblack a tighter fp32 evaluation of n (f - t) with a
 *           per-pixel bound, then double-float, then the fp64 definition near
 *           a tie),
 *       [1] ties: pixels with |f - t| < 1e-9,
 *       [2] bounded waits that timed out: a CTA that gives up writes no output
 *           of its part of the page.  The synchronous host-pointer calls
 *           return BNZ_ETIMEOUT then; asynchronous callers read this counter;
 *           the serving engine fails the requests of such a step with
 *           BNZ_ETIMEOUT,
 *       [3] bnz_dual_dev: ties of the Niblack mask; 0 for the other calls.
 */
#ifndef BNZ_H
#define BNZ_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BNZ_API __attribute__((visibility("default")))
#else
#define BNZ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BNZ_OK = 0,
    BNZ_EINVAL = 1,   /* bad argument (message in bnz_last_error) */
    BNZ_ENOMEM = 2,   /* device allocation failed or budget exhausted */
    BNZ_ECUDA = 3,    /* a CUDA runtime/driver call failed */
    BNZ_ETIMEOUT = 4, /* a bounded device-side wait gave up */
    BNZ_ENODEV = 5    /* no usable CUDA device */
} bnz_status;

typedef enum { BNZ_SAUVOLA = 0, BNZ_NIBLACK = 1 } bnz_rule;

#define BNZ_MAX_W 255
/* Accepted threshold parameters: |k| <= BNZ_MAX_ABS_K and, for Sauvola,
 * R >= BNZ_MIN_R.  Within this range every output equals the fp64 decision;
 * outside it the calls return BNZ_EINVAL. */
#define BNZ_MAX_ABS_K 1.0e6
#define BNZ_MIN_R 1.0e-6
#define BNZ_STATS_FALLBACKS 0
#define BNZ_STATS_TIES 1
#define BNZ_STATS_TIMEOUTS 2
#define BNZ_STATS_TIES_NIBLACK 3 /* bnz_dual_dev: ties of the Niblack mask (slot 1: the Sauvola mask's) */

/* Optional tile shape for the fused kernel (autotuner hook).  Zero fields
 * mean "library default".  tile_w: output columns per strip, 128, 256 or 512.
 * tile_h: approximate rows of work per CTA (sets the grid size).
 * chunk: rows per TMA load (8).  edge_weight: cost of a row of the page's
 * first or last strip (whose windows are clipped at the page's sides) against
 * a row of an inner strip, in sixteenths (16: equal); the CTAs are dealt out
 * per strip in that proportion. */
typedef struct {
    int tile_w;
    int tile_h;
    int chunk;
    int edge_weight;
} bnz_tile;

/* ---- synchronous host-pointer API (Eq. 3 with Eq. 4 / Niblack) ---------- */

/* src: height rows of width*channels bytes, tightly packed, host memory.
 * dst: height*width bytes, {0,255}, host memory.  Blocks until done.
 * k: |k| <= BNZ_MAX_ABS_K; R >= BNZ_MIN_R (the dynamic range of the standard
 * deviation, Sec. 1 after Eq. 4).
 * Page-locked host buffers copy fastest.  Pages of a megapixel or more are
 * processed in up to 4 row bands whose uploads, kernels and downloads overlap
 * on the calling thread's library streams; the result is the same as in one
 * piece.  A page whose input and mask take 256 MiB or more streams through
 * bnz_binarize_window with a quarter of those bytes as the window (more,
 * smaller bands overlap the copies better), and one that would take more than
 * half of the free device memory with that half as the window.  Thread-safe: every calling thread has its own streams and buffers. */
BNZ_API int bnz_sauvola(const uint8_t *src, int height, int width, int channels, int W, double k, double R,
                uint8_t *dst);

/* Niblack rule t = m + k*s (k may be negative, e.g. -0.2). */
BNZ_API int bnz_niblack(const uint8_t *src, int height, int width, int channels, int W, double k, uint8_t *dst);

/* One page, several settings: binarizes the host page src (as bnz_sauvola)
 * once for every entry of runs, each with its own rule (BNZ_SAUVOLA or
 * BNZ_NIBLACK; R ignored for Niblack), W, k and host output dst (height*width
 * bytes, {0,255}).  The page is copied to the device once, in as many row
 * bands as bnz_host_bands gives for the largest W, of equal height (several
 * masks per band make the downloads dominate); every band's kernels run as soon as
 * the rows their windows reach are up, and each mask band comes back while
 * later bands upload and compute.  Each dst equals what bnz_sauvola /
 * bnz_niblack writes for that setting.  1 <= nruns <= 1024.  Blocks until
 * done; BNZ_ETIMEOUT if a device wait gave up.  Thread-safe as bnz_sauvola. */
typedef struct {
    int W, rule;
    double k, R;
    uint8_t *dst;
} bnz_run;
BNZ_API int bnz_binarize_runs(const uint8_t *src, int height, int width, int channels, const bnz_run *runs,
                              int nruns);

/* Out-of-core form of bnz_sauvola / bnz_niblack (rule BNZ_SAUVOLA or
 * BNZ_NIBLACK, R ignored for Niblack): a host page of any height streams
 * through a device window of at most window_bytes (input and mask slots; the
 * calling thread's buffers grow to that size and are kept for later calls).
 * The page is cut into bands of B output rows, B as large as 3 slots of
 * (B + W - 1) input rows and (B + W/2) mask rows (16-byte padded) allow; each
 * band is uploaded with its read-only halo (the W/2 rows above and W - 1 - W/2
 * below that its windows reach), binarized and downloaded on the calling
 * thread's three library streams, overlapping the other bands.  dst equals
 * what bnz_sauvola / bnz_niblack writes.  BNZ_EINVAL if window_bytes holds no
 * 3 slots of 8 rows; otherwise errors as bnz_sauvola.  Blocks until done. */
BNZ_API int bnz_binarize_window(const uint8_t *src, int height, int width, int channels, int W, int rule, double k,
                                double R, uint8_t *dst, size_t window_bytes);

/* The row bands bnz_sauvola and bnz_niblack use for a page (host logic only, no
 * device needed): returns the band count nb (>= 1) and, if starts is not NULL,
 * writes the nb + 1 boundaries starts[0] = 0 < ... < starts[nb] = height
 * (max_bands: entries available in starts, at least nb + 1).  Band i starts at
 * row height - (height >> i); the smallest band has at least max(128, 2W)
 * rows; pages under 2^20 pixels are one band.  -BNZ_EINVAL for bad arguments. */
BNZ_API int bnz_host_bands(int height, int width, int W, int *starts, int max_bands);

/* ---- asynchronous device-pointer API -------------------------------------
 * d_src: device pointer, 16-byte aligned, rows src_pitch bytes apart,
 *   src_pitch a multiple of 16 and >= width*channels (TMA requirement).
 *   The buffer spans height * src_pitch bytes: the kernels read rows in
 *   8-byte units, so up to 7 padding bytes after a row's last pixel may be
 *   read (never used, never written).
 * d_dst: device pointer, rows dst_pitch bytes apart (>= width, or
 *   >= (width+7)/8 when packed).
 * stream: a cudaStream_t (NULL = legacy default stream).
 * d_stats: nullable device pointer to 4 uint64 counters (see above).
 * Returns after enqueueing; argument errors are reported immediately. */
BNZ_API int bnz_sauvola_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels, int W,
                    double k, double R, uint8_t *d_dst, size_t dst_pitch, int packed, void *stream,
                    unsigned long long *d_stats);

BNZ_API int bnz_niblack_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels, int W,
                    double k, uint8_t *d_dst, size_t dst_pitch, int packed, void *stream,
                    unsigned long long *d_stats);

/* Both rules from one pass over the window sums (Sec. 1: Sauvola, Eq. 4, and
 * Niblack share m and s; Eq. 3 is then taken once per rule): the page is read
 * once and S1, S2 are formed once.  d_dst_sauvola and d_dst_niblack receive
 * exactly what bnz_sauvola_dev(k_sauvola, R) and bnz_niblack_dev(k_niblack)
 * would write (same layout: dst_pitch, packed).  The two masks must not
 * overlap (BNZ_EINVAL).  d_stats (nullable, 4 counters): [0] pixels re-decided
 * past the fp32 filter, both rules; [1] Sauvola ties; [2] timeouts;
 * [3] Niblack ties.  Other arguments and errors as bnz_sauvola_dev. */
BNZ_API int bnz_dual_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels, int W,
                 double k_sauvola, double R, double k_niblack, uint8_t *d_dst_sauvola,
                 uint8_t *d_dst_niblack, size_t dst_pitch, int packed, void *stream,
                 unsigned long long *d_stats);

/* Global binarization, Eq. 2 (g = 0 if f < T, else 255, one T for the page),
 * with Otsu's threshold (Sec. 1 cites it as the best global method; the paper
 * gives no formula, Otsu's published definition is used): over the 256-bin
 * histogram of f (Eq. 1 gray), T in [1, 255] maximises the between-class
 * variance of the levels [0, T-1] and [T, 255], evaluated as
 * q = (D*D) / (n0*n1) in fp64 with D = N*s0 - S*n0 exact; the smallest T
 * among equal q wins; T = 0 (all 255) for a page of one gray level.
 * d_src: as bnz_sauvola_dev (16-byte aligned, pitch a multiple of 16); at most
 * 2^28 pixels.  d_dst: byte or packed mask as bnz_sauvola_dev.  d_scratch:
 * caller-owned device memory of BNZ_OTSU_SCRATCH_BYTES, 16-byte aligned; the
 * call leaves the histogram (256 x uint64) at offset 0 and T (int32) at offset
 * 2048 (bytes 2052..2055 hold a counter the call resets; bytes 4096..20479 the
 * histogram kernel's 16 partial tables).  A memset and two
 * kernels on `stream`, no host synchronization; calls that share a scratch
 * buffer must not overlap on the device.  Errors: BNZ_EINVAL
 * for bad arguments, BNZ_ECUDA for a failed launch. */
#define BNZ_OTSU_SCRATCH_BYTES 20480
BNZ_API int bnz_otsu_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels,
                 uint8_t *d_dst, size_t dst_pitch, int packed, void *d_scratch, void *stream);

/* ---- reduced sets S' (Sec. 2, Eq. 5) --------------------------------------
 * Sec. 2 thresholds with Eq. 5, t' = m' (1 + k (s'/R' - 1)), where m' and s'
 * are the mean and population deviation of a reduced set S' of O(W) window
 * pixels laid out along a geometric structure (Fig. 1).  The paper's drawings
 * are not available; the structures below are this library's proposals.  With
 * window offsets (dy, dx) in [-W/2, W - 1 - W/2]^2 (the same window as the
 * exact calls), S' holds the offsets on
 *   BNZ_GS_CROSS               dy == 0 or dx == 0                (2W - 1)
 *   BNZ_GS_DIAGONALS           dy == dx or dy == -dx             (2W - 1, odd W)
 *   BNZ_GS_STAR                cross or diagonals                (4W - 3)
 *   BNZ_GS_FRAME               dy or dx on the window's edge     (4W - 4)
 *   BNZ_GS_FRAME_CROSS         frame or cross                    (6W - 9, W >= 5)
 *   BNZ_GS_FRAME_DIAGONALS     frame or diagonals                (6W - 9, W >= 5)
 * Samples outside the image are dropped and n' counts the others. */
#define BNZ_GS_CROSS 1
#define BNZ_GS_DIAGONALS 2
#define BNZ_GS_STAR 3
#define BNZ_GS_FRAME 4
#define BNZ_GS_FRAME_CROSS 5
#define BNZ_GS_FRAME_DIAGONALS 6

/* Reduced-set binarization: g = 0 if f < t', else 255 (Eq. 3 on t').  For
 * BNZ_SAUVOLA t' is Eq. 5 with R' = R; for BNZ_NIBLACK t' = m' + k s' (R
 * ignored).  Every output equals the fp64 evaluation of t' on the exact
 * integer sums of S' (same order and tie rule as the exact calls).
 * d_src: gray or RGB (channels 1 or 3), any alignment, src_pitch >= width *
 * channels.  d_dst: byte mask (0 / 255), dst_pitch >= width.  W in [3,
 * BNZ_MAX_W]; k and R within the limits of bnz_sauvola_dev.  d_stats
 * (nullable, 4 counters, accumulated): [0] pixels re-decided past the fp32
 * filter, [1] ties |f - t'| < 1e-9.  One kernel on `stream`, no host
 * synchronization.  Errors: BNZ_EINVAL for bad arguments or an unknown
 * structure, BNZ_ECUDA for a failed launch. */
BNZ_API int bnz_gs_binarize_dev(const void *d_src, size_t src_pitch, int height, int width, int channels, int W,
                                int gs, int rule, double k, double R, void *d_dst, size_t dst_pitch,
                                unsigned long long *d_stats, void *stream);

/* Confusion counts for the F-measure of Eq. 6, FM = 2 R P / (R + P) with
 * R = TP / (TP + FN) and P = TP / (TP + FP): a pixel is text in d_mask where
 * it equals mask_ink and text in d_ref where it equals ref_ink (bytes).
 * Adds TP, FP, FN to d_counts[0..2] (device, caller-zeroed; TN = height *
 * width - the three).  Byte masks of height x width, any alignment.  One
 * kernel on `stream`.  Errors: BNZ_EINVAL, BNZ_ECUDA. */
BNZ_API int bnz_confusion_dev(const void *d_mask, size_t mask_pitch, int mask_ink, const void *d_ref,
                              size_t ref_pitch, int ref_ink, int height, int width, unsigned long long *d_counts,
                              void *stream);

/* Generic form of the two calls above with an explicit rule and optional
 * tile shape (tile may be NULL).  R is ignored for BNZ_NIBLACK. */
BNZ_API int bnz_binarize_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels, int W,
                     int rule, double k, double R, uint8_t *d_dst, size_t dst_pitch, int packed,
                     const bnz_tile *tile, void *stream, unsigned long long *d_stats);

/* ---- batches: many uneven pages in one persistent launch -------------------
 * Every page of a batch is binarized exactly as bnz_binarize_dev would do it
 * (same kernels, same bits), but all pages' work is split over one persistent
 * grid per channel count, so small pages do not each pay a launch and a
 * partly idle GPU.  The device pointers are bound at creation: running the
 * batch again reads the same d_src buffers and writes the same d_dst
 * buffers (refill the inputs between runs).  With use_graph != 0 the
 * launches are captured once into a CUDA graph and bnz_batch_run replays it. */
typedef struct {
    const uint8_t *d_src; /* device, 16-byte aligned, src_pitch % 16 == 0, height*src_pitch bytes */
    size_t src_pitch;
    int height, width, channels; /* channels 1 or 3 */
    int W, rule, packed;         /* as bnz_binarize_dev */
    double k, R;
    uint8_t *d_dst;
    size_t dst_pitch;
    int tile_w; /* preferred strip width 128, 256 or 512 (e.g. from an autotuner); 0 or a width that
                   does not fit shared memory = the widest that fits */
    int reserved;
} bnz_page;

typedef struct bnz_batch bnz_batch; /* opaque */

/* Validate and plan n pages, upload their descriptors (device memory owned
 * by the batch), optionally capture the launches in a CUDA graph.  d_stats:
 * nullable device counters as for bnz_binarize_dev.  On error *out is NULL. */
BNZ_API int bnz_batch_create(const bnz_page *pages, int n, int use_graph, unsigned long long *d_stats,
                             bnz_batch **out);
/* Bytes of device memory bnz_batch_create_async needs for n page descriptors. */
BNZ_API size_t bnz_batch_desc_bytes(int n);
/* Like bnz_batch_create without a graph and without allocating: the page
 * descriptors go to caller-provided device memory d_desc (128-byte aligned,
 * bnz_batch_desc_bytes(n) bytes), written by small kernels on `stream` that
 * carry them as launch parameters (the call never waits for the stream); run
 * the batch on the same stream (or after it).  d_desc must outlive the
 * batch's runs; destroying the batch does not synchronize. */
BNZ_API int bnz_batch_create_async(const bnz_page *pages, int n, void *d_desc, size_t desc_bytes, void *stream,
                                   unsigned long long *d_stats, bnz_batch **out);
/* Enqueue the whole batch on `stream` (one graph launch, or one kernel per channel count). */
BNZ_API int bnz_batch_run(bnz_batch *b, void *stream);
/* Pages, kernel launches per run, grid size, shared memory per CTA and total strip-rows. */
BNZ_API int bnz_batch_info(const bnz_batch *b, int *pages, int *launches, int *grid, size_t *smem,
                           long long *strip_rows);
/* Free the batch (after its last run has completed). */
BNZ_API int bnz_batch_destroy(bnz_batch *b);

/* ---- device-memory pool for the serving loop -----------------------------
 * Host-side bookkeeping (first fit, neighbours coalesced on free) over one
 * device range the caller allocated once, e.g. the serving loop's whole
 * memory budget.  Requests of mixed page sizes get their input and output
 * buffers from it without cudaMalloc/cudaFree, which would stall the device.
 * The pool never reads or writes the range, so it also works over a range no
 * device backs (tests).  Thread-safe.  No counterpart in the paper. */
typedef struct bnz_pool bnz_pool; /* opaque */

/* Manage [base, base+bytes); base must be 256-byte aligned.  The range stays
 * owned by the caller and must outlive the pool. */
BNZ_API int bnz_pool_create(void *base, size_t bytes, bnz_pool **out);
/* 256-byte-aligned block of at least `bytes` bytes.  BNZ_ENOMEM (not an
 * error to report: the caller waits for frees) when no free range fits. */
BNZ_API int bnz_pool_alloc(bnz_pool *p, size_t bytes, void **out);
/* Return a block.  The caller guarantees that no queued device work still
 * uses it (the pool cannot see streams).  BNZ_EINVAL for a pointer that is
 * not a live block of this pool. */
BNZ_API int bnz_pool_free(bnz_pool *p, void *ptr);
/* Bytes in live blocks, their high-water mark, the largest free range, and
 * the number of live blocks; any pointer may be NULL. */
BNZ_API int bnz_pool_stats(const bnz_pool *p, size_t *used, size_t *high_water, size_t *largest_free, int *live);
/* Fault injection: the next n calls of bnz_pool_alloc fail with BNZ_ENOMEM
 * (n=0 clears it).  Host-side only; nothing on the device is affected. */
BNZ_API int bnz_pool_fail_next(bnz_pool *p, int n);
/* Free the bookkeeping (live blocks are forgotten, the range is not freed). */
BNZ_API int bnz_pool_destroy(bnz_pool *p);

/* ---- native serving engine ------------------------------------------------
 * Requests of mixed page sizes and windows, submitted at any time from any
 * thread, are binarized by continuous batching: a scheduler thread admits
 * them in arrival order while their device buffers fit a budget reserved once
 * at creation (requests wait, none is dropped), copies host inputs up on a
 * copy stream, launches one batched kernel per step over admitted pages whose
 * input has arrived and that share a kernel instance (channels, rule, W mod 8;
 * the oldest ready page picks it; steps alternate over `compute_streams`),
 * copies the masks into the callers' host buffers on a second copy stream and
 * reports completions through bnz_server_poll.  No counterpart in the paper. */
typedef struct bnz_server bnz_server; /* opaque */

typedef struct {
    size_t budget_bytes;  /* device memory for request buffers, reserved at creation (>= 1 MiB) */
    int max_batch;        /* pages per launch step, 1..4096 */
    int compute_streams;  /* 1..4; 1 is fastest for mixed traffic (kernels of different instances running
                             side by side share the SMs' instruction caches) */
    int batched;          /* 1: one batched launch per step; 0: one plain launch per page */
    int reserved;         /* 0.  Test hook, host side only: n > 0 makes every n-th launch step report a
                             device timeout, as if a bounded wait had given up, so that callers can test
                             their handling of BNZ_ETIMEOUT */
} bnz_server_config;

typedef struct {
    const uint8_t *src;   /* host (pinned memory overlaps; pageable works) or device pointer */
    size_t src_pitch;     /* bytes between rows of src */
    int src_on_device;    /* 1: src is device memory, complete when submitted, 16-byte aligned,
                             pitch % 16 == 0, height*src_pitch bytes; it must stay valid until completion */
    int height, width, channels, W, rule;
    double k, R;
    int packed;
    uint8_t *dst;         /* host memory (pinned for overlap) receiving the mask, valid until completion */
    size_t dst_pitch;
    unsigned long long tag; /* returned by bnz_server_poll */
} bnz_request;

/* Reserve the budget, create the streams and start the scheduler thread.
 * BNZ_ENODEV without a device, BNZ_ENOMEM if the budget cannot be reserved. */
BNZ_API int bnz_server_create(const bnz_server_config *cfg, bnz_server **out);
/* Queue a request (the descriptor is copied; the buffers are not).  Argument
 * errors return BNZ_EINVAL, a request larger than the whole budget
 * BNZ_ENOMEM; neither is queued. */
BNZ_API int bnz_server_submit(bnz_server *s, const bnz_request *req);
/* Up to `max` completed requests: their tags, statuses (BNZ_OK or the error)
 * and latencies from submission to the mask in host memory, in seconds
 * (status and latency_s nullable).  Waits up to timeout_ms for the first one.
 * Returns the number written (0 on timeout). */
BNZ_API int bnz_server_poll(bnz_server *s, unsigned long long *tags, int *status, double *latency_s, int max,
                            int timeout_ms);
/* Requests submitted and not yet polled, completed, launch steps, admissions
 * deferred for memory, and the high-water mark of device bytes in use (any
 * pointer may be NULL). */
BNZ_API int bnz_server_stats(bnz_server *s, long long *outstanding, long long *completed, long long *steps,
                             long long *alloc_waits, size_t *high_water);
/* Copy the scheduler's last failure message (empty if none) into buf. */
BNZ_API int bnz_server_error(bnz_server *s, char *buf, size_t n);
/* Finish every submitted request, stop the thread, free the budget.  Requests
 * not yet polled are discarded. */
BNZ_API int bnz_server_destroy(bnz_server *s);

/* ---- integral-image comparison variant ------------------------------------
 * The O(N^2) method with summed-area tables that Sec. 1 cites (Shafait et
 * al.) and Sec. 3.3 charges 12 S_z bytes of memory: two (h+1) x (w+1) int64
 * tables of f and f^2 (int64 for both: sums of f over a 16384^2 page exceed
 * 2^32), then four corner lookups per pixel and the same Eq. 3 decision as
 * the fused path, so the outputs are identical.  The caller provides the
 * scratch (device memory, 32-byte aligned, at least
 * bnz_integral_scratch_bytes(height, width) bytes); height <= 65535. */

/* Scratch bytes the integral-image variant needs (0 for bad sizes). */
BNZ_API size_t bnz_integral_scratch_bytes(int height, int width);

/* Binarize through the integral images; arguments as bnz_binarize_dev plus
 * the scratch.  Asynchronous on `stream`. */
BNZ_API int bnz_binarize_integral_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels,
                                      int W, int rule, double k, double R, uint8_t *d_dst, size_t dst_pitch,
                                      int packed, void *d_scratch, size_t scratch_bytes, void *stream,
                                      unsigned long long *d_stats);

/* Only build the tables: I1 (sum of f over rows < y, columns < x) at
 * d_scratch and I2 (same for f^2) right after it, each (height+1) rows of
 * *ld_elems int64 values (row 0 and column 0 are zero). */
BNZ_API int bnz_integral_images_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels,
                                    void *d_scratch, size_t scratch_bytes, long long *ld_elems, void *stream);

/* Allocation-free form of bnz_binarize_integral_dev (the paper has no
 * counterpart; this serves callers that cannot allocate device memory, such
 * as code running inside a framework that owns every device allocation, or a
 * fixed-budget pipeline that must not reach the allocator while it runs).
 * The scratch is a library-owned device array of BNZ_INTEGRAL_STATIC_MAX_BYTES
 * that every GPU loading the library keeps until the process exits; pages
 * whose scratch (bnz_integral_scratch_bytes) exceeds it are rejected with
 * BNZ_EINVAL.  The first call on a device looks up the array's device address
 * (once per device); make that first call before any stream capture.  Every
 * call on a device uses the same array: calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialized by the caller.
 * The call itself allocates nothing.  The looked-up address is kept for the
 * life of the process: resetting a device (cudaDeviceReset) while the library
 * is loaded is not supported by this call.  Arguments as bnz_binarize_dev. */
#define BNZ_INTEGRAL_STATIC_MAX_BYTES (32u << 20)
BNZ_API int bnz_binarize_integral_static_dev(const uint8_t *d_src, size_t src_pitch, int height, int width,
                                             int channels, int W, int rule, double k, double R, uint8_t *d_dst,
                                             size_t dst_pitch, int packed, void *stream,
                                             unsigned long long *d_stats);

/* ---- library state ------------------------------------------------------ */

/* Message for the calling thread's most recent failure ("" if none). */
BNZ_API const char *bnz_last_error(void);

/* Stream-ordered 2-D copy of `height` rows of `width_bytes` bytes between
 * any two of host (pinned or pageable) and device memory (unified
 * addressing decides the direction).  A copy-engine transfer, no kernel; the
 * serving loop uses it to move pages between a caller's dense host buffers
 * and the 16-byte-pitched device buffers the kernels read.  It has no
 * counterpart in the paper.  Returns BNZ_EINVAL for a null pointer with a
 * non-empty extent or a pitch below width_bytes. */
BNZ_API int bnz_copy2d_async(void *dst, size_t dst_pitch, const void *src, size_t src_pitch, size_t width_bytes,
                             size_t height, void *stream);

/* Library ABI version (major*10000 + minor*100 + patch). */
BNZ_API int bnz_version(void);

/* Shared memory bytes and grid size the fused kernel would use for this
 * problem (no launch; for planning and autotuning).  Returns BNZ_OK. */
BNZ_API int bnz_fused_plan(int height, int width, int channels, int W, const bnz_tile *tile, size_t *smem_bytes,
                   int *grid_ctas, int *tile_w, int *tile_h);

/* The fused kernel's decision margins for (rule, k, R), computed on the host
 * as for a launch: *E, the fp32 filter's margin for any window; *E_int, the
 * tighter one of Niblack windows inside the page (E for Sauvola); *Tdf, the
 * double-float stage's cut.  The paper has no counterpart: this exposes the
 * fp32 error analysis to tests that check it against exact arithmetic.  Host
 * only (no device needed).  Returns BNZ_EINVAL for a null pointer, an unknown
 * rule, or k, R outside the accepted range. */
BNZ_API int bnz_decision_margins(int rule, double k, double R, float *E, float *E_int, float *Tdf);

/* Device self-test of the hardware square-root approximation the fused
 * kernel's fp32 margin assumes (relative error <= 2^-21): writes to
 * *max_rel_err an upper bound on |sqrt.approx(x) - sqrt(x)| / sqrt(x) over
 * every float x in [lo, hi).  Synchronous; for tests and diagnostics. */
BNZ_API int bnz_selftest_sqrt_approx(float lo, float hi, double *max_rel_err);

/* Same for the hardware reciprocal approximation over the integers
 * n_lo <= n < n_hi (the clipped window counts; assumed <= 2^-22). */
BNZ_API int bnz_selftest_rcp_approx(unsigned int n_lo, unsigned int n_hi, double *max_rel_err);

/* Device self-test of the fused kernel's Eq. 1 conversion (the producers'
 * code, four pixels per step): d_rgb holds npix interleaved r,g,b pixels,
 * d_gray receives npix gray bytes f = (299 r + 587 g + 114 b + 500) / 1000.
 * Asynchronous on `stream`; for tests and diagnostics. */
BNZ_API int bnz_selftest_gray(const uint8_t *d_rgb, size_t npix, uint8_t *d_gray, void *stream);

/* Self-test of the fused kernel's own abort path: one launch (byte mask, no
 * tile) in which every wait of the producers and of the TMA issuer gives up
 * as soon as its barrier phase is not already complete, so CTAs give up
 * while their first copies are still in flight; the issuer's final wait for
 * its copies in flight keeps the normal limit, so no CTA exits with a copy
 * outstanding.  d_stats (required, 4 counters zeroed by the caller) receives
 * the count of CTAs that gave up in [2].  Synchronizes `stream`; returns
 * BNZ_ETIMEOUT when any CTA gave up (the output is then incomplete), else
 * BNZ_OK.  Other arguments as bnz_binarize_dev.  For tests and diagnostics. */
BNZ_API int bnz_selftest_fused_timeout(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels,
                                       int W, int rule, double k, double R, uint8_t *d_dst, size_t dst_pitch,
                                       void *stream, unsigned long long *d_stats);

/* Device self-test of the bounded wait every kernel uses on its mbarriers:
 * one thread waits for a barrier phase with a limit of `limit_cycles` SM
 * cycles; with arrive = 0 nothing ever completes the phase, so the wait must
 * give up (*timed_out = 1) after about the limit and return, leaving the
 * context usable; with arrive = 1 the phase is complete and *timed_out = 0.
 * *waited_cycles (nullable) receives the cycles spent.  Synchronous. */
BNZ_API int bnz_selftest_wait_timeout(long long limit_cycles, int arrive, int *timed_out,
                                      long long *waited_cycles);

#ifdef __cplusplus
}
#endif
#endif /* BNZ_H */
