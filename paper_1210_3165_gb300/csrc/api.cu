// api.cu -- the C ABI declared in include/bnz.h: argument checks, error
// messages, TMA descriptor encoding, device bookkeeping and the synchronous
// host-pointer calls.  All pixel work happens in the CUDA kernels.
#include <algorithm>
#include <vector>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"

namespace bnz {

static thread_local std::string t_err;

int fail(int rc, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return rc;
}

int cuda_fail(cudaError_t e, const char *what)
{
    const int rc = (e == cudaErrorMemoryAllocation) ? BNZ_ENOMEM
                   : (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) ? BNZ_ENODEV
                                                                                   : BNZ_ECUDA;
    return fail(rc, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static std::mutex g_mu;
static EncodeTiledFn g_encode = nullptr;
static const int kMaxDev = 64;
static int g_sms[kMaxDev];
static unsigned int *g_err[kMaxDev];

int encode_span_map(CUtensorMap *map, const void *base, uint64_t row_bytes, uint64_t rows, uint64_t pitch,
                    uint32_t box_bytes, uint32_t box_rows)
{
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_encode) {
            void *fn = nullptr;
            cudaDriverEntryPointQueryResult q;
            cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                             cudaEnableDefault, &q);
            if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
                return fail(BNZ_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
            g_encode = reinterpret_cast<EncodeTiledFn>(fn);
        }
    }
    if ((box_bytes & 15u) || box_bytes / 8 > 256 || box_rows < 1 || box_rows > 256)
        return fail(BNZ_EINVAL, "span box %ux%u out of range", box_bytes, box_rows);
    cuuint64_t dims[2] = {(cuuint64_t)((row_bytes + 7) / 8), (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch};
    cuuint32_t box[2] = {box_bytes / 8, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(BNZ_EINVAL, "cuTensorMapEncodeTiled failed (%d): base=%p row=%llu rows=%llu pitch=%llu",
                    (int)r, base, (unsigned long long)row_bytes, (unsigned long long)rows,
                    (unsigned long long)pitch);
    return BNZ_OK;
}

static int current_device(int *dev)
{
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n < 1) {
        cudaGetLastError();
        return fail(BNZ_ENODEV, "no CUDA device available (%s); this library has no CPU path",
                    e == cudaSuccess ? "device count 0" : cudaGetErrorName(e));
    }
    e = cudaGetDevice(dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (*dev < 0 || *dev >= kMaxDev)
        return fail(BNZ_ENODEV, "device ordinal %d out of range", *dev);
    return BNZ_OK;
}

int device_sm_count(int *sms)
{
    int dev = 0;
    int rc = current_device(&dev);
    if (rc != BNZ_OK)
        return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_sms[dev]) {
        int v = 0;
        cudaError_t e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetAttribute(SM count)");
        g_sms[dev] = v;
    }
    *sms = g_sms[dev];
    return BNZ_OK;
}

int device_err_flag(unsigned int **flag)
{
    int dev = 0;
    int rc = current_device(&dev);
    if (rc != BNZ_OK)
        return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_err[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, 256);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(error word)");
        e = cudaMemset(p, 0, 256);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaMemset(error word)");
        g_err[dev] = static_cast<unsigned int *>(p);
    }
    *flag = g_err[dev];
    return BNZ_OK;
}

int check_common(const void *src, size_t src_pitch, int height, int width, int channels, int W, int rule,
                 double k, double R, const void *dst, size_t dst_pitch, int packed)
{
    if (!src || !dst)
        return fail(BNZ_EINVAL, "null image pointer");
    if (height < 1 || width < 1)
        return fail(BNZ_EINVAL, "height and width must be >= 1 (got %d x %d)", height, width);
    if (channels != 1 && channels != 3)
        return fail(BNZ_EINVAL, "channels must be 1 or 3 (got %d)", channels);
    if (W < 1 || W > BNZ_MAX_W)
        return fail(BNZ_EINVAL, "window size W must be in [1, %d] (got %d)", BNZ_MAX_W, W);
    if (rule != BNZ_SAUVOLA && rule != BNZ_NIBLACK)
        return fail(BNZ_EINVAL, "unknown rule %d", rule);
    // the range within which every fp32 and double-float constant of the
    // decision, and every intermediate of the filters, stays finite (so the
    // proven error bounds apply and every output equals the fp64 decision)
    if (!(std::fabs(k) <= BNZ_MAX_ABS_K))
        return fail(BNZ_EINVAL, "k must be finite with |k| <= %g (got %g)", BNZ_MAX_ABS_K, k);
    if (rule == BNZ_SAUVOLA && !(R >= BNZ_MIN_R && std::isfinite(R)))
        return fail(BNZ_EINVAL, "R must be finite and >= %g for Sauvola (got %g)", BNZ_MIN_R, R);
    if (src_pitch < (size_t)width * channels)
        return fail(BNZ_EINVAL, "src_pitch %zu < width*channels %zu", src_pitch, (size_t)width * channels);
    const size_t row_out = packed ? ((size_t)width + 7) / 8 : (size_t)width;
    if (dst_pitch < row_out)
        return fail(BNZ_EINVAL, "dst_pitch %zu < %zu bytes per output row", dst_pitch, row_out);
    if ((size_t)width * channels > ((size_t)1 << 31) || (size_t)height > ((size_t)1 << 31))
        return fail(BNZ_EINVAL, "image too large");
    return BNZ_OK;
}

static int binarize_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels, int W,
                        int rule, double k, double R, uint8_t *d_dst, size_t dst_pitch, int packed,
                        const bnz_tile *tile, void *stream, unsigned long long *d_stats, int y_lo = 0,
                        int y_hi = -1)
{
    int rc = check_common(d_src, src_pitch, height, width, channels, W, rule, k, R, d_dst, dst_pitch, packed);
    if (rc != BNZ_OK)
        return rc;
    if ((reinterpret_cast<uintptr_t>(d_src) & 15u) || (src_pitch & 15u))
        return fail(BNZ_EINVAL, "d_src must be 16-byte aligned with src_pitch a multiple of 16 (TMA)");
    if (rule == BNZ_NIBLACK)
        R = 1.0;
    unsigned int *err = nullptr;
    rc = device_err_flag(&err);
    if (rc != BNZ_OK)
        return rc;
    return launch_fused(d_src, src_pitch, height, width, channels, W, rule, k, R, d_dst, dst_pitch, packed ? 1 : 0,
                        tile, static_cast<cudaStream_t>(stream), d_stats, err, y_lo, y_hi);
}

// Synchronous host-pointer path: stream-ordered device buffers, copies in and
// out overlapped with the launches band by band, then a check of the
// statistics' timeout count.
// Per-thread, per-device resources of the synchronous host API, made once: a
// stream, grow-only device buffers for the page and its mask, and statistics
// counters with a pinned host copy.  Creating a stream, allocating and freeing
// tens of MB (the default pool returns freed memory at each synchronize), or a
// blocking read of the error word, per call would cost more than the kernel.
// A page is cut into up to kMaxBands row bands, so that the upload of band
// i + 1, the kernel on band i and the download of band i - 1 overlap (the
// host link, not the kernel, bounds this path).
constexpr int kMaxBands = 4;

struct HostCallState {
    struct PerDevice {
        cudaStream_t stream = nullptr, up = nullptr, down = nullptr;
        cudaEvent_t ev_up[kMaxBands] = {}, ev_k[kMaxBands] = {}, ev_dn[kMaxBands] = {};
        unsigned long long *stats = nullptr, *h_stats = nullptr;
        void *src = nullptr, *dst = nullptr;
        size_t src_cap = 0, dst_cap = 0;
        std::vector<cudaEvent_t> ev_run; // bnz_binarize_runs: one per (band, setting) kernel, grow-only
    };
    PerDevice dev[64];
    ~HostCallState()
    {
        for (int d = 0; d < 64; ++d) {
            PerDevice &v = dev[d];
            if (!v.stream && !v.stats && !v.src && !v.dst && !v.h_stats)
                continue;
            cudaSetDevice(d);
            for (int i = 0; i < kMaxBands; ++i) {
                if (v.ev_up[i])
                    cudaEventDestroy(v.ev_up[i]);
                if (v.ev_k[i])
                    cudaEventDestroy(v.ev_k[i]);
                if (v.ev_dn[i])
                    cudaEventDestroy(v.ev_dn[i]);
            }
            for (cudaEvent_t ev : v.ev_run)
                cudaEventDestroy(ev);
            if (v.up)
                cudaStreamDestroy(v.up);
            if (v.down)
                cudaStreamDestroy(v.down);
            if (v.stream)
                cudaStreamDestroy(v.stream);
            cudaFree(v.stats);
            cudaFree(v.src);
            cudaFree(v.dst);
            cudaFreeHost(v.h_stats);
        }
    }
};

static int grow(void **buf, size_t *cap, size_t need, const char *what)
{
    if (*cap >= need)
        return BNZ_OK;
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    const cudaError_t e = cudaMalloc(buf, need);
    if (e != cudaSuccess) {
        *buf = nullptr;
        return cuda_fail(e, what);
    }
    *cap = need;
    return BNZ_OK;
}

static HostCallState &host_calls()
{
    static thread_local HostCallState st;
    return st;
}

static size_t host_call_held(int d)
{
    if (d < 0 || d >= 64)
        return 0;
    const HostCallState::PerDevice &v = host_calls().dev[d];
    return v.src_cap + v.dst_cap;
}

static int host_call_state(int d, size_t src_bytes, size_t dst_bytes, HostCallState::PerDevice **out)
{
    HostCallState &st = host_calls();
    if (d < 0 || d >= 64)
        return fail(BNZ_ENODEV, "device ordinal %d out of range", d);
    HostCallState::PerDevice &v = st.dev[d];
    cudaError_t e = cudaSuccess;
    for (cudaStream_t *ps : {&v.stream, &v.up, &v.down})
        if (!*ps && (e = cudaStreamCreateWithFlags(ps, cudaStreamNonBlocking)) != cudaSuccess) {
            *ps = nullptr;
            return cuda_fail(e, "cudaStreamCreate");
        }
    for (int i = 0; i < kMaxBands; ++i)
        for (cudaEvent_t *pe : {&v.ev_up[i], &v.ev_k[i], &v.ev_dn[i]})
            if (!*pe && (e = cudaEventCreateWithFlags(pe, cudaEventDisableTiming)) != cudaSuccess) {
                *pe = nullptr;
                return cuda_fail(e, "cudaEventCreate");
            }
    if (!v.stats && (e = cudaMalloc(&v.stats, 4 * sizeof(unsigned long long))) != cudaSuccess) {
        v.stats = nullptr;
        return cuda_fail(e, "cudaMalloc(statistics)");
    }
    if (!v.h_stats && (e = cudaMallocHost(&v.h_stats, 4 * sizeof(unsigned long long))) != cudaSuccess) {
        v.h_stats = nullptr;
        return cuda_fail(e, "cudaMallocHost(statistics)");
    }
    int rc = grow(&v.src, &v.src_cap, src_bytes, "cudaMalloc(page)");
    if (rc == BNZ_OK)
        rc = grow(&v.dst, &v.dst_cap, dst_bytes, "cudaMalloc(mask)");
    if (rc != BNZ_OK)
        return rc;
    *out = &v;
    return BNZ_OK;
}

// Device bytes the calling thread's host-call buffers hold on device d.
static size_t host_call_held(int d);

// Both rules from one pass over the window sums (dual.cu).
int launch_dual(const uint8_t *d_src, size_t src_pitch, int h, int w, int ch, int W, double ks, double R, double kn,
                uint8_t *d_dst_s, uint8_t *d_dst_n, size_t dst_pitch, int packed, const bnz_tile *tile,
                cudaStream_t stream, unsigned long long *d_stats, unsigned int *d_err);

// Eq. 2 with Otsu's threshold (otsu.cu).
int launch_otsu(const uint8_t *d_src, size_t src_pitch, int h, int w, int ch, uint8_t *d_dst, size_t dst_pitch,
                int packed, void *d_scratch, cudaStream_t stream);

// Row bands for a page of h rows, halving towards the end: band i starts at
// row h - (h >> i) and the last one holds the final h >> (nb - 1) rows.  The
// early, large bands' kernels and downloads run under the rest of the upload;
// after the upload only the small last band's kernel and download remain.  The
// smallest band has at least max(128, 2W) rows (each band's CTAs first sum
// the W rows of their window), and pages under a megapixel stay in one piece
// (a launch and two events per band cost more than such a page's copies).
static int host_bands(int height, int width, int W)
{
    if ((long long)height * width < (1ll << 20))
        return 1;
    const int min_rows = std::max(128, 2 * W);
    int nb = 1;
    while (nb < kMaxBands && (height >> nb) >= min_rows)
        ++nb;
    return nb;
}

static int band_start(int height, int i) { return height - (height >> i); }

// Copies rows [y0, y1) of a page between host (tightly packed rows of `row`
// bytes) and device (rows `pitch` apart).
static cudaError_t copy_rows(void *dst_base, size_t dst_pitch, const void *src_base, size_t src_pitch, size_t row,
                             int y0, int y1, cudaMemcpyKind kind, cudaStream_t s)
{
    char *d = static_cast<char *>(dst_base) + (size_t)y0 * dst_pitch;
    const char *sp = static_cast<const char *>(src_base) + (size_t)y0 * src_pitch;
    const size_t n = (size_t)(y1 - y0);
    // rows already 16-byte multiples: one contiguous copy (the copy engines run
    // large linear copies faster than row-by-row 2-D ones)
    if (dst_pitch == row && src_pitch == row)
        return cudaMemcpyAsync(d, sp, row * n, kind, s);
    return cudaMemcpy2DAsync(d, dst_pitch, sp, src_pitch, row, n, kind, s);
}

// ---- pages larger than the device: a bounded window of row bands ----------
// The page streams through kSlots band slots in device memory.  Band i holds
// output rows [y0, y1) = [i B, i B + B) and its read-only halo: input rows
// [y0 - r_lo, y1 + r_hi) within the page, the rows its windows reach.  It is
// binarized as a sub-page of those rows with outputs [y0, y1) only: a window
// of an output row never reaches the sub-page's cut edges (it clips only
// where the page itself ends), so every mask row is the whole page's.  Three
// streams: the upload of band i waits until the kernel of band i - kSlots has
// read its slot; the kernel waits for its upload and for the download of
// band i - kSlots (its output slot); the download waits for the kernel.  The
// halo rows are uploaded again with each band ((W - 1) / B more input bytes).
constexpr int kSlots = 3;
constexpr size_t kWindowedBytes = (size_t)256 << 20; // page + mask bytes from which the host calls use the slots

static size_t window_slot_bytes(int B, int W, size_t sp, size_t dp)
{
    return (size_t)(B + W - 1) * sp + (size_t)(B + W / 2) * dp;
}

static int window_band_rows(int height, int W, size_t sp, size_t dp, size_t window_bytes, int *B_out)
{
    const size_t per = window_bytes / kSlots;
    const size_t fixed = (size_t)(W - 1) * sp + (size_t)(W / 2) * dp;
    const size_t B = per > fixed ? (per - fixed) / (sp + dp) : 0;
    if (B < 8)
        return fail(BNZ_EINVAL, "window_bytes %zu too small: %d slots of at least 8 rows and a %d-row halo need %zu",
                    window_bytes, kSlots, W - 1, (size_t)kSlots * window_slot_bytes(8, W, sp, dp));
    *B_out = (int)std::min<size_t>(B, (size_t)height);
    return BNZ_OK;
}

static int binarize_window_host(const uint8_t *src, int height, int width, int channels, int W, int rule, double k,
                                double R, uint8_t *dst, size_t window_bytes)
{
    int rc = check_common(src, (size_t)width * channels, height, width, channels, W, rule, k, R, dst,
                          (size_t)width, 0);
    if (rc != BNZ_OK)
        return rc;
    const size_t row_in = (size_t)width * channels;
    const size_t sp = (row_in + 15) & ~size_t(15);
    const size_t dp = ((size_t)width + 15) & ~size_t(15);
    int B = 0;
    if ((rc = window_band_rows(height, W, sp, dp, window_bytes, &B)) != BNZ_OK)
        return rc;
    int dev = 0, sms = 0;
    if ((rc = current_device(&dev)) != BNZ_OK || (rc = device_sm_count(&sms)) != BNZ_OK)
        return rc;
    const int r_lo = W / 2, r_hi = W - 1 - W / 2;
    const size_t in_slot = (size_t)(B + W - 1) * sp, out_slot = (size_t)(B + r_lo) * dp;
    HostCallState::PerDevice *v = nullptr;
    if ((rc = host_call_state(dev, kSlots * in_slot, kSlots * out_slot, &v)) != BNZ_OK)
        return rc;
    FusedPlan shape;
    if ((rc = plan_shape(std::min(height, B + W - 1), width, channels, W, 0, &shape)) != BNZ_OK)
        return rc;
    cudaStream_t s = v->stream;
    const int nb = (height + B - 1) / B;
    cudaError_t e;
    do {
        if ((e = cudaMemsetAsync(v->stats, 0, 4 * sizeof(unsigned long long), s)) != cudaSuccess) {
            rc = cuda_fail(e, "clear statistics");
            break;
        }
        for (int i = 0; i < nb && rc == BNZ_OK; ++i) {
            const int j = i % kSlots;
            const int y0 = i * B, y1 = std::min(height, y0 + B);
            const int in0 = std::max(0, y0 - r_lo), in1 = std::min(height, y1 + r_hi);
            uint8_t *sin = static_cast<uint8_t *>(v->src) + (size_t)j * in_slot;
            uint8_t *sout = static_cast<uint8_t *>(v->dst) + (size_t)j * out_slot;
            if (i >= kSlots && (e = cudaStreamWaitEvent(v->up, v->ev_k[j], 0)) != cudaSuccess) {
                rc = cuda_fail(e, "order slot reuse");
                break;
            }
            if ((e = copy_rows(sin, sp, src + (size_t)in0 * row_in, row_in, row_in, 0, in1 - in0,
                               cudaMemcpyHostToDevice, v->up)) != cudaSuccess) {
                rc = cuda_fail(e, "copy band to device");
                break;
            }
            if ((e = cudaEventRecord(v->ev_up[j], v->up)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(s, v->ev_up[j], 0)) != cudaSuccess ||
                (i >= kSlots && (e = cudaStreamWaitEvent(s, v->ev_dn[j], 0)) != cudaSuccess)) {
                rc = cuda_fail(e, "order band kernel");
                break;
            }
            bnz_tile tile = {0, 0, 0, 0};
            tile.tile_h = (int)std::max<long long>(8, ((long long)shape.tiles_x * (y1 - y0) + sms - 1) / sms);
            rc = binarize_dev(sin, sp, in1 - in0, width, channels, W, rule, k, R, sout, dp, 0, &tile, s, v->stats,
                              y0 - in0, y1 - in0);
            if (rc != BNZ_OK)
                break;
            if ((e = cudaEventRecord(v->ev_k[j], s)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(v->down, v->ev_k[j], 0)) != cudaSuccess) {
                rc = cuda_fail(e, "order band download");
                break;
            }
            if ((e = cudaMemcpy2DAsync(dst + (size_t)y0 * width, (size_t)width, sout + (size_t)(y0 - in0) * dp, dp,
                                       (size_t)width, (size_t)(y1 - y0), cudaMemcpyDeviceToHost, v->down)) !=
                    cudaSuccess ||
                (e = cudaEventRecord(v->ev_dn[j], v->down)) != cudaSuccess) {
                rc = cuda_fail(e, "copy band result to host");
                break;
            }
        }
        if (rc != BNZ_OK)
            break;
        if ((e = cudaStreamWaitEvent(v->down, v->ev_k[(nb - 1) % kSlots], 0)) != cudaSuccess ||
            (e = cudaMemcpyAsync(v->h_stats, v->stats, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 v->down)) != cudaSuccess) {
            rc = cuda_fail(e, "read statistics");
            break;
        }
    } while (0);
    for (cudaStream_t q : {v->up, s, v->down}) {
        e = cudaStreamSynchronize(q);
        if (rc == BNZ_OK && e != cudaSuccess)
            rc = cuda_fail(e, "cudaStreamSynchronize");
    }
    if (rc == BNZ_OK && v->h_stats[BNZ_STATS_TIMEOUTS] != 0)
        rc = fail(BNZ_ETIMEOUT, "a device-side wait timed out; output incomplete");
    return rc;
}

static int binarize_host(const uint8_t *src, int height, int width, int channels, int W, int rule, double k,
                         double R, uint8_t *dst)
{
    int rc = check_common(src, (size_t)width * channels, height, width, channels, W, rule, k, R, dst,
                          (size_t)width, 0);
    if (rc != BNZ_OK)
        return rc;
    int dev = 0;
    rc = current_device(&dev);
    if (rc != BNZ_OK)
        return rc;
    int sms = 0;
    rc = device_sm_count(&sms);
    if (rc != BNZ_OK)
        return rc;
    const size_t row_in = (size_t)width * channels;
    const size_t sp = (row_in + 15) & ~size_t(15);
    const size_t dp = ((size_t)width + 15) & ~size_t(15);
    // a page (and its mask) that would take more than half of the free device
    // memory streams through a window of that half instead
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
        const size_t avail = (free_b + host_call_held(dev)) / 2;
        if ((sp + dp) * (size_t)height > avail)
            return binarize_window_host(src, height, width, channels, W, rule, k, R, dst, avail);
    }
    // a large page also goes through the band slots (a window of a quarter of
    // its bytes: bands of ~1/12 of the page): the many bands overlap upload,
    // kernels and download better than four halving bands (16384^2 gray,
    // W = 101: 1.93 against 2.52 ms)
    if ((sp + dp) * (size_t)height >= kWindowedBytes)
        return binarize_window_host(src, height, width, channels, W, rule, k, R, dst, (sp + dp) * (size_t)height / 4);
    HostCallState::PerDevice *v = nullptr;
    rc = host_call_state(dev, sp * height, dp * height, &v);
    if (rc != BNZ_OK)
        return rc;
    cudaStream_t s = v->stream;
    const int nb = host_bands(height, width, W);
    const int r_hi = W - 1 - W / 2;
    long long strips = 1;
    if (nb > 1) {
        FusedPlan shape;
        if ((rc = plan_shape(height, width, channels, W, 0, &shape)) != BNZ_OK)
            return rc;
        strips = shape.tiles_x;
    }
    cudaError_t e;
    do {
        if ((e = cudaMemsetAsync(v->stats, 0, 4 * sizeof(unsigned long long), s)) != cudaSuccess) {
            rc = cuda_fail(e, "clear statistics");
            break;
        }
        // the upload runs ahead on its own stream; band i's kernel waits for the
        // rows its windows reach, its download waits for the kernel
        int uploaded = 0;
        for (int i = 0; i < nb && rc == BNZ_OK; ++i) {
            const int y0 = band_start(height, i), y1 = i + 1 < nb ? band_start(height, i + 1) : height;
            const int need = std::min(height, y1 + r_hi);
            if (need > uploaded) {
                e = copy_rows(v->src, sp, src, row_in, row_in, uploaded, need, cudaMemcpyHostToDevice,
                              nb > 1 ? v->up : s);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "copy input to device");
                    break;
                }
                uploaded = need;
            }
            if (nb > 1 && ((e = cudaEventRecord(v->ev_up[i], v->up)) != cudaSuccess ||
                           (e = cudaStreamWaitEvent(s, v->ev_up[i], 0)) != cudaSuccess)) {
                rc = cuda_fail(e, "order band upload");
                break;
            }
            // every SM on each band: its rows are few, the upload bounds the call
            bnz_tile tile = {0, 0, 0, 0};
            if (nb > 1)
                tile.tile_h = (int)std::max<long long>(8, (strips * (y1 - y0) + sms - 1) / sms);
            rc = binarize_dev(static_cast<const uint8_t *>(v->src), sp, height, width, channels, W, rule, k, R,
                              static_cast<uint8_t *>(v->dst), dp, 0, nb > 1 ? &tile : nullptr, s, v->stats, y0, y1);
            if (rc != BNZ_OK)
                break;
            if (nb > 1 && ((e = cudaEventRecord(v->ev_k[i], s)) != cudaSuccess ||
                           (e = cudaStreamWaitEvent(v->down, v->ev_k[i], 0)) != cudaSuccess)) {
                rc = cuda_fail(e, "order band download");
                break;
            }
            e = copy_rows(dst, (size_t)width, v->dst, dp, (size_t)width, y0, y1, cudaMemcpyDeviceToHost,
                          nb > 1 ? v->down : s);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "copy result to host");
                break;
            }
        }
        if (rc != BNZ_OK)
            break;
        // the download stream has waited for the last kernel
        if ((e = cudaMemcpyAsync(v->h_stats, v->stats, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 nb > 1 ? v->down : s)) != cudaSuccess) {
            rc = cuda_fail(e, "read statistics");
            break;
        }
    } while (0);
    // all three streams, also after an error, so no copy outlives the call
    for (cudaStream_t q : {v->up, s, v->down}) {
        e = cudaStreamSynchronize(q);
        if (rc == BNZ_OK && e != cudaSuccess)
            rc = cuda_fail(e, "cudaStreamSynchronize");
    }
    if (rc == BNZ_OK && v->h_stats[BNZ_STATS_TIMEOUTS] != 0)
        rc = fail(BNZ_ETIMEOUT, "a device-side wait timed out; output incomplete");
    return rc;
}

// One host page, several settings (bnz_binarize_runs): the page goes up once,
// in as many row bands as binarize_host uses but of equal height, and every
// band runs each setting's
// kernel as soon as the rows its windows reach are up; each (band, setting)
// mask comes down on the download stream as soon as its kernel is done.
static int binarize_runs_host(const uint8_t *src, int height, int width, int channels, const bnz_run *runs,
                              int nruns)
{
    if (!runs || nruns < 1 || nruns > 1024)
        return fail(BNZ_EINVAL, "bnz_binarize_runs: 1 to 1024 settings (got %d)", nruns);
    int Wmax = 1;
    for (int r = 0; r < nruns; ++r) {
        const bnz_run &u = runs[r];
        const double R = u.rule == BNZ_NIBLACK ? 1.0 : u.R;
        int rc = check_common(src, (size_t)width * channels, height, width, channels, u.W, u.rule, u.k, R, u.dst,
                              (size_t)width, 0);
        if (rc != BNZ_OK)
            return fail(rc, "setting %d: %s", r, bnz_last_error());
        Wmax = std::max(Wmax, u.W);
    }
    int dev = 0;
    int rc = current_device(&dev);
    if (rc != BNZ_OK)
        return rc;
    int sms = 0;
    rc = device_sm_count(&sms);
    if (rc != BNZ_OK)
        return rc;
    const size_t row_in = (size_t)width * channels;
    const size_t sp = (row_in + 15) & ~size_t(15);
    const size_t dp = ((size_t)width + 15) & ~size_t(15);
    const size_t mask_bytes = dp * height;
    HostCallState::PerDevice *v = nullptr;
    rc = host_call_state(dev, sp * height, mask_bytes * nruns, &v);
    if (rc != BNZ_OK)
        return rc;
    const int nb = host_bands(height, width, Wmax);
    cudaError_t e = cudaSuccess;
    while ((int)v->ev_run.size() < nb * nruns) {
        cudaEvent_t ev = nullptr;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate");
        v->ev_run.push_back(ev);
    }
    cudaStream_t s = v->stream;
    std::vector<long long> strips(nruns, 1);
    for (int r = 0; r < nruns && nb > 1; ++r) {
        FusedPlan shape;
        if ((rc = plan_shape(height, width, channels, runs[r].W, 0, &shape)) != BNZ_OK)
            return rc;
        strips[r] = shape.tiles_x;
    }
    do {
        if ((e = cudaMemsetAsync(v->stats, 0, 4 * sizeof(unsigned long long), s)) != cudaSuccess) {
            rc = cuda_fail(e, "clear statistics");
            break;
        }
        int uploaded = 0;
        for (int i = 0; i < nb && rc == BNZ_OK; ++i) {
            // equal bands: with several masks per band the downloads dominate, and they start as soon as the
            // first band's kernels are done (measured 4 % faster than halving bands for 8 settings)
            const int y0 = (int)((long long)height * i / nb), y1 = (int)((long long)height * (i + 1) / nb);
            const int need = std::min(height, y1 + (Wmax - 1 - Wmax / 2));
            if (need > uploaded) {
                e = copy_rows(v->src, sp, src, row_in, row_in, uploaded, need, cudaMemcpyHostToDevice, v->up);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "copy input to device");
                    break;
                }
                uploaded = need;
            }
            if ((e = cudaEventRecord(v->ev_up[i], v->up)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(s, v->ev_up[i], 0)) != cudaSuccess) {
                rc = cuda_fail(e, "order band upload");
                break;
            }
            for (int r = 0; r < nruns && rc == BNZ_OK; ++r) {
                const bnz_run &u = runs[r];
                uint8_t *dmask = static_cast<uint8_t *>(v->dst) + (size_t)r * mask_bytes;
                bnz_tile tile = {0, 0, 0, 0};
                if (nb > 1)
                    tile.tile_h = (int)std::max<long long>(8, (strips[r] * (y1 - y0) + sms - 1) / sms);
                rc = binarize_dev(static_cast<const uint8_t *>(v->src), sp, height, width, channels, u.W, u.rule, u.k,
                                  u.rule == BNZ_NIBLACK ? 1.0 : u.R, dmask, dp, 0, nb > 1 ? &tile : nullptr, s,
                                  v->stats, y0, y1);
                if (rc != BNZ_OK)
                    break;
                cudaEvent_t ev = v->ev_run[(size_t)i * nruns + r];
                if ((e = cudaEventRecord(ev, s)) != cudaSuccess || (e = cudaStreamWaitEvent(v->down, ev, 0)) != cudaSuccess) {
                    rc = cuda_fail(e, "order mask download");
                    break;
                }
                e = copy_rows(u.dst, (size_t)width, dmask, dp, (size_t)width, y0, y1, cudaMemcpyDeviceToHost, v->down);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "copy result to host");
                    break;
                }
            }
        }
        if (rc != BNZ_OK)
            break;
        if ((e = cudaMemcpyAsync(v->h_stats, v->stats, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 v->down)) != cudaSuccess) {
            rc = cuda_fail(e, "read statistics");
            break;
        }
    } while (0);
    for (cudaStream_t q : {v->up, s, v->down}) {
        e = cudaStreamSynchronize(q);
        if (rc == BNZ_OK && e != cudaSuccess)
            rc = cuda_fail(e, "cudaStreamSynchronize");
    }
    if (rc == BNZ_OK && v->h_stats[BNZ_STATS_TIMEOUTS] != 0)
        rc = fail(BNZ_ETIMEOUT, "a device-side wait timed out; output incomplete");
    return rc;
}

} // namespace bnz

using namespace bnz;

extern "C" {

int bnz_binarize_runs(const uint8_t *src, int height, int width, int channels, const bnz_run *runs, int nruns)
{
    return binarize_runs_host(src, height, width, channels, runs, nruns);
}

int bnz_binarize_window(const uint8_t *src, int height, int width, int channels, int W, int rule, double k, double R,
                        uint8_t *dst, size_t window_bytes)
{
    return binarize_window_host(src, height, width, channels, W, rule, k, rule == BNZ_NIBLACK ? 1.0 : R, dst,
                                window_bytes);
}

int bnz_sauvola(const uint8_t *src, int height, int width, int channels, int W, double k, double R, uint8_t *dst)
{
    return binarize_host(src, height, width, channels, W, BNZ_SAUVOLA, k, R, dst);
}

int bnz_niblack(const uint8_t *src, int height, int width, int channels, int W, double k, uint8_t *dst)
{
    return binarize_host(src, height, width, channels, W, BNZ_NIBLACK, k, 1.0, dst);
}

int bnz_sauvola_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels, int W, double k,
                    double R, uint8_t *d_dst, size_t dst_pitch, int packed, void *stream,
                    unsigned long long *d_stats)
{
    return binarize_dev(d_src, src_pitch, height, width, channels, W, BNZ_SAUVOLA, k, R, d_dst, dst_pitch, packed,
                        nullptr, stream, d_stats);
}

int bnz_niblack_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels, int W, double k,
                    uint8_t *d_dst, size_t dst_pitch, int packed, void *stream, unsigned long long *d_stats)
{
    return binarize_dev(d_src, src_pitch, height, width, channels, W, BNZ_NIBLACK, k, 1.0, d_dst, dst_pitch,
                        packed, nullptr, stream, d_stats);
}

int bnz_binarize_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels, int W, int rule,
                     double k, double R, uint8_t *d_dst, size_t dst_pitch, int packed, const bnz_tile *tile,
                     void *stream, unsigned long long *d_stats)
{
    return binarize_dev(d_src, src_pitch, height, width, channels, W, rule, k, R, d_dst, dst_pitch, packed, tile,
                        stream, d_stats);
}

int bnz_dual_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels, int W, double k_sauvola,
                 double R, double k_niblack, uint8_t *d_dst_sauvola, uint8_t *d_dst_niblack, size_t dst_pitch,
                 int packed, void *stream, unsigned long long *d_stats)
{
    int rc = check_common(d_src, src_pitch, height, width, channels, W, BNZ_SAUVOLA, k_sauvola, R, d_dst_sauvola,
                          dst_pitch, packed);
    if (rc != BNZ_OK)
        return rc;
    if (!d_dst_niblack)
        return fail(BNZ_EINVAL, "null image pointer");
    if (!std::isfinite(k_niblack))
        return fail(BNZ_EINVAL, "k must be finite");
    const size_t mask_bytes = (size_t)(height - 1) * dst_pitch + (packed ? ((size_t)width + 7) / 8 : (size_t)width);
    const uintptr_t a = reinterpret_cast<uintptr_t>(d_dst_sauvola), b = reinterpret_cast<uintptr_t>(d_dst_niblack);
    if (a < b + mask_bytes && b < a + mask_bytes)
        return fail(BNZ_EINVAL, "the two masks overlap");
    if ((reinterpret_cast<uintptr_t>(d_src) & 15u) || (src_pitch & 15u))
        return fail(BNZ_EINVAL, "d_src must be 16-byte aligned with src_pitch a multiple of 16 (TMA)");
    unsigned int *err = nullptr;
    rc = device_err_flag(&err);
    if (rc != BNZ_OK)
        return rc;
    return launch_dual(d_src, src_pitch, height, width, channels, W, k_sauvola, R, k_niblack, d_dst_sauvola,
                       d_dst_niblack, dst_pitch, packed ? 1 : 0, nullptr, static_cast<cudaStream_t>(stream), d_stats,
                       err);
}

int bnz_otsu_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels, uint8_t *d_dst,
                 size_t dst_pitch, int packed, void *d_scratch, void *stream)
{
    // the window arguments of the shared checks do not apply: valid placeholders
    int rc = check_common(d_src, src_pitch, height, width, channels, 1, BNZ_SAUVOLA, 0.5, 1.0, d_dst, dst_pitch,
                          packed);
    if (rc != BNZ_OK)
        return rc;
    if ((long long)height * width > (1ll << 28))
        return fail(BNZ_EINVAL, "Otsu: at most 2^28 pixels (got %lld)", (long long)height * width);
    if ((reinterpret_cast<uintptr_t>(d_src) & 15u) || (src_pitch & 15u))
        return fail(BNZ_EINVAL, "d_src must be 16-byte aligned with src_pitch a multiple of 16");
    if (!d_scratch || (reinterpret_cast<uintptr_t>(d_scratch) & 15u))
        return fail(BNZ_EINVAL, "d_scratch must be a 16-byte aligned buffer of BNZ_OTSU_SCRATCH_BYTES");
    return launch_otsu(d_src, src_pitch, height, width, channels, d_dst, dst_pitch, packed ? 1 : 0, d_scratch,
                       static_cast<cudaStream_t>(stream));
}

int bnz_host_bands(int height, int width, int W, int *starts, int max_bands)
{
    if (height < 1 || width < 1 || W < 1 || W > BNZ_MAX_W)
        return -fail(BNZ_EINVAL, "height, width >= 1 and W in [1, %d] required", BNZ_MAX_W);
    const int nb = host_bands(height, width, W);
    if (starts) {
        if (max_bands < nb + 1)
            return -fail(BNZ_EINVAL, "starts must hold %d entries", nb + 1);
        for (int i = 0; i < nb; ++i)
            starts[i] = band_start(height, i);
        starts[nb] = height;
    }
    return nb;
}

size_t bnz_integral_scratch_bytes(int height, int width) { return integral_scratch_bytes(height, width); }

int bnz_binarize_integral_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels, int W,
                              int rule, double k, double R, uint8_t *d_dst, size_t dst_pitch, int packed,
                              void *d_scratch, size_t scratch_bytes, void *stream, unsigned long long *d_stats)
{
    int rc = check_common(d_src, src_pitch, height, width, channels, W, rule, k, R, d_dst, dst_pitch, packed);
    if (rc != BNZ_OK)
        return rc;
    if (height > 65535)
        return fail(BNZ_EINVAL, "the integral-image variant supports height <= 65535 (got %d)", height);
    const size_t need = integral_scratch_bytes(height, width);
    if (!d_scratch || scratch_bytes < need)
        return fail(BNZ_EINVAL, "scratch of %zu bytes needed (got %zu)", need, scratch_bytes);
    if (reinterpret_cast<uintptr_t>(d_scratch) & 31u)
        return fail(BNZ_EINVAL, "d_scratch must be 32-byte aligned");
    int dev = 0;
    rc = device_sm_count(&dev);
    if (rc != BNZ_OK)
        return rc;
    if (rule == BNZ_NIBLACK)
        R = 1.0;
    return launch_integral(d_src, src_pitch, height, width, channels, W, rule, k, R, d_dst, dst_pitch, packed,
                           d_scratch, static_cast<cudaStream_t>(stream), d_stats);
}

int bnz_integral_images_dev(const uint8_t *d_src, size_t src_pitch, int height, int width, int channels,
                            void *d_scratch, size_t scratch_bytes, long long *ld_elems, void *stream)
{
    if (!d_src || !d_scratch || !ld_elems)
        return fail(BNZ_EINVAL, "null pointer");
    if (height < 1 || width < 1 || (channels != 1 && channels != 3) || src_pitch < (size_t)width * channels)
        return fail(BNZ_EINVAL, "bad image geometry");
    const size_t need = integral_scratch_bytes(height, width);
    if (scratch_bytes < need || (reinterpret_cast<uintptr_t>(d_scratch) & 31u))
        return fail(BNZ_EINVAL, "scratch of %zu bytes (32-byte aligned) needed", need);
    int dev = 0;
    int rc = device_sm_count(&dev);
    if (rc != BNZ_OK)
        return rc;
    return launch_integral_tables(d_src, src_pitch, height, width, channels, d_scratch,
                                  static_cast<cudaStream_t>(stream), ld_elems);
}

const char *bnz_last_error(void) { return t_err.c_str(); }

int bnz_copy2d_async(void *dst, size_t dst_pitch, const void *src, size_t src_pitch, size_t width_bytes,
                     size_t height, void *stream)
{
    if (width_bytes == 0 || height == 0)
        return BNZ_OK;
    if (!dst || !src || dst_pitch < width_bytes || src_pitch < width_bytes)
        return fail(BNZ_EINVAL, "bnz_copy2d_async: null pointer or pitch below the row width");
    int dev = 0;
    int rc = current_device(&dev);
    if (rc != BNZ_OK)
        return rc;
    cudaError_t e = cudaMemcpy2DAsync(dst, dst_pitch, src, src_pitch, width_bytes, height, cudaMemcpyDefault,
                                      static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? BNZ_OK : cuda_fail(e, "cudaMemcpy2DAsync");
}

int bnz_decision_margins(int rule, double k, double R, float *E, float *E_int, float *Tdf)
{
    if (!E || !E_int || !Tdf)
        return fail(BNZ_EINVAL, "null output pointer");
    if (rule != BNZ_SAUVOLA && rule != BNZ_NIBLACK)
        return fail(BNZ_EINVAL, "rule must be BNZ_SAUVOLA or BNZ_NIBLACK (got %d)", rule);
    if (!(std::fabs(k) <= BNZ_MAX_ABS_K))
        return fail(BNZ_EINVAL, "k must be finite with |k| <= %g (got %g)", BNZ_MAX_ABS_K, k);
    if (rule == BNZ_SAUVOLA && !(R >= BNZ_MIN_R && std::isfinite(R)))
        return fail(BNZ_EINVAL, "R must be finite and >= %g for Sauvola (got %g)", BNZ_MIN_R, R);
    if (rule == BNZ_NIBLACK)
        R = 1.0;
    *E = decision_margin(rule, k, R);
    *E_int = decision_margin_interior(rule, k, R);
    *Tdf = double_float_cut(rule, k, R);
    return BNZ_OK;
}

int bnz_version(void) { return 200; } // 0.2.0: the Otsu scratch grew to BNZ_OTSU_SCRATCH_BYTES = 20480

int bnz_fused_plan(int height, int width, int channels, int W, const bnz_tile *tile, size_t *smem_bytes,
                   int *grid_ctas, int *tile_w, int *tile_h)
{
    if (height < 1 || width < 1 || (channels != 1 && channels != 3) || W < 1 || W > BNZ_MAX_W)
        return fail(BNZ_EINVAL, "bad plan arguments");
    FusedPlan pl;
    int rc = plan_fused(height, width, channels, W, tile, &pl);
    if (rc != BNZ_OK)
        return rc;
    if (smem_bytes)
        *smem_bytes = pl.smem;
    if (grid_ctas)
        *grid_ctas = pl.grid;
    if (tile_w)
        *tile_w = pl.TW;
    if (tile_h)
        *tile_h = pl.rows_per_cta;
    return BNZ_OK;
}

} // extern "C"
