// batch.cu -- many uneven pages in one persistent launch (row a9).
//
// The strip-rows of all pages of a batch (strip-major within each page,
// pages one after another, largest window first) form one index range, a
// work queue that the persistent CTAs take from in pieces: a device cursor
// hands each CTA the next max(128, remaining / (2 * grid)) strip-rows (large
// pieces first, small ones at the end, so the CTAs finish together whatever
// the pages cost).  Each CTA walks its piece segment by segment; a segment
// never crosses a page, and for each one the CTA reads the page's descriptor
// (TMA tensor map, geometry, threshold constants) from device memory and runs
// the same producer / consumer code as the single-page kernel, instantiated
// for the page's rule and W mod 8.  Gray and RGB pages go to two launches
// (one per channel count); with a CUDA graph the whole batch, cursor resets
// included, is replayed with one call.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "segment.cuh"

namespace bnz {
namespace {

constexpr size_t kCursorBytes = 128; // one work-queue cursor per channel group, 128-byte aligned

struct alignas(128) PageDesc {
    CUtensorMap map;  // 128 bytes, 128-byte aligned (as cuda.h declares it): TMA reads it from global memory
    FusedParams p;
    long long t0;     // first strip-row of this page in the batch's index range
    int sel;          // rule * 8 + (W mod 8)
    int pad;
};

// Descriptors of an asynchronous batch reach the device as kernel parameters
// (the launch copies them), not through a copy from pageable host memory: the
// driver may order such a copy after the stream's earlier work, which would
// block the calling thread (a serving loop) until the previous step is done.
constexpr int kDescWords = (int)(sizeof(PageDesc) / 16);
constexpr int kDescPerPut = 3968 / (int)sizeof(PageDesc); // 4 KB of kernel parameters at most
static_assert(sizeof(PageDesc) % 16 == 0 && kDescPerPut >= 1, "descriptor upload chunk");

struct DescPut {
    uint4 w[kDescPerPut * kDescWords];
};

__global__ void __launch_bounds__(256) put_descs(const __grid_constant__ DescPut src, int words, uint4 *dst)
{
    for (int i = threadIdx.x; i < words; i += blockDim.x)
        dst[i] = src.w[i];
}

template <int CIN>
__device__ __forceinline__ void dispatch(int sel, const CUtensorMap *map, const FusedParams &p, const Segment &sg,
                                         uint8_t *smem, uint64_t &phase, uint64_t &ephase, uint64_t &eused,
                                         uint32_t &nfb, uint32_t &nties,
                                         volatile int *s_abort)
{
#define BNZ_CASE(R, M)                                                                                             \
    case (R) * 8 + (M):                                                                                            \
        run_segment<CIN, R, M>(map, p, sg, smem, phase, ephase, eused, nfb, nties, s_abort);                      \
        break;
    switch (sel) {
        BNZ_CASE(0, 0) BNZ_CASE(0, 1) BNZ_CASE(0, 2) BNZ_CASE(0, 3)
        BNZ_CASE(0, 4) BNZ_CASE(0, 5) BNZ_CASE(0, 6) BNZ_CASE(0, 7)
        BNZ_CASE(1, 0) BNZ_CASE(1, 1) BNZ_CASE(1, 2) BNZ_CASE(1, 3)
        BNZ_CASE(1, 4) BNZ_CASE(1, 5) BNZ_CASE(1, 6) BNZ_CASE(1, 7)
    default:
        break;
    }
#undef BNZ_CASE
}

constexpr long long kMinPiece = 128; // strip-rows of the smallest piece a CTA takes from the queue

template <int CIN>
__global__ void __launch_bounds__(NT, 1)
    batch_kernel(const PageDesc *__restrict__ pages, int npages, long long total, unsigned long long *stats,
                 unsigned int *err_flag, unsigned long long *cursor)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_abort;
    __shared__ FusedParams s_p;
    __shared__ long long s_piece[2];
    if (threadIdx.x == 0) {
        init_barriers(smem, kEmpty);
        s_abort = 0;
    }
    init_recip_table(smem);
    __syncthreads();
    uint64_t phase = 0, ephase = 0, eused = 0;
    uint32_t nfb = 0, nties = 0;
    for (;;) {
    if (threadIdx.x == 0) { // the next piece of the queue
        const long long seen = (long long)*reinterpret_cast<volatile unsigned long long *>(cursor);
        const long long size = max(kMinPiece, (total - seen) / (2 * (long long)gridDim.x));
        const long long st = (long long)atomicAdd(cursor, (unsigned long long)size);
        s_piece[0] = st;
        s_piece[1] = min(st + size, total);
    }
    __syncthreads();
    const long long L0 = s_piece[0], L1 = s_piece[1];
    if (L0 >= total)
        break;
    int pi = 0;
    for (long long cur = L0; cur < L1;) {
        // the page holding strip-row cur (pages are few; ranges are sorted)
        int lo = pi, hi = npages - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pages[mid].t0 <= cur)
                lo = mid;
            else
                hi = mid - 1;
        }
        pi = lo;
        const PageDesc &pd = pages[pi];
        const long long page_end = (pi + 1 < npages) ? pages[pi + 1].t0 : total;
        // the page's parameters in shared memory for the segment
        for (int i = threadIdx.x; i < (int)(sizeof(FusedParams) / 4); i += NT)
            reinterpret_cast<uint32_t *>(&s_p)[i] = reinterpret_cast<const uint32_t *>(&pd.p)[i];
        __syncthreads();
        const Segment sg = make_segment(s_p, cur - pd.t0, min(L1, page_end) - pd.t0);
        cur += sg.th_eff;
        dispatch<CIN>(pd.sel, &pd.map, s_p, sg, smem, phase, ephase, eused, nfb, nties, &s_abort);
        __syncthreads(); // the next segment reuses the ring and s_p
        if (s_abort)
            break;
    }
    if (s_abort)
        break;
    }
    report(stats, err_flag, nfb, nties, s_abort != 0);
}

struct Group {
    int ch = 0;
    std::vector<PageDesc> host;
    PageDesc *dev = nullptr;
    unsigned long long *cursor = nullptr; // the group's work-queue cursor (device, after the descriptors)
    bool owned = false; // dev allocated by the batch (freed with it)
    long long total = 0;
    size_t smem = 0;
    int grid = 0;
};

} // namespace
} // namespace bnz

struct bnz_batch {
    bnz::Group groups[2]; // gray, RGB
    int npages = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long *stats = nullptr;
    unsigned int *err = nullptr;
    int device = 0;
};

namespace bnz {
namespace {

int launch_group(const Group &g, unsigned long long *stats, unsigned int *err, cudaStream_t stream)
{
    if (g.host.empty())
        return BNZ_OK;
    const void *fn = g.ch == 1 ? reinterpret_cast<const void *>(&batch_kernel<1>)
                               : reinterpret_cast<const void *>(&batch_kernel<3>);
    const PageDesc *pages = g.dev;
    int npages = (int)g.host.size();
    long long total = g.total;
    unsigned long long *cursor = g.cursor;
    cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "reset batch work queue");
    void *args[] = {(void *)&pages, (void *)&npages, (void *)&total, (void *)&stats, (void *)&err, (void *)&cursor};
    e = cudaLaunchKernel(fn, dim3((unsigned)g.grid), dim3(NT), args, g.smem, stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "launch batch kernel");
    return BNZ_OK;
}

int launch_batch(const bnz_batch *b, cudaStream_t stream)
{
    for (const Group &g : b->groups) {
        int rc = launch_group(g, b->stats, b->err, stream);
        if (rc != BNZ_OK)
            return rc;
    }
    return BNZ_OK;
}

void free_batch(bnz_batch *b)
{
    if (!b)
        return;
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    for (Group &g : b->groups)
        if (g.dev && g.owned)
            cudaFree(g.dev);
    delete b;
}

} // namespace
} // namespace bnz

using namespace bnz;

extern "C" {

static int plan_batch(const bnz_page *pages, int n, unsigned long long *d_stats, bnz_batch **out)
{
    if (!out)
        return fail(BNZ_EINVAL, "null output handle");
    *out = nullptr;
    if (!pages || n < 1)
        return fail(BNZ_EINVAL, "a batch needs at least one page");
    int sms = 0;
    int rc = device_sm_count(&sms);
    if (rc != BNZ_OK)
        return rc;
    unsigned int *err = nullptr;
    rc = device_err_flag(&err);
    if (rc != BNZ_OK)
        return rc;
    bnz_batch *b = new (std::nothrow) bnz_batch();
    if (!b)
        return fail(BNZ_ENOMEM, "host allocation failed");
    b->npages = n;
    b->stats = d_stats;
    b->err = err;
    cudaGetDevice(&b->device);
    b->groups[0].ch = 1;
    b->groups[1].ch = 3;
    for (int i = 0; i < n; ++i) {
        const bnz_page &pg = pages[i];
        rc = check_common(pg.d_src, pg.src_pitch, pg.height, pg.width, pg.channels, pg.W, pg.rule, pg.k, pg.R,
                          pg.d_dst, pg.dst_pitch, pg.packed);
        if (rc == BNZ_OK && ((reinterpret_cast<uintptr_t>(pg.d_src) & 15u) || (pg.src_pitch & 15u)))
            rc = fail(BNZ_EINVAL, "page %d: d_src must be 16-byte aligned with src_pitch a multiple of 16", i);
        FusedPlan pl;
        if (rc == BNZ_OK) { // tile_w is a preference: fall back to the default shape if it does not fit
            rc = plan_shape(pg.height, pg.width, pg.channels, pg.W, pg.tile_w, &pl);
            if (rc != BNZ_OK && pg.tile_w)
                rc = plan_shape(pg.height, pg.width, pg.channels, pg.W, 0, &pl);
        }
        if (rc != BNZ_OK) {
            free_batch(b);
            return fail(rc, "page %d: %s", i, bnz_last_error());
        }
        Group &g = b->groups[pg.channels == 1 ? 0 : 1];
        PageDesc d;
        memset(&d, 0, sizeof d);
        rc = encode_span_map(&d.map, pg.d_src, (uint64_t)pg.width * pg.channels, (uint64_t)pg.height,
                             (uint64_t)pg.src_pitch, (uint32_t)(pl.SWP * pg.channels), (uint32_t)CH);
        if (rc != BNZ_OK) {
            free_batch(b);
            return rc;
        }
        const double R = pg.rule == BNZ_NIBLACK ? 1.0 : pg.R;
        fill_fused_params(&d.p, pl, pg.height, pg.width, pg.W, pg.rule, pg.k, R, pg.d_dst, pg.dst_pitch, pg.packed,
                          d_stats, err);
        d.t0 = (long long)pl.tiles_x * pg.height; // strip rows of this page; turned into offsets below
        d.sel = pg.rule * 8 + (pg.W & 7);
        g.smem = std::max(g.smem, pl.smem);
        g.host.push_back(d);
    }
    for (Group &g : b->groups) {
        if (g.host.empty())
            continue;
        // largest window first (its pages cost the most per pixel: they should not be
        // left for the end of the queue), and pages of the same kernel instance
        // (rule, W mod 8) next to each other: the CTAs take consecutive pieces, so
        // most of them then run the same code at any time instead of thrashing the
        // instruction caches
        std::stable_sort(g.host.begin(), g.host.end(), [](const PageDesc &a, const PageDesc &c) {
            return a.p.W != c.p.W ? a.p.W > c.p.W : a.sel < c.sel;
        });
        for (PageDesc &d : g.host) {
            const long long rows = d.t0;
            d.t0 = g.total;
            g.total += rows;
        }
        const void *fn = g.ch == 1 ? reinterpret_cast<const void *>(&batch_kernel<1>)
                                   : reinterpret_cast<const void *>(&batch_kernel<3>);
        const int occ = 1; // 512 threads x up to 128 registers: one CTA per SM
        rc = ensure_smem_optin(fn);
        if (rc != BNZ_OK) {
            free_batch(b);
            return rc;
        }
        g.grid = (int)std::max<long long>(1, std::min<long long>((long long)sms * std::max(occ, 1), g.total / 32 + 1));
    }
    *out = b;
    return BNZ_OK;
}

int bnz_batch_create(const bnz_page *pages, int n, int use_graph, unsigned long long *d_stats, bnz_batch **out)
{
    bnz_batch *b = nullptr;
    int rc = plan_batch(pages, n, d_stats, &b);
    if (rc != BNZ_OK)
        return rc;
    for (Group &g : b->groups) {
        if (g.host.empty())
            continue;
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, g.host.size() * sizeof(PageDesc) + kCursorBytes);
        if (e == cudaSuccess) {
            g.dev = static_cast<PageDesc *>(p);
            g.cursor = reinterpret_cast<unsigned long long *>(g.dev + g.host.size());
            g.owned = true;
            e = cudaMemcpy(g.dev, g.host.data(), g.host.size() * sizeof(PageDesc), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) {
            free_batch(b);
            return cuda_fail(e, "batch descriptors");
        }
    }
    if (use_graph) {
        cudaStream_t s = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = launch_batch(b, s);
            cudaError_t e2 = cudaStreamEndCapture(s, &b->graph);
            if (rc == BNZ_OK && e2 != cudaSuccess)
                e = e2;
        }
        if (e == cudaSuccess && rc == BNZ_OK)
            e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (s)
            cudaStreamDestroy(s);
        if (e != cudaSuccess || rc != BNZ_OK) {
            free_batch(b);
            return rc != BNZ_OK ? rc : cuda_fail(e, "capture batch graph");
        }
    }
    *out = b;
    return BNZ_OK;
}

size_t bnz_batch_desc_bytes(int n) { return n > 0 ? (size_t)n * sizeof(PageDesc) + 2 * kCursorBytes : 0; }

int bnz_batch_create_async(const bnz_page *pages, int n, void *d_desc, size_t desc_bytes, void *stream,
                           unsigned long long *d_stats, bnz_batch **out)
{
    if (!d_desc || (reinterpret_cast<uintptr_t>(d_desc) & 127u) || desc_bytes < bnz_batch_desc_bytes(n))
        return fail(BNZ_EINVAL, "d_desc must be 128-byte aligned device memory of bnz_batch_desc_bytes(n) bytes");
    bnz_batch *b = nullptr;
    int rc = plan_batch(pages, n, d_stats, &b);
    if (rc != BNZ_OK)
        return rc;
    PageDesc *next = static_cast<PageDesc *>(d_desc);
    unsigned long long *cursors = reinterpret_cast<unsigned long long *>(static_cast<uint8_t *>(d_desc) +
                                                                         (size_t)n * sizeof(PageDesc));
    for (int gi = 0; gi < 2; ++gi) {
        Group &g = b->groups[gi];
        if (g.host.empty())
            continue;
        g.dev = next;
        g.cursor = cursors + gi * (kCursorBytes / sizeof(unsigned long long));
        next += g.host.size();
        for (size_t i0 = 0; i0 < g.host.size(); i0 += kDescPerPut) {
            const int m = (int)std::min<size_t>(kDescPerPut, g.host.size() - i0);
            DescPut put;
            memcpy(put.w, &g.host[i0], (size_t)m * sizeof(PageDesc));
            put_descs<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(put, m * kDescWords,
                                                                         reinterpret_cast<uint4 *>(g.dev + i0));
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            free_batch(b);
            return cuda_fail(e, "batch descriptors");
        }
    }
    *out = b;
    return BNZ_OK;
}

int bnz_batch_run(bnz_batch *b, void *stream)
{
    if (!b)
        return fail(BNZ_EINVAL, "null batch");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (b->exec) {
        cudaError_t e = cudaGraphLaunch(b->exec, s);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaGraphLaunch(batch)");
        return BNZ_OK;
    }
    return launch_batch(b, s);
}

int bnz_batch_info(const bnz_batch *b, int *pages, int *launches, int *grid, size_t *smem, long long *strip_rows)
{
    if (!b)
        return fail(BNZ_EINVAL, "null batch");
    int nl = 0, gmax = 0;
    size_t smax = 0;
    long long rows = 0;
    for (const Group &g : b->groups)
        if (!g.host.empty()) {
            ++nl;
            gmax = std::max(gmax, g.grid);
            smax = std::max(smax, g.smem);
            rows += g.total;
        }
    if (pages)
        *pages = b->npages;
    if (launches)
        *launches = nl;
    if (grid)
        *grid = gmax;
    if (smem)
        *smem = smax;
    if (strip_rows)
        *strip_rows = rows;
    return BNZ_OK;
}

int bnz_batch_destroy(bnz_batch *b)
{
    free_batch(b);
    return BNZ_OK;
}

} // extern "C"
