// integral.cu -- the integral-image comparison variant (row a8).
//
// Sec. 1 cites Shafait et al.: m and s from two summed-area tables ("integral
// images") of f and f^2, O(N^2) work but, per Sec. 3.3, 12 S_z bytes of
// memory (the paper's widths: 32-bit for f, 64-bit for f^2).  Here both tables
// are int64, because the sum of f over a 16384^2 page exceeds 2^32:
//   I1[y][x] = sum of f over rows < y and columns < x,  I2 likewise for f^2,
// both (h+1) x (w+1), first row and column zero, in caller-provided scratch.
// Three passes build them (row prefix; column prefix in 256-row segments:
// segment sums, a scan over segments, then the in-segment prefix); a fourth
// reads four corners of each table per pixel and takes the same Eq. 3
// decision as the fused kernel (fp32 filter with the proven margin, fp64
// re-evaluation inside it), so the masks are identical bit for bit.
#include <algorithm>
#include <mutex>

#include "decide.cuh"
#include "internal.h"

namespace bnz {
namespace {

constexpr int SEG = 256;  // rows per column-prefix segment
constexpr int RT = 256;   // threads of the row-prefix kernel, 4 px each per tile
constexpr int TILE = 4 * RT;

struct IntegralGeom {
    int h, w;
    long long ld;   // row stride of I1/I2 in elements
    int nseg;       // ceil((h + 1) / SEG)
    int64_t *I1, *I2, *G1, *G2; // tables and per-segment column sums
};

template <int CIN>
__device__ __forceinline__ uint32_t gray_at(const uint8_t *row, int x)
{
    if (CIN == 1)
        return row[x];
    return gray_rgb(row + 3 * x);
}

// Pass 1: I[y+1][x+1] = sum over columns <= x of row y (f and f^2); I[y+1][0] = 0.
// Row 0 of the tables is written by pass 1's block y = -1 (blockIdx.x == 0).
template <int CIN>
__global__ void __launch_bounds__(RT) row_prefix_kernel(const uint8_t *src, size_t pitch, IntegralGeom g)
{
    __shared__ long long s_a[RT / 32], s_b[RT / 32];
    const int yb = (int)blockIdx.x - 1; // -1: the zero row of the tables
    int64_t *o1 = g.I1 + (long long)(yb + 1) * g.ld;
    int64_t *o2 = g.I2 + (long long)(yb + 1) * g.ld;
    if (yb < 0) {
        for (int x = threadIdx.x; x <= g.w; x += RT)
            o1[x] = o2[x] = 0;
        return;
    }
    const uint8_t *row = src + (size_t)yb * pitch;
    if (threadIdx.x == 0)
        o1[0] = o2[0] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long carry1 = 0, carry2 = 0;
    for (int t0 = 0; t0 < g.w; t0 += TILE) {
        const int x = t0 + 4 * threadIdx.x;
        long long v1[4], v2[4];
        long long a = 0, b = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t f = (x + j < g.w) ? gray_at<CIN>(row, x + j) : 0u;
            a += f;
            b += (long long)f * f;
            v1[j] = a;
            v2[j] = b;
        }
        // block-wide inclusive scan of the thread totals
        long long ia = a, ib = b;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long ta = __shfl_up_sync(0xffffffffu, ia, off);
            const long long tb = __shfl_up_sync(0xffffffffu, ib, off);
            if (lane >= off) {
                ia += ta;
                ib += tb;
            }
        }
        if (lane == 31) {
            s_a[warp] = ia;
            s_b[warp] = ib;
        }
        __syncthreads();
        long long wa = 0, wb = 0, ta = 0, tb = 0;
        for (int k = 0; k < RT / 32; ++k) {
            if (k < warp) {
                wa += s_a[k];
                wb += s_b[k];
            }
            ta += s_a[k];
            tb += s_b[k];
        }
        const long long base1 = carry1 + wa + ia - a, base2 = carry2 + wb + ib - b;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (x + j < g.w) {
                o1[x + j + 1] = base1 + v1[j];
                o2[x + j + 1] = base2 + v2[j];
            }
        carry1 += ta;
        carry2 += tb;
        __syncthreads();
    }
}

// Pass 2a: per (segment, column) sums of the row-prefixed table over the segment's rows.
__global__ void seg_sum_kernel(IntegralGeom g)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (x > g.w)
        return;
    const int r0 = s * SEG, r1 = min(r0 + SEG, g.h + 1);
    long long a = 0, b = 0;
    for (int r = r0; r < r1; ++r) {
        a += g.I1[(long long)r * g.ld + x];
        b += g.I2[(long long)r * g.ld + x];
    }
    g.G1[(long long)s * g.ld + x] = a;
    g.G2[(long long)s * g.ld + x] = b;
}

// Pass 2b: exclusive scan of the segment sums down each column.
__global__ void seg_scan_kernel(IntegralGeom g)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x > g.w)
        return;
    long long a = 0, b = 0;
    for (int s = 0; s < g.nseg; ++s) {
        const long long ta = g.G1[(long long)s * g.ld + x], tb = g.G2[(long long)s * g.ld + x];
        g.G1[(long long)s * g.ld + x] = a;
        g.G2[(long long)s * g.ld + x] = b;
        a += ta;
        b += tb;
    }
}

// Pass 2c: in-segment prefix down each column plus the segment's offset.
__global__ void seg_apply_kernel(IntegralGeom g)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (x > g.w)
        return;
    const int r0 = s * SEG, r1 = min(r0 + SEG, g.h + 1);
    long long a = g.G1[(long long)s * g.ld + x], b = g.G2[(long long)s * g.ld + x];
    for (int r = r0; r < r1; ++r) {
        a += g.I1[(long long)r * g.ld + x];
        b += g.I2[(long long)r * g.ld + x];
        g.I1[(long long)r * g.ld + x] = a;
        g.I2[(long long)r * g.ld + x] = b;
    }
}

// Pass 3: four corners per table, then the decision.  One thread per 8
// consecutive pixels (one packed byte).
template <int CIN, int RULE>
__global__ void __launch_bounds__(256) lookup_kernel(const uint8_t *src, size_t pitch, IntegralGeom g,
                                                     const FusedParams p)
{
    const int x8 = (blockIdx.x * blockDim.x + threadIdx.x) * 8;
    const int y = blockIdx.y;
    uint32_t nfb = 0, nties = 0;
    if (x8 < g.w) {
        const uint8_t *row = src + (size_t)y * pitch;
        const int ya = max(y - p.r_lo, 0), yb = min(y + p.r_hi, g.h - 1) + 1;
        const long long ra = (long long)ya * g.ld, rb = (long long)yb * g.ld;
        uint32_t bits = 0;
        uint8_t outb[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int x = x8 + j;
            uint32_t gv = 0;
            if (x < g.w) {
                const int xa = max(x - p.r_lo, 0), xb = min(x + p.r_hi, g.w - 1) + 1;
                const long long s1 = g.I1[rb + xb] - g.I1[ra + xb] - g.I1[rb + xa] + g.I1[ra + xa];
                const long long s2 = g.I2[rb + xb] - g.I2[ra + xb] - g.I2[rb + xa] + g.I2[ra + xa];
                const uint32_t n = (uint32_t)((yb - ya) * (xb - xa));
                gv = decide_pixel<RULE>(gray_at<CIN>(row, x), n, (uint32_t)s1, (uint32_t)s2, p, nfb, nties);
            }
            outb[j] = (uint8_t)gv;
            bits |= (gv & 1u) << j;
        }
        if (p.packed) {
            p.dst[(size_t)y * p.dst_pitch + (x8 >> 3)] = (uint8_t)bits;
        } else {
            uint8_t *d = p.dst + (size_t)y * p.dst_pitch + x8;
            if (p.vec_ok && x8 + 8 <= g.w) {
                *reinterpret_cast<uint2 *>(d) =
                    make_uint2(outb[0] | (outb[1] << 8) | (outb[2] << 16) | ((uint32_t)outb[3] << 24),
                               outb[4] | (outb[5] << 8) | (outb[6] << 16) | ((uint32_t)outb[7] << 24));
            } else {
                for (int j = 0; j < 8 && x8 + j < g.w; ++j)
                    d[j] = outb[j];
            }
        }
    }
    for (int off = 16; off; off >>= 1) {
        nfb += __shfl_xor_sync(0xffffffffu, nfb, off);
        nties += __shfl_xor_sync(0xffffffffu, nties, off);
    }
    if ((threadIdx.x & 31) == 0 && p.stats && (nfb | nties)) {
        atomicAdd(&p.stats[BNZ_STATS_FALLBACKS], (unsigned long long)nfb);
        atomicAdd(&p.stats[BNZ_STATS_TIES], (unsigned long long)nties);
    }
}

void geometry(int h, int w, void *scratch, IntegralGeom *g)
{
    g->h = h;
    g->w = w;
    g->ld = ((long long)w + 1 + 3) & ~3ll; // 32-byte aligned rows
    g->nseg = (h + 1 + SEG - 1) / SEG;
    int64_t *base = static_cast<int64_t *>(scratch);
    g->I1 = base;
    g->I2 = g->I1 + (long long)(h + 1) * g->ld;
    g->G1 = g->I2 + (long long)(h + 1) * g->ld;
    g->G2 = g->G1 + (long long)g->nseg * g->ld;
}

} // namespace

size_t integral_scratch_bytes(int h, int w)
{
    if (h < 1 || w < 1)
        return 0;
    IntegralGeom g;
    geometry(h, w, nullptr, &g);
    return (size_t)(2 * (long long)(h + 1) * g.ld + 2 * (long long)g.nseg * g.ld) * sizeof(int64_t);
}

int launch_integral_tables(const uint8_t *d_src, size_t src_pitch, int h, int w, int ch, void *scratch,
                           cudaStream_t stream, long long *ld_out)
{
    IntegralGeom g;
    geometry(h, w, scratch, &g);
    if (ld_out)
        *ld_out = g.ld;
    if (ch == 1)
        row_prefix_kernel<1><<<h + 1, RT, 0, stream>>>(d_src, src_pitch, g);
    else
        row_prefix_kernel<3><<<h + 1, RT, 0, stream>>>(d_src, src_pitch, g);
    const dim3 cb(256), cg((unsigned)((w + 1 + 255) / 256), (unsigned)g.nseg);
    seg_sum_kernel<<<cg, cb, 0, stream>>>(g);
    seg_scan_kernel<<<dim3(cg.x), cb, 0, stream>>>(g);
    seg_apply_kernel<<<cg, cb, 0, stream>>>(g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "integral-image kernels");
    return BNZ_OK;
}

int launch_integral(const uint8_t *d_src, size_t src_pitch, int h, int w, int ch, int W, int rule, double k, double R,
                    uint8_t *d_dst, size_t dst_pitch, int packed, void *scratch, cudaStream_t stream,
                    unsigned long long *d_stats)
{
    int rc = launch_integral_tables(d_src, src_pitch, h, w, ch, scratch, stream, nullptr);
    if (rc != BNZ_OK)
        return rc;
    IntegralGeom g;
    geometry(h, w, scratch, &g);
    FusedParams p;
    fill_decision_params(&p, h, w, W, rule, k, R);
    p.dst = d_dst;
    p.dst_pitch = (long long)dst_pitch;
    p.stats = d_stats;
    p.packed = packed ? 1 : 0;
    p.vec_ok = ((reinterpret_cast<uintptr_t>(d_dst) | dst_pitch) & 7u) == 0 ? 1 : 0;
    const dim3 blk(256), grd((unsigned)(((w + 7) / 8 + 255) / 256), (unsigned)h);
    if (ch == 1) {
        if (rule == BNZ_SAUVOLA)
            lookup_kernel<1, BNZ_SAUVOLA><<<grd, blk, 0, stream>>>(d_src, src_pitch, g, p);
        else
            lookup_kernel<1, BNZ_NIBLACK><<<grd, blk, 0, stream>>>(d_src, src_pitch, g, p);
    } else {
        if (rule == BNZ_SAUVOLA)
            lookup_kernel<3, BNZ_SAUVOLA><<<grd, blk, 0, stream>>>(d_src, src_pitch, g, p);
        else
            lookup_kernel<3, BNZ_NIBLACK><<<grd, blk, 0, stream>>>(d_src, src_pitch, g, p);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "integral-image lookup kernel");
    return BNZ_OK;
}

} // namespace bnz

// ---- allocation-free entry point -------------------------------------------
// Some callers cannot allocate device memory themselves: code hosted inside a
// framework that owns every device allocation through its own pool, or a
// fixed-budget pipeline that must not reach the allocator (and risk its
// latency or an out-of-memory failure) once it is running.  For them the
// integral-image scratch lives in this file-scope device array.  Every GPU
// that loads the library keeps it until the process exits.
namespace bnz {
namespace {

__device__ __align__(256) static unsigned char g_integral_static[BNZ_INTEGRAL_STATIC_MAX_BYTES];

std::mutex g_static_mu;
void *g_static_ptr[64];

// The array's device address for the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
int static_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64)
        return fail(BNZ_ENODEV, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_integral_static);
        if (e != cudaSuccess || !ptr)
            return cuda_fail(e, "cudaGetSymbolAddress(integral scratch)");
        g_static_ptr[dev] = ptr;
    }
    *out = g_static_ptr[dev];
    return BNZ_OK;
}

} // namespace
} // namespace bnz

extern "C" BNZ_API int bnz_binarize_integral_static_dev(const uint8_t *d_src, size_t src_pitch, int height,
                                                        int width, int channels, int W, int rule, double k,
                                                        double R, uint8_t *d_dst, size_t dst_pitch, int packed,
                                                        void *stream, unsigned long long *d_stats)
{
    using namespace bnz;
    int rc = check_common(d_src, src_pitch, height, width, channels, W, rule, k, R, d_dst, dst_pitch, packed);
    if (rc != BNZ_OK)
        return rc;
    const size_t need = integral_scratch_bytes(height, width);
    if (need > (size_t)BNZ_INTEGRAL_STATIC_MAX_BYTES || height > 65535)
        return fail(BNZ_EINVAL,
                    "a %d x %d page needs %zu bytes of integral-image scratch; the allocation-free entry point "
                    "holds at most %zu (about 2 Mpixel): pass your own scratch to bnz_binarize_integral_dev",
                    height, width, need, (size_t)BNZ_INTEGRAL_STATIC_MAX_BYTES);
    void *scratch = nullptr;
    rc = static_scratch(&scratch);
    if (rc != BNZ_OK)
        return rc;
    if (rule == BNZ_NIBLACK)
        R = 1.0;
    // The tables are rewritten completely by every call (their zero row and
    // column included), so nothing left by the previous call needs clearing.
    return launch_integral(d_src, src_pitch, height, width, channels, W, rule, k, R, d_dst, dst_pitch, packed,
                           scratch, static_cast<cudaStream_t>(stream), d_stats);
}
