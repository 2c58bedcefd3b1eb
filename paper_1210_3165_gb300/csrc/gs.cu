// gs.cu -- the reduced-set rule of Sec. 2 (Eq. 5) and the Eq. 6 confusion counts.
//
// Sec. 2 replaces the window set S by a reduced set S' of O(W) pixels taken
// from the window along geometric structures (Fig. 1) and thresholds with
// Eq. 5, t' = m' (1 + k (s'/R' - 1)), on the mean and deviation of S'.  The
// paper's drawings are not available; the structures here are this library's
// proposals, each a union of straight lines through the window (offsets
// (dy, dx) in [a, b]^2, a = -r_lo, b = r_hi):
//   cross      the centre row and the centre column
//   diagonals  dy = dx (|S'| = W) and dy = -dx (|dy| <= mm = min(r_lo, r_hi))
//   star       cross and diagonals
//   frame      rows a, b and columns a, b
//   frame + cross, frame + diagonals
// Samples outside the image are dropped (n' counts the rest), as for S.
//
// The paper evaluates every pixel's |S'| samples directly, O(W) per pixel.
// Here every line sum is carried from the row above in O(1), as the exact
// kernel carries its column sums: one CTA walks a 256-column strip down a
// segment of rows, one output column per thread, with
//   * a ring of the last W + 1 gray rows of the strip's span (the outputs
//     plus the window halo and one more column each side) in shared memory;
//   * vertical W-sums of every span column (the centre column and the
//     frame's side columns), updated by the entering and leaving rows;
//   * the two diagonal sums of every output column in slots indexed by
//     x - y and x + y, so that the sum of (y, x) continues the sum of
//     (y - 1, x - 1) (resp. (y - 1, x + 1)) with one entering and one leaving
//     pixel; the one diagonal per row that enters the strip is summed afresh
//     by a warp;
//   * the row sums (centre row, frame rows) from inclusive prefix sums of
//     those ring rows, one warp per row;
//   * the points where lines cross, counted twice or three times, taken off
//     once per extra count (a host-built list of at most kMaxCorr offsets).
// Every sum is an exact integer, and the decision of Eq. 3 on t' is the one
// every other kernel takes (fp32 filter with a proven margin, then the
// double-float and fp64 evaluations of the definition), so the mask equals
// the fp64 definition on (n', S1', S2') bit for bit.  Warm-up: a segment
// starts W - 1 rows above its first output row with empty sums and adds
// rows only; rows above the segment's first window are treated as zero
// there and never reach an output.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "decide.cuh"
#include "internal.h"

namespace bnz {
namespace {

constexpr int GT = 256;      // threads of a CTA = output columns of a strip
constexpr int kMaxCorr = 12; // crossing points of the structures (at most 9 for W >= 3)
constexpr int kPRow = 512;   // entries of a prefix row (the span is at most GT + BNZ_MAX_W + 1)
constexpr int kPF = 8;       // entering rows loaded ahead

enum : uint32_t { L_HC = 1u, L_VC = 2u, L_DP = 4u, L_DM = 8u, L_FRAME = 16u };

struct GsParams {
    const uint8_t *src;
    long long src_pitch;
    int a, b, mm;     // window offsets [a, b]; anti-diagonal offsets |d| <= mm
    int span, sp, nr; // span columns (GT + W + 1), their padded bytes, ring rows (W + 1)
    int seg_rows;     // output rows per CTA
    uint32_t lines;   // L_* bits of the structure
    int nh;           // prefix rows per step: centre row, frame top, frame bottom (in that order)
    int ncorr;
    int cdy[kMaxCorr], cdx[kMaxCorr], cex[kMaxCorr]; // crossing points and their extra counts
    uint32_t off_v, off_d, off_p;                    // shared-memory offsets
    FusedParams d;                                   // h, w, W, output, statistics, decision constants
};

__device__ __forceinline__ int back(int s, int k, int nr) // ring slot k rows above slot s (0 <= k < nr)
{
    return s >= k ? s - k : s - k + nr;
}

template <int CIN>
__device__ __forceinline__ uint32_t fetch(const GsParams &g, int row, int col)
{
    if ((unsigned)row >= (unsigned)g.d.h || (unsigned)col >= (unsigned)g.d.w)
        return 0u;
    const uint8_t *px = g.src + (long long)row * g.src_pitch + (long long)col * CIN;
    if (CIN == 1)
        return __ldg(px);
    return (uint32_t)__ldg(px) | ((uint32_t)__ldg(px + 1) << 8) | ((uint32_t)__ldg(px + 2) << 16);
}

template <int CIN>
__device__ __forceinline__ uint32_t to_gray(uint32_t v)
{
    if (CIN == 1)
        return v;
    // Eq. 1, integer round-half-up (the same rule as every other kernel)
    return (299u * (v & 0xffu) + 587u * ((v >> 8) & 0xffu) + 114u * (v >> 16) + 500u) / 1000u;
}

// Inclusive prefix sums of f and f^2 along one ring row: lane l covers span
// columns [16 l, 16 l + 16); P[i] = sums over columns 0..i.
__device__ __forceinline__ void prefix_row(const uint8_t *row, int sp, uint2 *P, int lane)
{
    uint32_t q[4] = {0u, 0u, 0u, 0u};
    if (16 * lane < sp) {
        const uint4 v = *reinterpret_cast<const uint4 *>(row + 16 * lane);
        q[0] = v.x;
        q[1] = v.y;
        q[2] = v.z;
        q[3] = v.w;
    }
    uint32_t s1[16], s2[16], a1 = 0u, a2 = 0u;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint32_t f = (q[i >> 2] >> (8 * (i & 3))) & 0xffu;
        a1 += f;
        a2 += f * f;
        s1[i] = a1;
        s2[i] = a2;
    }
    uint32_t e1 = a1, e2 = a2; // inclusive warp scan of the lane totals
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t u1 = __shfl_up_sync(0xffffffffu, e1, off);
        const uint32_t u2 = __shfl_up_sync(0xffffffffu, e2, off);
        if (lane >= off) {
            e1 += u1;
            e2 += u2;
        }
    }
    e1 -= a1; // exclusive
    e2 -= a2;
    uint4 *dst = reinterpret_cast<uint4 *>(P + 16 * lane);
#pragma unroll
    for (int i = 0; i < 8; ++i)
        dst[i] = make_uint4(e1 + s1[2 * i], e2 + s2[2 * i], e1 + s1[2 * i + 1], e2 + s2[2 * i + 1]);
}

template <int CIN, int RULE>
__global__ void __launch_bounds__(GT) gs_kernel(const __grid_constant__ GsParams g)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const FusedParams &p = g.d;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int x0 = blockIdx.x * GT, x = x0 + t;
    const int ya = blockIdx.y * g.seg_rows;
    const int yb = min(p.h, ya + g.seg_rows);
    const int a = g.a, b = g.b, mm = g.mm, W = p.W, nr = g.nr, span = g.span, sp = g.sp;
    const int cs = x0 + a - 1; // first span column
    const uint32_t lines = g.lines;
    uint8_t *ring = smem;
    uint2 *V = reinterpret_cast<uint2 *>(smem + g.off_v);
    uint2 *Dp = reinterpret_cast<uint2 *>(smem + g.off_d);
    uint2 *Dm = Dp + GT;
    uint2 *P = reinterpret_cast<uint2 *>(smem + g.off_p);

    for (int i = t; i < nr * sp / 16; i += GT)
        reinterpret_cast<uint4 *>(ring)[i] = make_uint4(0u, 0u, 0u, 0u);
    Dp[t] = make_uint2(0u, 0u);
    Dm[t] = make_uint2(0u, 0u);
    uint2 va = make_uint2(0u, 0u), vb = make_uint2(0u, 0u); // vertical sums of span columns t, t + GT

    // per-column constants of the output pixel (clipped line lengths)
    const bool xin = x < p.w;
    const int cnt_h = min(x + b, p.w - 1) - max(x + a, 0) + 1;
    const int cin_a = (unsigned)(x + a) < (unsigned)p.w, cin_b = (unsigned)(x + b) < (unsigned)p.w;

    const int y_first = ya - (W - 1); // entering row ya + a: the first row of the first output's window
    int es = (y_first + b) % nr;
    if (es < 0)
        es += nr;
    // the entering rows of the next kPF steps are in flight in registers (a
    // step is far shorter than a DRAM round trip)
    uint32_t r0[kPF], r1[kPF];
#pragma unroll
    for (int i = 0; i < kPF; ++i) {
        r0[i] = fetch<CIN>(g, y_first + b + i, cs + t);
        r1[i] = (t + GT < span) ? fetch<CIN>(g, y_first + b + i, cs + t + GT) : 0u;
    }
    uint32_t nfb = 0, nties = 0;
    __syncthreads();

    for (int y0 = y_first; y0 < yb; y0 += kPF) {
#pragma unroll
    for (int i = 0; i < kPF; ++i) {
        const int y = y0 + i;
        if (y >= yb) // uniform over the CTA
            break;
        const int e = y + b; // entering row
        uint8_t *re = ring + es * sp;
        re[t] = (uint8_t)to_gray<CIN>(r0[i]);
        if (t + GT < span)
            re[t + GT] = (uint8_t)to_gray<CIN>(r1[i]);
        if (y + kPF < yb) { // the entering row of step y + kPF
            r0[i] = fetch<CIN>(g, e + kPF, cs + t);
            if (t + GT < span)
                r1[i] = fetch<CIN>(g, e + kPF, cs + t + GT);
        }
        __syncthreads();

        const int ls = back(es, W, nr); // leaving row e - W
        const uint8_t *rl = ring + ls * sp;
        if (lines & (L_VC | L_FRAME)) {
            const uint32_t u = re[t], v = rl[t];
            va.x += u - v;
            va.y += u * u - v * v;
            V[t] = va;
            if (t + GT < span) {
                const uint32_t u2 = re[t + GT], v2 = rl[t + GT];
                vb.x += u2 - v2;
                vb.y += u2 * u2 - v2 * v2;
                V[t + GT] = vb;
            }
        }
        if (lines & L_DP) {
            const int s = (t - y) & (GT - 1);
            if (t != 0) { // continue the diagonal of (y - 1, x - 1)
                const uint32_t u = re[t + W], v = rl[t];
                uint2 d = Dp[s];
                d.x += u - v;
                d.y += u * u - v * v;
                Dp[s] = d;
            }
            if (warp == 0) { // the diagonal entering at the strip's first column: sum it afresh
                uint32_t s1 = 0u, s2 = 0u;
                for (int j = lane; j < W; j += 32) { // offset d = a + j: row y + d, span column j + 1
                    const uint32_t f = ring[back(es, W - 1 - j, nr) * sp + j + 1];
                    s1 += f;
                    s2 += f * f;
                }
                s1 = __reduce_add_sync(0xffffffffu, s1);
                s2 = __reduce_add_sync(0xffffffffu, s2);
                if (t == 0) // the slot of that column
                    Dp[s] = make_uint2(s1, s2);
            }
        }
        if (lines & L_DM) {
            const int s = (t + y) & (GT - 1);
            if (t != GT - 1) { // continue the anti-diagonal of (y - 1, x + 1)
                const uint8_t *rdl = ring + back(es, b + mm + 1, nr) * sp;
                const uint32_t u = re[t - mm - a + 1], v = rdl[t + W + 1];
                uint2 d = Dm[s];
                d.x += u - v;
                d.y += u * u - v * v;
                Dm[s] = d;
            }
            if (warp == GT / 32 - 1) { // the anti-diagonal entering at the strip's last column
                uint32_t s1 = 0u, s2 = 0u;
                for (int j = lane; j <= 2 * mm; j += 32) { // d = j - mm: row y + d, span column GT - d - a
                    const int d = j - mm;
                    const uint32_t f = ring[back(es, b - d, nr) * sp + GT - d - a];
                    s1 += f;
                    s2 += f * f;
                }
                s1 = __reduce_add_sync(0xffffffffu, s1);
                s2 = __reduce_add_sync(0xffffffffu, s2);
                if (t == GT - 1) // the slot of that column
                    Dm[s] = make_uint2(s1, s2);
            }
        }
        const bool out_row = y >= ya;
        if (out_row && warp < g.nh) { // row sums: prefix of row y (centre), y + a (frame top) or e (frame bottom)
            const int kb = (lines & L_HC) ? (warp == 0 ? b : (warp == 1 ? W - 1 : 0)) : (warp == 0 ? W - 1 : 0);
            prefix_row(ring + back(es, kb, nr) * sp, sp, P + warp * kPRow, lane);
        }
        __syncthreads();

        if (out_row && xin) {
            const int ys = back(es, b, nr); // row y
            const uint32_t f = ring[ys * sp + t - a + 1];
            uint32_t n = 0u, S1 = 0u, S2 = 0u;
            const int cnt_v = min(y + b, p.h - 1) - max(y + a, 0) + 1;
            int pr = 0;
            if (lines & L_HC) {
                const uint2 hi = P[t + W], lo = P[t];
                S1 += hi.x - lo.x;
                S2 += hi.y - lo.y;
                n += cnt_h;
                pr = 1;
            }
            if (lines & L_VC) {
                const uint2 v = V[t - a + 1];
                S1 += v.x;
                S2 += v.y;
                n += cnt_v;
            }
            if (lines & L_FRAME) {
                const uint2 th = P[pr * kPRow + t + W], tl = P[pr * kPRow + t];
                const uint2 bh = P[(pr + 1) * kPRow + t + W], bl = P[(pr + 1) * kPRow + t];
                const uint2 vl = V[t + 1], vr = V[t + W];
                S1 += (th.x - tl.x) + (bh.x - bl.x) + vl.x + vr.x;
                S2 += (th.y - tl.y) + (bh.y - bl.y) + vl.y + vr.y;
                n += ((unsigned)(y + a) < (unsigned)p.h ? cnt_h : 0) + ((unsigned)(y + b) < (unsigned)p.h ? cnt_h : 0) +
                     (cin_a ? cnt_v : 0) + (cin_b ? cnt_v : 0);
            }
            if (lines & L_DP) {
                const uint2 d = Dp[(t - y) & (GT - 1)];
                S1 += d.x;
                S2 += d.y;
                const int lo = max(a, max(-y, -x)), hi = min(b, min(p.h - 1 - y, p.w - 1 - x));
                n += max(0, hi - lo + 1);
            }
            if (lines & L_DM) {
                const uint2 d = Dm[(t + y) & (GT - 1)];
                S1 += d.x;
                S2 += d.y;
                const int lo = max(-mm, max(-y, x - (p.w - 1))), hi = min(mm, min(p.h - 1 - y, x));
                n += max(0, hi - lo + 1);
            }
            for (int c = 0; c < g.ncorr; ++c) { // crossing points counted more than once
                const int dy = g.cdy[c], dx = g.cdx[c], ex = g.cex[c];
                const uint32_t v = ring[back(es, b - dy, nr) * sp + t + dx - a + 1];
                S1 -= ex * v;
                S2 -= ex * v * v;
                if ((unsigned)(y + dy) < (unsigned)p.h && (unsigned)(x + dx) < (unsigned)p.w)
                    n -= ex;
            }
            const uint32_t r = decide_pixel<RULE>(f, n, S1, S2, p, nfb, nties);
            p.dst[(long long)y * p.dst_pitch + x] = (uint8_t)r;
        }
        es = es + 1 == nr ? 0 : es + 1;
    }
    }
    if (p.stats) {
        nfb = __reduce_add_sync(0xffffffffu, nfb);
        nties = __reduce_add_sync(0xffffffffu, nties);
        if (lane == 0 && (nfb | nties)) {
            atomicAdd(p.stats, (unsigned long long)nfb);
            atomicAdd(p.stats + 1, (unsigned long long)nties);
        }
    }
}

// Confusion counts of Eq. 6: TP, FP, FN, TN of `mask` against `ref`.
__global__ void __launch_bounds__(256) confusion_kernel(const uint8_t *mask, long long mp, uint32_t mink,
                                                        const uint8_t *ref, long long rp, uint32_t rink, int h,
                                                        int w, unsigned long long *counts)
{
    uint32_t c0 = 0, c1 = 0, c2 = 0;
    const long long total = (long long)h * w;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / w), x = (int)(i - (long long)y * w);
        const bool am = mask[(long long)y * mp + x] == mink;
        const bool br = ref[(long long)y * rp + x] == rink;
        c0 += am && br;
        c1 += am && !br;
        c2 += !am && br;
    }
    c0 = __reduce_add_sync(0xffffffffu, c0);
    c1 = __reduce_add_sync(0xffffffffu, c1);
    c2 = __reduce_add_sync(0xffffffffu, c2);
    __shared__ unsigned long long s[3];
    if (threadIdx.x < 3)
        s[threadIdx.x] = 0ull;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s[0], (unsigned long long)c0);
        atomicAdd(&s[1], (unsigned long long)c1);
        atomicAdd(&s[2], (unsigned long long)c2);
    }
    __syncthreads();
    if (threadIdx.x < 3 && s[threadIdx.x])
        atomicAdd(counts + threadIdx.x, s[threadIdx.x]);
}

struct Line {
    int kind; // 0 row dy = v, 1 column dx = v, 2 diagonal, 3 anti-diagonal
    int v;
};

// Lines of a structure, its L_* bits, and the crossing points with their extra counts.
int structure(int gs, int W, GsParams *g)
{
    const int a = -(W / 2), b = W - 1 - W / 2, mm = std::min(W / 2, W - 1 - W / 2);
    Line ls[8];
    int nl = 0;
    uint32_t bits = 0;
    const bool cross = gs == BNZ_GS_CROSS || gs == BNZ_GS_STAR || gs == BNZ_GS_FRAME_CROSS;
    const bool diag = gs == BNZ_GS_DIAGONALS || gs == BNZ_GS_STAR || gs == BNZ_GS_FRAME_DIAGONALS;
    const bool frame = gs == BNZ_GS_FRAME || gs == BNZ_GS_FRAME_CROSS || gs == BNZ_GS_FRAME_DIAGONALS;
    if (cross) {
        ls[nl++] = {0, 0};
        ls[nl++] = {1, 0};
        bits |= L_HC | L_VC;
    }
    if (diag) {
        ls[nl++] = {2, 0};
        ls[nl++] = {3, 0};
        bits |= L_DP | L_DM;
    }
    if (frame) {
        ls[nl++] = {0, a};
        ls[nl++] = {0, b};
        ls[nl++] = {1, a};
        ls[nl++] = {1, b};
        bits |= L_FRAME;
    }
    auto on = [&](const Line &l, int dy, int dx) {
        switch (l.kind) {
        case 0: return dy == l.v;
        case 1: return dx == l.v;
        case 2: return dy == dx;
        default: return dy == -dx && dy >= -mm && dy <= mm;
        }
    };
    g->a = a;
    g->b = b;
    g->mm = mm;
    g->lines = bits;
    g->nh = ((bits & L_HC) ? 1 : 0) + ((bits & L_FRAME) ? 2 : 0);
    g->ncorr = 0;
    for (int dy = a; dy <= b; ++dy)
        for (int dx = a; dx <= b; ++dx) {
            int c = 0;
            for (int i = 0; i < nl; ++i)
                c += on(ls[i], dy, dx) ? 1 : 0;
            if (c > 1) {
                if (g->ncorr == kMaxCorr)
                    return fail(BNZ_EINVAL, "structure %d: too many crossing points for W = %d", gs, W);
                g->cdy[g->ncorr] = dy;
                g->cdx[g->ncorr] = dx;
                g->cex[g->ncorr] = c - 1;
                ++g->ncorr;
            }
        }
    return BNZ_OK;
}

size_t round16(size_t v) { return (v + 15) / 16 * 16; }

template <int CIN, int RULE>
const void *kernel_fn()
{
    return reinterpret_cast<const void *>(&gs_kernel<CIN, RULE>);
}

std::once_flag g_attr_once[64];
int g_attr_rc[64];

int set_attributes(int dev)
{
    if (dev < 0 || dev >= 64)
        return fail(BNZ_ENODEV, "device ordinal %d out of range", dev);
    std::call_once(g_attr_once[dev], [dev] {
        int rc = BNZ_OK;
        const void *fns[4] = {kernel_fn<1, BNZ_SAUVOLA>(), kernel_fn<1, BNZ_NIBLACK>(), kernel_fn<3, BNZ_SAUVOLA>(),
                              kernel_fn<3, BNZ_NIBLACK>()};
        for (const void *fn : fns) {
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "cudaFuncSetAttribute(gs kernel)");
                break;
            }
        }
        g_attr_rc[dev] = rc;
    });
    return g_attr_rc[dev];
}

} // namespace

int launch_gs(const uint8_t *d_src, size_t src_pitch, int h, int w, int ch, int W, int gs, int rule, double k,
              double R, uint8_t *d_dst, size_t dst_pitch, unsigned long long *d_stats, cudaStream_t stream)
{
    GsParams g;
    memset(&g, 0, sizeof g);
    int rc = structure(gs, W, &g);
    if (rc != BNZ_OK)
        return rc;
    fill_decision_params(&g.d, h, w, W, rule, k, R);
    g.d.dst = d_dst;
    g.d.dst_pitch = (long long)dst_pitch;
    g.d.stats = d_stats;
    g.src = d_src;
    g.src_pitch = (long long)src_pitch;
    g.span = GT + W + 1;
    g.sp = (int)round16((size_t)g.span);
    g.nr = W + 1;
    size_t off = round16((size_t)g.nr * g.sp);
    g.off_v = (uint32_t)off;
    off = round16(off + (size_t)g.span * sizeof(uint2));
    g.off_d = (uint32_t)off;
    off += 2 * GT * sizeof(uint2);
    g.off_p = (uint32_t)off;
    off += (size_t)std::max(g.nh, 1) * kPRow * sizeof(uint2);
    const size_t smem = off;
    int dev = 0, occ = 0, sms = 0;
    rc = device_sm_count(&sms);
    if (rc != BNZ_OK)
        return rc;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    rc = set_attributes(dev);
    if (rc != BNZ_OK)
        return rc;
    const void *fn = ch == 1 ? (rule == BNZ_SAUVOLA ? kernel_fn<1, BNZ_SAUVOLA>() : kernel_fn<1, BNZ_NIBLACK>())
                             : (rule == BNZ_SAUVOLA ? kernel_fn<3, BNZ_SAUVOLA>() : kernel_fn<3, BNZ_NIBLACK>());
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, GT, smem);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(gs kernel)");
    if (occ < 1)
        return fail(BNZ_EINVAL, "reduced-set kernel does not fit an SM (W = %d, %zu bytes of shared memory)", W, smem);
    // segments: enough CTAs for every SM's resident slots, each at least 64 rows tall
    // (a segment's W - 1 rows of warm-up only add rows: no row sums, no decisions)
    const int strips = (w + GT - 1) / GT;
    const long long target = (long long)sms * occ;
    int segs = (int)std::min<long long>((target + strips - 1) / strips, (h + 63) / 64);
    segs = std::max(segs, 1);
    g.seg_rows = (h + segs - 1) / segs;
    segs = (h + g.seg_rows - 1) / g.seg_rows;
    void *args[] = {(void *)&g};
    e = cudaLaunchKernel(fn, dim3((unsigned)strips, (unsigned)segs), dim3(GT), args, smem, stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "reduced-set kernel launch");
    return BNZ_OK;
}

int launch_confusion(const uint8_t *d_mask, size_t mask_pitch, int mask_ink, const uint8_t *d_ref, size_t ref_pitch,
                     int ref_ink, int h, int w, unsigned long long *d_counts, cudaStream_t stream)
{
    int sms = 0;
    int rc = device_sm_count(&sms);
    if (rc != BNZ_OK)
        return rc;
    const long long total = (long long)h * w;
    const long long blocks = std::max<long long>(1, std::min<long long>((long long)sms * 8, (total + 255) / 256));
    confusion_kernel<<<(unsigned)blocks, 256, 0, stream>>>(d_mask, (long long)mask_pitch, (uint32_t)mask_ink, d_ref,
                                                           (long long)ref_pitch, (uint32_t)ref_ink, h, w, d_counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "confusion kernel launch");
    return BNZ_OK;
}

} // namespace bnz

extern "C" {

int bnz_gs_binarize_dev(const void *d_src, size_t src_pitch, int height, int width, int channels, int W, int gs,
                        int rule, double k, double R, void *d_dst, size_t dst_pitch, unsigned long long *d_stats,
                        void *stream)
{
    int rc = bnz::check_common(d_src, src_pitch, height, width, channels, W, rule, k, R, d_dst, dst_pitch, 0);
    if (rc != BNZ_OK)
        return rc;
    if (gs < BNZ_GS_CROSS || gs > BNZ_GS_FRAME_DIAGONALS)
        return bnz::fail(BNZ_EINVAL, "unknown structure %d (BNZ_GS_CROSS .. BNZ_GS_FRAME_DIAGONALS)", gs);
    if (W < 3)
        return bnz::fail(BNZ_EINVAL, "reduced sets need W >= 3 (got %d)", W);
    if (rule == BNZ_NIBLACK)
        R = 1.0;
    return bnz::launch_gs(static_cast<const uint8_t *>(d_src), src_pitch, height, width, channels, W, gs, rule, k, R,
                          static_cast<uint8_t *>(d_dst), dst_pitch, d_stats, static_cast<cudaStream_t>(stream));
}

int bnz_confusion_dev(const void *d_mask, size_t mask_pitch, int mask_ink, const void *d_ref, size_t ref_pitch,
                      int ref_ink, int height, int width, unsigned long long *d_counts, void *stream)
{
    if (!d_mask || !d_ref || !d_counts)
        return bnz::fail(BNZ_EINVAL, "null pointer");
    if (height < 0 || width < 0 || mask_pitch < (size_t)width || ref_pitch < (size_t)width)
        return bnz::fail(BNZ_EINVAL, "bad size or pitch");
    if (mask_ink < 0 || mask_ink > 255 || ref_ink < 0 || ref_ink > 255)
        return bnz::fail(BNZ_EINVAL, "ink values must be bytes");
    if (height == 0 || width == 0)
        return BNZ_OK;
    return bnz::launch_confusion(static_cast<const uint8_t *>(d_mask), mask_pitch, mask_ink,
                                 static_cast<const uint8_t *>(d_ref), ref_pitch, ref_ink, height, width, d_counts,
                                 static_cast<cudaStream_t>(stream));
}

} // extern "C"
