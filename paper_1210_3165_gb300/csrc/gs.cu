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

constexpr int GT = 256;    // threads of a CTA = output columns of a strip
constexpr int kPRow = 768; // entries of a prefix row: up to three 256-column parts (span <= 512 + 256)
constexpr int kPF = 2;     // entering rows loaded ahead

// The lines of a structure, as disjoint pieces where possible (frame sides
// and, with the frame, the centre row and column stop short of the frame):
//   HC     centre row: offsets [a, b] (cross, star) or (a, b) (frame + cross)
//   VFULL  centre column, rows [a, b] (cross, star)
//   DIAG   dy = dx over [a, b] and dy = -dx over [-mm, mm]
//   FRAME  rows a and b over [a, b]; columns a and b over rows (a, b)
//   VCUT   column sums over rows (a, b): the frame's sides, and the centre
//          column of frame + cross
// CENTRE: extra counts of the centre pixel (lines through it beyond the first).
// Frame + diagonals also counts the diagonals' four end points twice (they
// lie on the frame).
template <int GS>
struct Shape {
    static constexpr bool HC = GS == BNZ_GS_CROSS || GS == BNZ_GS_STAR || GS == BNZ_GS_FRAME_CROSS;
    static constexpr bool HC_CUT = GS == BNZ_GS_FRAME_CROSS;
    static constexpr bool VFULL = GS == BNZ_GS_CROSS || GS == BNZ_GS_STAR;
    static constexpr bool DIAG = GS == BNZ_GS_DIAGONALS || GS == BNZ_GS_STAR || GS == BNZ_GS_FRAME_DIAGONALS;
    static constexpr bool FRAME = GS >= BNZ_GS_FRAME;
    static constexpr bool VCUT = FRAME;
    static constexpr bool ENDS = GS == BNZ_GS_FRAME_DIAGONALS;
    static constexpr int NH = (HC ? 1 : 0) + (FRAME ? 2 : 0); // prefix rows per output row
    static constexpr int CENTRE = GS == BNZ_GS_STAR ? 3 : (GS == BNZ_GS_FRAME ? 0 : 1);
};

struct GsParams {
    const uint8_t *src;
    long long src_pitch;
    int a, b, mm;     // window offsets [a, b]; anti-diagonal offsets |d| <= mm
    int span, sp, nr; // span columns (GT + W + 1), their padded bytes, ring rows (W + 1)
    int seg_rows;     // output rows per CTA
    int small;        // |S'|^2 * 255^2 < 2^32: the variance numerator fits 32 bits
    uint32_t off_v, off_d, off_p; // shared-memory offsets
    FusedParams d;    // h, w, W, output, statistics, decision constants (nW = |S'|)
};

__device__ __forceinline__ int back(int s, int k, int nr) // ring slot k rows above slot s (0 <= k < nr)
{
    return s >= k ? s - k : s - k + nr;
}

__device__ __forceinline__ int clip_len(int lo, int hi, int n) // |[lo, hi] within [0, n)|
{
    return max(0, min(hi, n - 1) - max(lo, 0) + 1);
}

// The raw bytes of one span column of a row (zero outside the page), each in
// its own register: they are combined only when the row is used, kPF steps
// later, so the loads stay in flight meanwhile.
template <int CIN>
__device__ __forceinline__ void fetch(const GsParams &g, int row, int col, uint32_t (&v)[CIN])
{
    const bool in = (unsigned)row < (unsigned)g.d.h && (unsigned)col < (unsigned)g.d.w;
    const uint8_t *px = g.src + (long long)row * g.src_pitch + (long long)col * CIN;
#pragma unroll
    for (int c = 0; c < CIN; ++c)
        v[c] = in ? (uint32_t)__ldg(px + c) : 0u;
}

// Eq. 1, integer round-half-up (the same rule as every other kernel)
template <int CIN>
__device__ __forceinline__ uint32_t to_gray(const uint32_t (&v)[CIN])
{
    if (CIN == 1)
        return v[0];
    return (299u * v[0] + 587u * v[1 % CIN] + 114u * v[2 % CIN] + 500u) / 1000u;
}

// Inclusive prefix sums of f and f^2 over one half (256 span columns) of a
// ring row: lane l covers columns [256 hf + 8 l, +8).  Each half is summed on
// its own: a reader adds the first half's total P[255] to entries >= 256.
__device__ __forceinline__ void prefix_half(const uint8_t *row, int sp, uint2 *P, int hf, int lane)
{
    const int c0 = 256 * hf + 8 * lane;
    uint2 q = make_uint2(0u, 0u);
    if (c0 < sp)
        q = *reinterpret_cast<const uint2 *>(row + c0);
    uint32_t s1[8], s2[8], a1 = 0u, a2 = 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t f = ((i < 4 ? q.x : q.y) >> (8 * (i & 3))) & 0xffu;
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
    uint4 *dst = reinterpret_cast<uint4 *>(P + c0);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        dst[i] = make_uint4(e1 + s1[2 * i], e2 + s2[2 * i], e1 + s1[2 * i + 1], e2 + s2[2 * i + 1]);
}

// Sums over span columns (i0, i1] of a prefix row written in 256-column
// parts, each summed on its own: the totals of the parts between are added.
__device__ __forceinline__ uint2 seg(const uint2 *P, int i0, int i1)
{
    const uint2 hi = P[i1], lo = P[i0];
    uint2 r = make_uint2(hi.x - lo.x, hi.y - lo.y);
    if (i1 >= 256 && i0 < 256) {
        const uint2 t = P[255];
        r.x += t.x;
        r.y += t.y;
    }
    if (i1 >= 512 && i0 < 512) {
        const uint2 t = P[511];
        r.x += t.x;
        r.y += t.y;
    }
    return r;
}

// Eq. 3 on t' past the fp32 filter: the double-float and fp64 stages, out of
// line (a few pixels per page reach them).
template <int RULE>
__device__ __noinline__ uint32_t gs_decide_exact(uint32_t f, uint32_t n, uint32_t S1, uint32_t S2,
                                                 const FusedParams &p)
{
    return decide_exact<RULE>(f, n, S1, S2, p);
}

// Eq. 3 on t' for one pixel: the fp32 filter with the constants for n = |S'|
// when the structure lies whole in the page, with 1/n from rcp.approx
// otherwise (the margin of decision_margin covers both); small: every
// n S2 < 2^32, so V is formed and converted in 32 bits.
template <int RULE>
__device__ __forceinline__ uint32_t gs_decide(uint32_t f, uint32_t n, uint32_t S1, uint32_t S2, bool whole, int small,
                                              const FusedParams &p, uint32_t &nfb, uint32_t &nties)
{
    float vf;
    if (small)
        vf = __uint2float_rn(n * S2 - S1 * S1);
    else
        vf = v_to_float((unsigned long long)n * S2 - (unsigned long long)S1 * S1);
    const float sq = sqrt_approx(vf);
    const float ff = __uint2float_rn(f), S1f = __uint2float_rn(S1);
    const float d = whole ? filter_int<RULE>(ff, S1f, sq, p)
                          : filter_n<RULE>(ff, S1f, sq, rcp_approx(__uint2float_rn(n)), p);
    if (fabsf(d) >= p.E)
        return d < 0.0f ? 0u : 255u;
    const uint32_t r = gs_decide_exact<RULE>(f, n, S1, S2, p);
    ++nfb;
    nties += (r >> 9) & 1u;
    return r & 0xffu;
}

// CPT output columns per thread (strip = CPT x 256 columns): column c of the
// strip is handled by thread c mod 256.
template <int CIN, int RULE, int GS, int CPT>
__global__ void __launch_bounds__(GT, CPT == 1 ? 4 : 3) gs_kernel(const __grid_constant__ GsParams g)
{
    using S = Shape<GS>;
    constexpr int TWS = CPT * GT;  // strip width
    constexpr int NQ = CPT + 1;    // span columns per thread (the span is at most TWS + 256)
    constexpr int NPART = CPT + 1; // 256-column parts of a prefix row
    extern __shared__ __align__(16) uint8_t smem[];
    const FusedParams &p = g.d;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int x0 = blockIdx.x * TWS;
    const int ya = blockIdx.y * g.seg_rows;
    const int yb = min(p.h, ya + g.seg_rows);
    const int a = g.a, b = g.b, mm = g.mm, W = p.W, nr = g.nr, span = g.span, sp = g.sp;
    const int cs = x0 + a - 1; // first span column
    uint8_t *ring = smem;
    uint2 *V = reinterpret_cast<uint2 *>(smem + g.off_v); // column sums of every span column (W or W - 2 rows)
    uint2 *Dp = reinterpret_cast<uint2 *>(smem + g.off_d);
    uint2 *Dm = Dp + TWS;
    uint2 *P = reinterpret_cast<uint2 *>(smem + g.off_p);

    for (int i = t; i < nr * sp / 16; i += GT)
        reinterpret_cast<uint4 *>(ring)[i] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int h = 0; h < CPT; ++h) {
        Dp[t + h * GT] = make_uint2(0u, 0u);
        Dm[t + h * GT] = make_uint2(0u, 0u);
    }
    uint2 vs[NQ]; // column sums of span columns t + q * 256
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        vs[q] = make_uint2(0u, 0u);

    const int y_first = ya - (W - 1); // entering row ya + a: the first row of the first output's window
    int es = (y_first + b) % nr;
    if (es < 0)
        es += nr;
    // the entering rows of the next kPF steps are in flight in registers (a
    // step is far shorter than a DRAM round trip)
    uint32_t rr[kPF][NQ][CIN];
#pragma unroll
    for (int i = 0; i < kPF; ++i)
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            fetch<CIN>(g, y_first + b + i, t + q * GT < span ? cs + t + q * GT : -1, rr[i][q]);
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
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            if (t + q * GT < span) {
                re[t + q * GT] = (uint8_t)to_gray<CIN>(rr[i][q]);
                if (y + kPF < yb) // the entering row of step y + kPF
                    fetch<CIN>(g, e + kPF, cs + t + q * GT, rr[i][q]);
            }
        __syncthreads();

        if (S::VFULL || S::VCUT) { // rows [y + a, y + b] (entering e, leaving e - W) or (y + a, y + b)
            const uint8_t *ri = S::VFULL ? re : ring + back(es, 1, nr) * sp;
            const uint8_t *ro = ring + back(es, S::VFULL ? W : W - 1, nr) * sp;
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (t + q * GT < span) {
                    const uint32_t u = ri[t + q * GT], v = ro[t + q * GT];
                    vs[q].x += u - v;
                    vs[q].y += u * u - v * v;
                    V[t + q * GT] = vs[q];
                }
        }
        if (S::DIAG) {
            const uint8_t *rl = ring + back(es, W, nr) * sp; // row y + a - 1
            const uint8_t *rdl = ring + back(es, b + mm + 1, nr) * sp;
#pragma unroll
            for (int h = 0; h < CPT; ++h) {
                const int c = t + h * GT;
                if (c != 0) { // continue the diagonal of (y - 1, x - 1)
                    const int s = (c - y) & (TWS - 1);
                    const uint32_t u = re[c + W], v = rl[c];
                    uint2 d = Dp[s];
                    d.x += u - v;
                    d.y += u * u - v * v;
                    Dp[s] = d;
                }
                if (c != TWS - 1) { // continue the anti-diagonal of (y - 1, x + 1)
                    const int sm = (c + y) & (TWS - 1);
                    const uint32_t u = re[c - mm - a + 1], v = rdl[c + W + 1];
                    uint2 d = Dm[sm];
                    d.x += u - v;
                    d.y += u * u - v * v;
                    Dm[sm] = d;
                }
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
                    Dp[(0 - y) & (TWS - 1)] = make_uint2(s1, s2);
            }
            if (warp == GT / 32 - 1) { // the anti-diagonal entering at the strip's last column
                uint32_t s1 = 0u, s2 = 0u;
                for (int j = lane; j <= 2 * mm; j += 32) { // d = j - mm: row y + d, span column TWS - d - a
                    const int d = j - mm;
                    const uint32_t f = ring[back(es, b - d, nr) * sp + TWS - d - a];
                    s1 += f;
                    s2 += f * f;
                }
                s1 = __reduce_add_sync(0xffffffffu, s1);
                s2 = __reduce_add_sync(0xffffffffu, s2);
                if (t == GT - 1) // the slot of that column
                    Dm[(TWS - 1 + y) & (TWS - 1)] = make_uint2(s1, s2);
            }
        }
        const bool out_row = y >= ya;
        if (S::NH > 0 && out_row) {
            // prefix rows in 256-column parts, one warp per part: centre row y (back b), frame top y + a
            // (back W - 1), frame bottom e (back 0)
            for (int task = warp; task < S::NH * NPART; task += GT / 32) {
                const int j = task / NPART;
                const int kb = S::HC ? (j == 0 ? b : (j == 1 ? W - 1 : 0)) : (j == 0 ? W - 1 : 0);
                prefix_half(ring + back(es, kb, nr) * sp, sp, P + j * kPRow, task - j * NPART, lane);
            }
        }
        __syncthreads();

        if (out_row) {
            const uint8_t *rc = ring + back(es, b, nr) * sp; // row y
            const bool y_inner = y + a >= 0 && y + b < p.h;
            const bool ra = (unsigned)(y + a) < (unsigned)p.h, rb = (unsigned)(y + b) < (unsigned)p.h;
#pragma unroll
            for (int h = 0; h < CPT; ++h) {
                const int c = t + h * GT, x = x0 + c;
                if (x >= p.w)
                    break;
                const uint32_t f = rc[c - a + 1];
                uint32_t S1 = 0u, S2 = 0u;
                int pr = 0;
                if (S::HC) { // span columns of x + a .. x + b are c + 1 .. c + W
                    const uint2 hs = S::HC_CUT ? seg(P, c + 1, c + W - 1) : seg(P, c, c + W);
                    S1 += hs.x;
                    S2 += hs.y;
                    pr = 1;
                }
                if (S::VFULL || S::HC_CUT) { // centre column
                    const uint2 v = V[c - a + 1];
                    S1 += v.x;
                    S2 += v.y;
                }
                if (S::FRAME) {
                    const uint2 top = seg(P + pr * kPRow, c, c + W), bot = seg(P + (pr + 1) * kPRow, c, c + W);
                    const uint2 vl = V[c + 1], vr = V[c + W];
                    S1 += top.x + bot.x + vl.x + vr.x;
                    S2 += top.y + bot.y + vl.y + vr.y;
                }
                if (S::DIAG) {
                    const uint2 d = Dp[(c - y) & (TWS - 1)], m = Dm[(c + y) & (TWS - 1)];
                    S1 += d.x + m.x;
                    S2 += d.y + m.y;
                }
                S1 -= S::CENTRE * f;
                S2 -= S::CENTRE * f * f;
                const bool x_inner = x + a >= 0 && x + b < p.w;
                const bool cin_a = (unsigned)(x + a) < (unsigned)p.w, cin_b = (unsigned)(x + b) < (unsigned)p.w;
                int nends = 0;
                if (S::ENDS) { // the diagonals' end points, also on the frame
                    const uint2 *Pt = P + pr * kPRow, *Pb = P + (pr + 1) * kPRow;
                    const uint2 e0 = seg(Pt, c, c + 1);          // (a, a)
                    const uint2 e1 = seg(Pb, c + W - 1, c + W);  // (b, b)
                    uint2 e2, e3;
                    if (mm == b && a == -b) {                    // odd W: (a, b) and (b, a)
                        e2 = seg(Pt, c + W - 1, c + W);
                        e3 = seg(Pb, c, c + 1);
                    } else {                                     // even W: (-b, b) on column b, (b, -b) on row b
                        const uint32_t v = ring[back(es, 2 * b, nr) * sp + c + W];
                        e2 = make_uint2(v, v * v);
                        e3 = seg(Pb, c + 1, c + 2);
                    }
                    S1 -= e0.x + e1.x + e2.x + e3.x;
                    S2 -= e0.y + e1.y + e2.y + e3.y;
                    if (!(x_inner && y_inner)) {
                        const int ye = mm == b && a == -b ? a : -b, xe = -ye; // the anti-diagonal's upper end
                        nends = (ra && cin_a) + (rb && cin_b) +
                                ((unsigned)(y + ye) < (unsigned)p.h && (unsigned)(x + xe) < (unsigned)p.w) +
                                ((unsigned)(y - ye) < (unsigned)p.h && (unsigned)(x - xe) < (unsigned)p.w);
                    }
                }
                uint32_t n;
                const bool whole = x_inner && y_inner;
                if (whole) {
                    n = p.nW; // the whole structure inside the page: |S'|
                } else {
                    const int cnt_h = clip_len(x + a, x + b, p.w), cnt_hc = clip_len(x + a + 1, x + b - 1, p.w);
                    const int cnt_v = clip_len(y + a, y + b, p.h), cnt_vc = clip_len(y + a + 1, y + b - 1, p.h);
                    int cnt = 0;
                    if (S::HC)
                        cnt += S::HC_CUT ? cnt_hc : cnt_h;
                    if (S::VFULL)
                        cnt += cnt_v;
                    if (S::HC_CUT)
                        cnt += cnt_vc;
                    if (S::FRAME)
                        cnt += (ra ? cnt_h : 0) + (rb ? cnt_h : 0) + (cin_a ? cnt_vc : 0) + (cin_b ? cnt_vc : 0);
                    if (S::DIAG) {
                        cnt += max(0, min(b, min(p.h - 1 - y, p.w - 1 - x)) - max(a, max(-y, -x)) + 1);
                        cnt += max(0, min(mm, min(p.h - 1 - y, x)) - max(-mm, max(-y, x - (p.w - 1))) + 1);
                    }
                    n = (uint32_t)(cnt - S::CENTRE - nends);
                }
                const uint32_t r = gs_decide<RULE>(f, n, S1, S2, whole, g.small, p, nfb, nties);
                p.dst[(long long)y * p.dst_pitch + x] = (uint8_t)r;
            }
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

// |S'|: the structure's offsets in the W x W window (the definition, counted).
int structure_size(int gs, int W)
{
    const int a = -(W / 2), b = W - 1 - W / 2;
    int n = 0;
    for (int dy = a; dy <= b; ++dy)
        for (int dx = a; dx <= b; ++dx) {
            const bool cross = dy == 0 || dx == 0;
            const bool diag = dy == dx || dy == -dx;
            const bool frame = dy == a || dy == b || dx == a || dx == b;
            bool in = false;
            switch (gs) {
            case BNZ_GS_CROSS: in = cross; break;
            case BNZ_GS_DIAGONALS: in = diag; break;
            case BNZ_GS_STAR: in = cross || diag; break;
            case BNZ_GS_FRAME: in = frame; break;
            case BNZ_GS_FRAME_CROSS: in = frame || cross; break;
            default: in = frame || diag; break;
            }
            n += in ? 1 : 0;
        }
    return n;
}

size_t round16(size_t v) { return (v + 15) / 16 * 16; }

template <int CIN, int RULE, int CPT>
const void *kernel_fn(int gs)
{
    switch (gs) {
    case BNZ_GS_CROSS: return reinterpret_cast<const void *>(&gs_kernel<CIN, RULE, BNZ_GS_CROSS, CPT>);
    case BNZ_GS_DIAGONALS: return reinterpret_cast<const void *>(&gs_kernel<CIN, RULE, BNZ_GS_DIAGONALS, CPT>);
    case BNZ_GS_STAR: return reinterpret_cast<const void *>(&gs_kernel<CIN, RULE, BNZ_GS_STAR, CPT>);
    case BNZ_GS_FRAME: return reinterpret_cast<const void *>(&gs_kernel<CIN, RULE, BNZ_GS_FRAME, CPT>);
    case BNZ_GS_FRAME_CROSS: return reinterpret_cast<const void *>(&gs_kernel<CIN, RULE, BNZ_GS_FRAME_CROSS, CPT>);
    default: return reinterpret_cast<const void *>(&gs_kernel<CIN, RULE, BNZ_GS_FRAME_DIAGONALS, CPT>);
    }
}

template <int CPT>
const void *kernel_cpt(int ch, int rule, int gs)
{
    if (ch == 1)
        return rule == BNZ_SAUVOLA ? kernel_fn<1, BNZ_SAUVOLA, CPT>(gs) : kernel_fn<1, BNZ_NIBLACK, CPT>(gs);
    return rule == BNZ_SAUVOLA ? kernel_fn<3, BNZ_SAUVOLA, CPT>(gs) : kernel_fn<3, BNZ_NIBLACK, CPT>(gs);
}

const void *kernel_for(int ch, int rule, int gs, int cpt)
{
    return cpt == 2 ? kernel_cpt<2>(ch, rule, gs) : kernel_cpt<1>(ch, rule, gs);
}

// Two output columns per thread (512-column strips) halve the per-step work
// that does not depend on the column (the barriers, the ring and slot
// bookkeeping, the warp sums of the diagonals entering the strip); measured on
// 4096^2 RGB pages it pays for the structures with diagonals up to W = 128
// (15-25 % faster) and not for the others (0-4 % slower), whose wider span
// costs shared memory that 256-column strips keep for more CTAs.
constexpr int kCpt2MaxW = 128;

int columns_per_thread(int gs, int W)
{
    const bool diag = gs == BNZ_GS_DIAGONALS || gs == BNZ_GS_STAR || gs == BNZ_GS_FRAME_DIAGONALS;
    return diag && W <= kCpt2MaxW ? 2 : 1;
}

std::once_flag g_attr_once[64];
int g_attr_rc[64];

int set_attributes(int dev)
{
    if (dev < 0 || dev >= 64)
        return fail(BNZ_ENODEV, "device ordinal %d out of range", dev);
    std::call_once(g_attr_once[dev], [dev] {
        int rc = BNZ_OK;
        for (int ch : {1, 3})
            for (int rule : {BNZ_SAUVOLA, BNZ_NIBLACK})
                for (int gs = BNZ_GS_CROSS; gs <= BNZ_GS_FRAME_DIAGONALS; ++gs)
                    for (int cpt = 1; cpt <= 2 && rc == BNZ_OK; ++cpt) {
                        cudaError_t e = cudaFuncSetAttribute(kernel_for(ch, rule, gs, cpt),
                                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
                        if (e != cudaSuccess)
                            rc = cuda_fail(e, "cudaFuncSetAttribute(gs kernel)");
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
    g.a = -(W / 2);
    g.b = W - 1 - W / 2;
    g.mm = std::min(W / 2, W - 1 - W / 2);
    const bool hc = gs == BNZ_GS_CROSS || gs == BNZ_GS_STAR || gs == BNZ_GS_FRAME_CROSS;
    const int nh = (hc ? 1 : 0) + (gs >= BNZ_GS_FRAME ? 2 : 0);
    fill_decision_params(&g.d, h, w, W, rule, k, R);
    // the fp32 filter's constants for the unclipped structure, n = |S'|
    const double n = (double)structure_size(gs, W);
    g.d.nW = (uint32_t)n;
    g.small = n <= 256.0 ? 1 : 0;
    g.d.omkn = (float)((1.0 - k) / n);
    g.d.kRn2 = (float)(k / (R * n * n));
    g.d.invn = (float)(1.0 / n);
    g.d.kn = (float)(k / n);
    g.d.dst = d_dst;
    g.d.dst_pitch = (long long)dst_pitch;
    g.d.stats = d_stats;
    g.src = d_src;
    g.src_pitch = (long long)src_pitch;
    const int cpt = columns_per_thread(gs, W);
    const int tws = cpt * GT;
    g.span = tws + W + 1;
    g.sp = (int)round16((size_t)g.span);
    g.nr = W + 1;
    size_t off = round16((size_t)g.nr * g.sp);
    g.off_v = (uint32_t)off;
    off = round16(off + (size_t)g.span * sizeof(uint2));
    g.off_d = (uint32_t)off;
    off += 2 * (size_t)tws * sizeof(uint2);
    g.off_p = (uint32_t)off;
    off += (size_t)std::max(nh, 1) * kPRow * sizeof(uint2);
    const size_t smem = off;
    int dev = 0, occ = 0, sms = 0, rc = BNZ_OK;
    rc = device_sm_count(&sms);
    if (rc != BNZ_OK)
        return rc;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    rc = set_attributes(dev);
    if (rc != BNZ_OK)
        return rc;
    const void *fn = kernel_for(ch, rule, gs, cpt);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, GT, smem);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(gs kernel)");
    if (occ < 1)
        return fail(BNZ_EINVAL, "reduced-set kernel does not fit an SM (W = %d, %zu bytes of shared memory)", W, smem);
    // segments: as many CTAs as the SMs hold at once (one wave: a second,
    // partial wave would double the time), each at least 64 rows tall (a
    // segment's W - 1 rows of warm-up only add rows: no row sums, no decisions)
    const int strips = (w + tws - 1) / tws;
    const long long target = (long long)sms * occ;
    int segs = (int)std::min<long long>(target / strips, (h + 63) / 64);
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
