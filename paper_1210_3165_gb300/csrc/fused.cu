// fused.cu -- the fused tile kernel for exact Sauvola / Niblack binarization.
//
// One persistent CTA walks a contiguous range of "strip rows": the image is
// cut into vertical strips of 512 output columns, the strips are laid end to
// end (strip-major), and the total is split evenly over the grid.  For each
// run of rows it owns in a strip the CTA
//   a1  loads the strip plus its halo (W-1 columns, 16-aligned on the left)
//       row-chunk by row-chunk with 2-D TMA boxes into a shared-memory ring
//       that holds the last W + 2*chunk rows, so every input byte comes from
//       global memory once per strip;
//   a2  for RGB input converts each chunk to gray in shared memory with the
//       integer rule of Eq. 1, f = (299 r + 587 g + 114 b + 500) / 1000
//       (two byte dot products and a multiply-high per pixel);
//   a3  keeps exact column sums c1 = sum f and c2 = sum f^2 over the W window
//       rows in registers (4 columns per thread), publishes them for the
//       current row, then adds the entering row and drops the leaving one;
//   a4  forms the horizontal window sums S1, S2 from the published column
//       sums: each lane slides over 16 consecutive outputs (128-bit loads,
//       realigned at compile time), the lanes' partial sums are joined with a
//       warp scan, and a warp reduction gives the first window of the row;
//   a5  takes n = W*W for windows inside the image and the clipped count at
//       the borders;
//   a6  decides f < t (Eq. 3) for Sauvola (Eq. 4) or Niblack with an fp32
//       filter whose error is bounded (decision_margin); pixels inside the
//       bound re-run the fp64 sequence m = S1/n, s = sqrt(V)/n, t = ..., so
//       every output equals that fp64 decision;
//   a7  writes the byte mask {0,255} or the packed 1-bit mask.
// The sums are never rounded: S1 < 2^24 and S2 < 2^32 for W <= 255, and
// V = n*S2 - S1^2 is formed in 64-bit integers.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>

#include "internal.h"
#include "ptx.cuh"

namespace bnz {
namespace {

constexpr int NT = 256;
constexpr int NWARP = NT / 32;
constexpr int L = 16;  // outputs per lane per row; a strip is 32 * L = 512 columns wide
constexpr int TW = 32 * L; // widest strip; 256 is used when the ring would not fit
constexpr int MAX_DYN_SMEM = 232448 - 1024; // 227 KB opt-in limit, minus slack

template <int CIN>
struct PanelWidth;
template <>
struct PanelWidth<1> {
    static constexpr int PWP = 128; // one 128-byte TMA box per panel
};
template <>
struct PanelWidth<3> {
    static constexpr int PWP = 80; // 240-byte boxes: whole r,g,b triples
};

__device__ __forceinline__ uint32_t byte_of(uint32_t w, int k)
{
    return (w >> (8 * k)) & 0xffu;
}

// Position of span column c in a column-sum row: 4 words of padding after
// every 16 columns keep the lanes' 128-bit loads free of bank conflicts.
__device__ __forceinline__ int cpos(int c)
{
    return c + ((c >> 4) << 2);
}

// exact uint -> float for v < 2^23: 2^23 + v has v in its mantissa
__device__ __forceinline__ float u23_to_float(uint32_t v)
{
    return __fsub_rn(__uint_as_float(v | 0x4B000000u), 8388608.0f);
}

// byte J of `word` as an exact float (same trick, byte moved by a permute)
template <int J>
__device__ __forceinline__ float byte_to_float(uint32_t word)
{
    return __fsub_rn(__uint_as_float(__byte_perm(word, 0x4B000000u, 0x7440u | J)), 8388608.0f);
}

// PTX prmt (default mode): a selector nibble with bit 3 set yields the sign
// of the selected byte replicated over the result byte.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
    return r;
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// V (< 2^48) as float: high word exact, low word rounded, one more rounding
// in the fma -- relative error <= 2u (u = 2^-24); no 64-bit conversion, which
// would run on the fp64 pipe.
__device__ __forceinline__ float v_to_float(unsigned long long V)
{
    return __fmaf_rn(__uint2float_rn((uint32_t)(V >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)V));
}

// Eq. 1 for one pixel whose r, g, b are bytes 0..2 of px (byte 3 ignored):
// x = 299 r + 587 g + 114 b + 500 = (43 r + 75 g + 114 b) + 256 (r + 2 g) + 500,
// q = floor(x / 1000) = high word of x * ceil(2^32 / 1000) (exact for x < 6.1e6).
__device__ __forceinline__ uint32_t gray1(uint32_t px)
{
    const uint32_t hi = __dp4a(px, 0x00000201u, 0u);
    const uint32_t x = __dp4a(px, 0x00724B2Bu, hi * 256u + 500u);
    return __umulhi(x, 4294968u);
}

// Four gray pixels from 12 interleaved bytes r0 g0 b0 r1 | g1 b1 r2 g2 | b2 r3 g3 b3.
__device__ __forceinline__ uint32_t gray4(uint32_t w0, uint32_t w1, uint32_t w2)
{
    const uint32_t g0 = gray1(w0);
    const uint32_t g1 = gray1(__funnelshift_r(w0, w1, 24));
    const uint32_t g2 = gray1(__funnelshift_r(w1, w2, 16));
    const uint32_t g3 = gray1(w2 >> 8);
    return g0 | (g1 << 8) | (g2 << 16) | (g3 << 24);
}

// fp32 filter value d ~ f - t for a window of n = W*W pixels.
template <int RULE>
__device__ __forceinline__ float filter_d(float ff, float S1f, float sq, const FusedParams &p)
{
    if (RULE == BNZ_SAUVOLA)
        return __fmaf_rn(-S1f, __fmaf_rn(p.kRn2, sq, p.omkn), ff);
    return __fmaf_rn(-p.kn, sq, __fmaf_rn(-p.invn, S1f, ff));
}

// Exact decision for one pixel whose window may be clipped or whose fp32
// value fell inside the margin.  Returns g | 0x100 (fp64 used) | 0x200 (tie).
template <int RULE>
__device__ __noinline__ uint32_t slow_decide(uint32_t f, uint32_t S1, uint32_t S2, int y, int xg,
                                             const FusedParams &p)
{
    const int nr = min(y + p.r_hi, p.h - 1) - max(y - p.r_lo, 0) + 1;
    const int nc = min(xg + p.r_hi, p.w - 1) - max(xg - p.r_lo, 0) + 1;
    const uint32_t n = (uint32_t)(nr * nc);
    const unsigned long long V = (unsigned long long)n * S2 - (unsigned long long)S1 * S1;
    const float sq = sqrt_approx(v_to_float(V));
    const float invn = __frcp_rn(__uint2float_rn(n));
    const float S1f = __uint2float_rn(S1), ff = __uint2float_rn(f);
    float d;
    if (RULE == BNZ_SAUVOLA) {
        const float a = __fmul_rn(p.omk, invn);
        const float b = __fmul_rn(__fmul_rn(p.kR, invn), invn);
        d = __fmaf_rn(-S1f, __fmaf_rn(b, sq, a), ff);
    } else {
        d = __fmaf_rn(-__fmul_rn(p.kf, invn), sq, __fmaf_rn(-invn, S1f, ff));
    }
    if (fabsf(d) >= p.E)
        return d < 0.0f ? 0u : 255u;
    // the fp64 sequence of the definition, same order, no contraction
    const double nd = (double)n;
    const double md = __ddiv_rn((double)S1, nd);
    const double sd = __ddiv_rn(__dsqrt_rn(__ull2double_rn(V)), nd);
    double td;
    if (RULE == BNZ_SAUVOLA)
        td = __dmul_rn(md, __dadd_rn(1.0, __dmul_rn(p.k, __dsub_rn(__ddiv_rn(sd, p.R), 1.0))));
    else
        td = __dadd_rn(md, __dmul_rn(p.k, sd));
    const double fd = (double)f;
    const uint32_t tie = fabs(__dsub_rn(fd, td)) < 1e-9 ? 0x200u : 0u;
    return (fd < td ? 0u : 255u) | 0x100u | tie;
}

// 16-byte load of 4 column sums (group a = columns 4a..4a+3)
__device__ __forceinline__ uint4 ld_group(const uint32_t *C, int a)
{
    return *reinterpret_cast<const uint4 *>(C + 4 * a + ((a >> 2) << 2));
}

template <int CIN, int RULE, int WM8>
__global__ void __launch_bounds__(NT, 1)
    fused_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ FusedParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr int PWP = PanelWidth<CIN>::PWP;
    constexpr int PWB = PWP * CIN;
    // o = (-r_lo) mod 16 and r_lo = W/2, so the misalignments of the leaving
    // (span column o + x) and entering (o + W + x) streams are fixed by W mod 8
    constexpr int KO = (4 - ((WM8 >> 1) & 3)) & 3;
    constexpr int KI = (KO + WM8) & 3;

    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    uint8_t *ring = smem + p.off_ring;
    uint8_t *stage = smem + p.off_stage;
    uint32_t *cb1 = reinterpret_cast<uint32_t *>(smem + p.off_c1);
    uint32_t *cb2 = reinterpret_cast<uint32_t *>(smem + p.off_c2);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int CH = p.CH;
    const int W = p.W;
    const int D = (CH + W - 1) / CH; // chunks ahead of the current one that its outputs need
    const int nbar = CIN == 1 ? p.NS : p.NSS;
    const uint32_t chunk_bytes = (uint32_t)(p.NPAN * CH * PWB);
    const int ng = p.SWP >> 2;
    const long long limit = p.timeout_cycles;

    if (tid == 0) {
        for (int i = 0; i < nbar; ++i)
            mbar_init(&bars[i], 1);
        fence_mbar_init();
        fence_proxy_async_smem();
        prefetch_tmap(&tmap);
    }
    __syncthreads();

    uint64_t phase = 0; // bit i: parity to wait for next on barrier i (uniform)
    uint32_t nfb = 0, nties = 0;
    bool ok = true;

    // column-owner geometry (a3): 4 consecutive span columns per thread
    const bool owner = tid < ng;
    const int gcol = tid * 4;
    const int gpn = gcol / PWP, gip = gcol - gpn * PWP;
    const int gpos = cpos(gcol);

    // centre-pixel geometry (a6): the lane's 16 outputs start at span column
    // lane*16 + o + r_lo, a multiple of 16 because o + r_lo = 0 (mod 16)
    // (a strip may be 256 wide for very large W: lanes 16..31 then only join the shuffles)
    const bool active = lane * L < p.TW;
    const int fcol = active ? lane * L + p.o + p.r_lo : 0;
    const int fpn = fcol / PWP;
    const int foff = fpn * p.ring_rows * PWP + (fcol - fpn * PWP);

    const long long T = (long long)p.tiles_x * p.h;
    const long long L0 = T * blockIdx.x / gridDim.x, L1 = T * (blockIdx.x + 1) / gridDim.x;

    for (long long cur = L0; cur < L1 && ok;) {
        const int tx = (int)(cur / p.h);
        const int y0 = (int)(cur - (long long)tx * p.h);
        const int th_eff = (int)min((long long)(p.h - y0), L1 - cur);
        cur += th_eff;

        const int x0 = tx * p.TW;
        const int xs = x0 - p.r_lo - p.o; // span start column (multiple of 16, may be < 0)
        const int ys = y0 - p.r_lo;       // first input row (may be < 0: zero-filled)
        const int nchk = (th_eff + W - 1 + CH - 1) / CH;
        const bool xin = (x0 - p.r_lo >= 0) && (x0 + p.TW - 1 + p.r_hi <= p.w - 1);

        int issued = 0, waited = 0;
        auto issue = [&](int j) {
            const int slot = j % nbar;
            uint64_t *bar = &bars[slot];
            mbar_arrive_expect_tx(bar, chunk_bytes);
            for (int pn = 0; pn < p.NPAN; ++pn) {
                uint8_t *dst = (CIN == 1) ? ring + (size_t)pn * p.ring_rows * PWP + (size_t)slot * CH * PWP
                                          : stage + ((size_t)slot * p.NPAN + pn) * CH * PWB;
                tma_load_2d(dst, &tmap, (xs + pn * PWP) * CIN, ys + j * CH, bar);
            }
        };
        auto wait_next = [&]() -> bool { // wait for chunk `waited` and advance
            const int slot = waited % nbar;
            const bool r = mbar_wait_bounded(&bars[slot], (uint32_t)((phase >> slot) & 1ull), limit);
            phase ^= 1ull << slot;
            ++waited;
            return r;
        };
        auto convert = [&](int j) { // RGB staging slot -> gray ring slot (a2), column group = thread
            if (!owner)
                return;
            const int sslot = j % p.NSS, rslot = j % p.NS;
            const uint8_t *src = stage + ((size_t)sslot * p.NPAN + gpn) * CH * PWB + 3 * gip;
            uint8_t *dst = ring + (size_t)gpn * p.ring_rows * PWP + (size_t)rslot * CH * PWP + gip;
            for (int r = 0; r < CH; ++r) {
                const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src + r * PWB);
                *reinterpret_cast<uint32_t *>(dst + r * PWP) = gray4(s32[0], s32[1], s32[2]);
            }
        };
        // Make chunks [0, upto] available as gray rows in the ring.
        auto acquire = [&](int upto) -> bool {
            bool good = true;
            if constexpr (CIN == 1) {
                while (waited <= upto)
                    good &= wait_next();
                return !__syncthreads_or(!good);
            } else {
                while (waited <= upto) {
                    const int j = waited;
                    good &= wait_next();
                    if (__syncthreads_or(!good))
                        return false;
                    convert(j);
                    __syncthreads();
                    if (issued < nchk) {
                        if (tid == 0)
                            issue(issued);
                        ++issued;
                    }
                }
                return true;
            }
        };

        // prologue: gray fills chunks 0..D (the ring has D+2 slots); RGB fills its staging slots
        {
            const int pre = CIN == 1 ? min(nchk, D + 1) : min(nchk, p.NSS);
            if (tid == 0)
                for (int j = 0; j < pre; ++j)
                    issue(j);
            issued = pre;
        }
        uint32_t c1[4] = {0u, 0u, 0u, 0u}, c2[4] = {0u, 0u, 0u, 0u};
        const uint8_t *gbase = ring + (size_t)gpn * p.ring_rows * PWP + gip;

        // warm-up: column sums over input rows 0 .. W-1 (the window of output row 0)
        ok = acquire(min(D - 1, nchk - 1));
        if (ok && owner) {
            int rr = 0;
            for (int r = 0; r < W; ++r) {
                const uint32_t v = *reinterpret_cast<const uint32_t *>(gbase + (size_t)rr * PWP);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t b = byte_of(v, j);
                    c1[j] += b;
                    c2[j] += b * b;
                }
                if (++rr == p.ring_rows)
                    rr = 0;
            }
        }
        int rr_in = W % p.ring_rows, rr_out = 0, rr_ctr = p.r_lo % p.ring_rows;

        for (int k = 0; ok && k * CH < th_eff; ++k) {
            if (CIN == 1 && issued < nchk) { // prefetch the chunk after the ones this step needs
                if (tid == 0)
                    issue(issued);
                ++issued;
            }
            if (!acquire(min(k + D, nchk - 1))) {
                ok = false;
                break;
            }
            const int rows_k = min(CH, th_eff - k * CH);

            // ---- a3: publish column sums of row i, then slide to row i+1 ------------
            if (owner) {
                for (int ii = 0; ii < rows_k; ++ii) {
                    *reinterpret_cast<uint4 *>(cb1 + ii * p.RSW + gpos) = make_uint4(c1[0], c1[1], c1[2], c1[3]);
                    *reinterpret_cast<uint4 *>(cb2 + ii * p.RSW + gpos) = make_uint4(c2[0], c2[1], c2[2], c2[3]);
                    if (k * CH + ii + 1 < th_eff) {
                        const uint32_t vin = *reinterpret_cast<const uint32_t *>(gbase + (size_t)rr_in * PWP);
                        const uint32_t vout = *reinterpret_cast<const uint32_t *>(gbase + (size_t)rr_out * PWP);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint32_t bi = byte_of(vin, j), bo = byte_of(vout, j);
                            c1[j] = c1[j] + bi - bo;
                            c2[j] = c2[j] + bi * bi - bo * bo;
                        }
                    }
                    if (++rr_in == p.ring_rows)
                        rr_in = 0;
                    if (++rr_out == p.ring_rows)
                        rr_out = 0;
                }
            } else {
                rr_in = (rr_in + rows_k) % p.ring_rows;
                rr_out = (rr_out + rows_k) % p.ring_rows;
            }
            __syncthreads();

            // ---- a4-a7: one warp per output row --------------------------------------
            for (int ii = warp; ii < rows_k; ii += NWARP) {
                const int i = k * CH + ii;
                const int y = y0 + i;
                const uint32_t *C1 = cb1 + ii * p.RSW;
                const uint32_t *C2 = cb2 + ii * p.RSW;
                const int cw = lane * L + p.o; // leaving-stream start; entering = cw + W
                const int ao = cw >> 2, ai = (cw + W) >> 2;

                uint32_t d1[L], d2[L];
                uint32_t a1 = 0, a2 = 0;
                if (active) {
                    uint4 o1 = ld_group(C1, ao), o2 = ld_group(C2, ao);
                    uint4 i1 = ld_group(C1, ai), i2 = ld_group(C2, ai);
#pragma unroll
                    for (int j = 0; j < L / 4; ++j) {
                        uint4 o1n = make_uint4(0, 0, 0, 0), o2n = o1n, i1n = o1n, i2n = o1n;
                        if (KO != 0 || j + 1 < L / 4) {
                            o1n = ld_group(C1, ao + j + 1);
                            o2n = ld_group(C2, ao + j + 1);
                        }
                        if (KI != 0 || j + 1 < L / 4) {
                            i1n = ld_group(C1, ai + j + 1);
                            i2n = ld_group(C2, ai + j + 1);
                        }
                        const uint32_t vo1[8] = {o1.x, o1.y, o1.z, o1.w, o1n.x, o1n.y, o1n.z, o1n.w};
                        const uint32_t vo2[8] = {o2.x, o2.y, o2.z, o2.w, o2n.x, o2n.y, o2n.z, o2n.w};
                        const uint32_t vi1[8] = {i1.x, i1.y, i1.z, i1.w, i1n.x, i1n.y, i1n.z, i1n.w};
                        const uint32_t vi2[8] = {i2.x, i2.y, i2.z, i2.w, i2n.x, i2n.y, i2n.z, i2n.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            d1[4 * j + e] = a1;
                            d2[4 * j + e] = a2;
                            a1 = a1 + vi1[e + KI] - vo1[e + KO];
                            a2 = a2 + vi2[e + KI] - vo2[e + KO];
                        }
                        o1 = o1n;
                        o2 = o2n;
                        i1 = i1n;
                        i2 = i2n;
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < L; ++t)
                        d1[t] = d2[t] = 0;
                }
                // window of the strip's first output: span columns [o, o + W)
                uint32_t s1 = 0, s2 = 0;
                for (int c = p.o + lane; c < p.o + W; c += 32) {
                    const int q = cpos(c);
                    s1 += C1[q];
                    s2 += C2[q];
                }
#pragma unroll
                for (int off = 16; off; off >>= 1) {
                    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
                    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
                }
                uint32_t i1s = a1, i2s = a2;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t t1 = __shfl_up_sync(0xffffffffu, i1s, off);
                    const uint32_t t2 = __shfl_up_sync(0xffffffffu, i2s, off);
                    if (lane >= off) {
                        i1s += t1;
                        i2s += t2;
                    }
                }
                const uint32_t base1 = s1 + i1s - a1, base2 = s2 + i2s - a2;

                int rc = rr_ctr + ii;
                if (rc >= p.ring_rows)
                    rc -= p.ring_rows;
                const uint4 fv = *reinterpret_cast<const uint4 *>(ring + foff + rc * PWP);
                const uint32_t fw[4] = {fv.x, fv.y, fv.z, fv.w};

                const int xg0 = x0 + lane * L;
                // a window is clipped when it leaves the image on any side
                const bool yclip = (y < p.r_lo) || (y + p.r_hi > p.h - 1);
                bool amb = yclip || (!xin && (xg0 < p.r_lo || xg0 + L - 1 + p.r_hi > p.w - 1));
                uint32_t outw[4];
                auto fast_block = [&](auto magic) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float dd[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int t = 4 * q + e;
                            const uint32_t S1 = base1 + d1[t], S2 = base2 + d2[t];
                            const unsigned long long V = (unsigned long long)p.nW * S2 -
                                                         (unsigned long long)S1 * S1;
                            const float sq = sqrt_approx(v_to_float(V));
                            const float S1f = decltype(magic)::value ? u23_to_float(S1) : __uint2float_rn(S1);
                            float ff;
                            if (e == 0)
                                ff = byte_to_float<0>(fw[q]);
                            else if (e == 1)
                                ff = byte_to_float<1>(fw[q]);
                            else if (e == 2)
                                ff = byte_to_float<2>(fw[q]);
                            else
                                ff = byte_to_float<3>(fw[q]);
                            dd[e] = filter_d<RULE>(ff, S1f, sq, p);
                            amb = amb || (fabsf(dd[e]) < p.E);
                        }
                        // byte = 0xFF where d >= +0, 0x00 where d < 0 (sign bit replicated)
                        const uint32_t lo = prmt(__float_as_uint(dd[0]), __float_as_uint(dd[1]), 0xFBu);
                        const uint32_t hi = prmt(__float_as_uint(dd[2]), __float_as_uint(dd[3]), 0xFBu);
                        outw[q] = ~prmt(lo, hi, 0x5410u);
                    }
                };
                if (p.s1_magic)
                    fast_block(std::true_type{});
                else
                    fast_block(std::false_type{});

                if (!active)
                    continue; // (after the warp-wide shuffles above)
                if (amb) { // rare: clipped windows, or values inside the fp32 margin
#pragma unroll
                    for (int t = 0; t < L; ++t) {
                        const int xg = xg0 + t;
                        if (xg >= p.w)
                            continue;
                        const uint32_t S1 = base1 + d1[t], S2 = base2 + d2[t];
                        const uint32_t f = byte_of(fw[t >> 2], t & 3);
                        bool need = yclip || xg < p.r_lo || xg + p.r_hi > p.w - 1;
                        if (!need) {
                            const unsigned long long V = (unsigned long long)p.nW * S2 -
                                                         (unsigned long long)S1 * S1;
                            const float d = filter_d<RULE>(__uint2float_rn(f), __uint2float_rn(S1),
                                                           sqrt_approx(v_to_float(V)), p);
                            need = fabsf(d) < p.E;
                        }
                        if (need) {
                            const uint32_t r = slow_decide<RULE>(f, S1, S2, y, xg, p);
                            nfb += (r >> 8) & 1u;
                            nties += (r >> 9) & 1u;
                            const int sh = 8 * (t & 3);
                            outw[t >> 2] = (outw[t >> 2] & ~(0xffu << sh)) | ((r & 0xffu) << sh);
                        }
                    }
                }

                if (!p.packed) {
                    uint8_t *drow = p.dst + (size_t)y * p.dst_pitch + xg0;
                    if (p.vec_ok && xg0 + L <= p.w) {
                        *reinterpret_cast<uint4 *>(drow) = make_uint4(outw[0], outw[1], outw[2], outw[3]);
                    } else {
#pragma unroll
                        for (int t = 0; t < L; ++t)
                            if (xg0 + t < p.w)
                                drow[t] = (uint8_t)byte_of(outw[t >> 2], t & 3);
                    }
                } else {
                    // gather the msb of each byte: bit t <-> pixel xg0 + t
                    uint32_t bits = 0;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        bits |= ((((outw[q] >> 7) & 0x01010101u) * 0x01020408u) >> 24) << (4 * q);
                    const int valid = p.w - xg0; // pixels of this lane inside the image
                    if (valid < L)
                        bits &= (valid <= 0) ? 0u : ((1u << valid) - 1u);
                    uint8_t *drow = p.dst + (size_t)y * p.dst_pitch + (xg0 >> 3);
                    const int nbytes_row = (p.w + 7) >> 3;
                    if ((xg0 >> 3) < nbytes_row)
                        drow[0] = (uint8_t)(bits & 0xffu);
                    if ((xg0 >> 3) + 1 < nbytes_row)
                        drow[1] = (uint8_t)(bits >> 8);
                }
            }
            rr_ctr = (rr_ctr + rows_k) % p.ring_rows;
            __syncthreads();
        }
        if (!ok) {
            // give up: drain this segment's outstanding copies (bounded) before leaving
            while (waited < issued)
                wait_next();
        }
    }

    // statistics: one atomic per warp
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        nfb += __shfl_xor_sync(0xffffffffu, nfb, off);
        nties += __shfl_xor_sync(0xffffffffu, nties, off);
    }
    if (lane == 0 && p.stats && (nfb | nties)) {
        atomicAdd(&p.stats[BNZ_STATS_FALLBACKS], (unsigned long long)nfb);
        atomicAdd(&p.stats[BNZ_STATS_TIES], (unsigned long long)nties);
    }
    if (!ok && tid == 0) {
        if (p.stats)
            atomicAdd(&p.stats[BNZ_STATS_TIMEOUTS], 1ull);
        atomicAdd(p.err_flag, 1u);
    }
}

template <int CIN, int RULE>
const void *pick_wm8(int wm8)
{
    switch (wm8) {
    case 0: return reinterpret_cast<const void *>(&fused_kernel<CIN, RULE, 0>);
    case 1: return reinterpret_cast<const void *>(&fused_kernel<CIN, RULE, 1>);
    case 2: return reinterpret_cast<const void *>(&fused_kernel<CIN, RULE, 2>);
    case 3: return reinterpret_cast<const void *>(&fused_kernel<CIN, RULE, 3>);
    case 4: return reinterpret_cast<const void *>(&fused_kernel<CIN, RULE, 4>);
    case 5: return reinterpret_cast<const void *>(&fused_kernel<CIN, RULE, 5>);
    case 6: return reinterpret_cast<const void *>(&fused_kernel<CIN, RULE, 6>);
    default: return reinterpret_cast<const void *>(&fused_kernel<CIN, RULE, 7>);
    }
}

const void *kernel_for(int ch, int rule, int W)
{
    const int wm8 = W & 7;
    if (ch == 1)
        return rule == BNZ_SAUVOLA ? pick_wm8<1, 0>(wm8) : pick_wm8<1, 1>(wm8);
    return rule == BNZ_SAUVOLA ? pick_wm8<3, 0>(wm8) : pick_wm8<3, 1>(wm8);
}

size_t round128(size_t v) { return (v + 127) & ~size_t(127); }

// Shared-memory layout for one (CH, NSS) choice; false if it does not fit.
bool layout(int ch, int W, int tw, int CH, int NSS, FusedPlan *pl)
{
    const int r_lo = W / 2;
    const int PWP = ch == 1 ? PanelWidth<1>::PWP : PanelWidth<3>::PWP;
    const int PWB = PWP * ch;
    pl->TW = tw;
    pl->CH = CH;
    pl->o = (16 - (r_lo % 16)) % 16;
    pl->PWP = PWP;
    // window columns of every output plus the 128-bit over-read of the streams
    const int need = pl->o + tw + W + 4;
    pl->NPAN = (need + PWP - 1) / PWP;
    pl->SWP = pl->NPAN * PWP;
    if (pl->SWP / 4 > NT)
        return false;
    // cpos() of the last group read: (SWP/4 + 1) groups of 4 words, 4 pad words per 4 groups
    pl->RSW = ((pl->SWP + 4) / 16 + 1) * 20;
    const int D = (CH + W - 1) / CH;
    pl->NS = D + 2;
    pl->NSS = ch == 3 ? NSS : 0;
    pl->ring_rows = pl->NS * CH;
    const int nbar = std::max(pl->NS, pl->NSS);
    if (nbar > 64)
        return false;
    size_t off = round128((size_t)nbar * 8);
    pl->off_ring = (uint32_t)off;
    off = round128(off + (size_t)pl->NPAN * pl->ring_rows * PWP);
    pl->off_stage = (uint32_t)off;
    off = round128(off + (size_t)pl->NSS * pl->NPAN * CH * PWB);
    pl->off_c1 = (uint32_t)off;
    off = round128(off + (size_t)CH * pl->RSW * 4);
    pl->off_c2 = (uint32_t)off;
    off += (size_t)CH * pl->RSW * 4;
    pl->smem = off;
    return off <= (size_t)MAX_DYN_SMEM;
}

} // namespace

// Error bound of the fp32 filter, u = 2^-24, e = relative error of sqrt.approx;
// V is converted with relative error <= 2u, so sqrt(V) carries <= u + e:
//   Sauvola, d32 = f - S1 * (a + b * sqrt(V)) with a ~ (1-k)/n, b ~ k/(R n^2)
//   rounded with relative error <= 3u (a) and <= 5u (b) on every path:
//     |d32 - (f - t)| <= 4u T + m |k| (s/R) (7u + e) + u (255 + T),
//     T = m (|1-k| + |k| s/R) >= |t|;
//   Niblack, d32 = f - S1/n - (k/n) sqrt(V):
//     |d32 - (f - t)| <= u (255 + 510 + 510 + |k| s_max) + |k| s (4u + e).
// With m <= 255 and s <= 127.5 this gives Emax; E = 2 Emax + 1e-6 also covers
// the fp64 definition's own rounding (< 1e-12) and keeps every pixel with
// |f - t| < 1e-9 inside the margin, so ties are always decided in fp64.
float decision_margin(int rule, double k, double R)
{
    const double u = 1.0 / 16777216.0;
    const double e = kSqrtApproxRelErr;
    const double ak = std::fabs(k);
    const double m = 255.0, smax = 127.5;
    double em;
    if (rule == BNZ_SAUVOLA) {
        const double T = m * (std::fabs(1.0 - k) + ak * smax / R);
        em = 4.0 * u * T + m * ak * (smax / R) * (7.0 * u + e) + u * (255.0 + T);
    } else {
        em = u * (255.0 + 510.0 + 510.0 + ak * smax) + ak * smax * (4.0 * u + e);
    }
    double E = 2.0 * em + 1e-6;
    if (!(E < 1e30))
        E = 1e30;
    return (float)E;
}

int plan_fused(int h, int w, int ch, int W, const bnz_tile *tile, FusedPlan *pl)
{
    int sms = 0;
    int rc = device_sm_count(&sms);
    if (rc != BNZ_OK)
        return rc;
    const int want_tw = tile ? tile->tile_w : 0;
    const int want_ch = tile && tile->chunk ? tile->chunk : 8;
    if (want_ch != 8 && want_ch != 16)
        return fail(BNZ_EINVAL, "bnz_tile.chunk must be 0, 8 or 16 (got %d)", want_ch);
    if (want_tw && want_tw != TW && want_tw != TW / 2)
        return fail(BNZ_EINVAL, "bnz_tile.tile_w must be 0, %d or %d (got %d)", TW / 2, TW, want_tw);
    bool found = false;
    for (int tw = TW; tw >= TW / 2 && !found; tw /= 2) {
        if (want_tw && tw != want_tw)
            continue;
        for (int nss = 3; nss >= 2 && !found; --nss)
            found = layout(ch, W, tw, want_ch, nss, pl);
    }
    if (!found)
        return fail(BNZ_EINVAL, "no tile shape fits shared memory for W=%d, chunk=%d", W, want_ch);
    pl->tiles_x = (w + pl->TW - 1) / pl->TW;
    int occ = 1;
    const void *fn = kernel_for(ch, BNZ_SAUVOLA, W);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl->smem);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaFuncSetAttribute(fused)");
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, NT, pl->smem);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    occ = std::max(occ, 1);
    // persistent grid: one CTA per resident slot, but at least ~2W rows of work per CTA
    const long long T = (long long)pl->tiles_x * h;
    const long long min_rows = std::max(2 * W, 32);
    long long G = std::min<long long>((long long)sms * occ, (T + min_rows - 1) / min_rows);
    if (tile && tile->tile_h > 0)
        G = (T + tile->tile_h - 1) / tile->tile_h;
    G = std::max<long long>(1, std::min<long long>(G, 1 << 30));
    pl->grid = (int)G;
    pl->rows_per_cta = (int)((T + G - 1) / G);
    return BNZ_OK;
}

int launch_fused(const uint8_t *d_src, size_t src_pitch, int h, int w, int ch, int W, int rule, double k, double R,
                 uint8_t *d_dst, size_t dst_pitch, int packed, const bnz_tile *tile, cudaStream_t stream,
                 unsigned long long *d_stats, unsigned int *d_err)
{
    FusedPlan pl;
    int rc = plan_fused(h, w, ch, W, tile, &pl);
    if (rc != BNZ_OK)
        return rc;
    CUtensorMap map;
    const int PWB = pl.PWP * ch;
    rc = encode_u8_map(&map, d_src, (uint64_t)w * ch, (uint64_t)h, (uint64_t)src_pitch, (uint32_t)PWB,
                       (uint32_t)pl.CH);
    if (rc != BNZ_OK)
        return rc;
    FusedParams p;
    p.dst = d_dst;
    p.dst_pitch = (long long)dst_pitch;
    p.stats = d_stats;
    p.err_flag = d_err;
    p.h = h;
    p.w = w;
    p.W = W;
    p.r_lo = W / 2;
    p.r_hi = W - 1 - W / 2;
    p.o = pl.o;
    p.TW = pl.TW;
    p.CH = pl.CH;
    p.NS = pl.NS;
    p.NSS = pl.NSS;
    p.NPAN = pl.NPAN;
    p.SWP = pl.SWP;
    p.RSW = pl.RSW;
    p.ring_rows = pl.ring_rows;
    p.tiles_x = pl.tiles_x;
    p.off_ring = pl.off_ring;
    p.off_stage = pl.off_stage;
    p.off_c1 = pl.off_c1;
    p.off_c2 = pl.off_c2;
    p.packed = packed ? 1 : 0;
    p.vec_ok = ((reinterpret_cast<uintptr_t>(d_dst) | dst_pitch) & 15u) == 0 ? 1 : 0;
    p.s1_magic = (long long)W * W * 255 < (1ll << 23) ? 1 : 0;
    p.nW = (uint32_t)(W * W);
    p.k = k;
    p.R = R;
    const double n = (double)W * (double)W;
    p.omkn = (float)((1.0 - k) / n);
    p.kRn2 = (float)(k / (R * n * n));
    p.invn = (float)(1.0 / n);
    p.kn = (float)(k / n);
    p.kf = (float)k;
    p.omk = (float)(1.0 - k);
    p.kR = (float)(k / R);
    p.E = decision_margin(rule, k, R);
    p.timeout_cycles = 4000000000ll; // ~2 s at 2 GHz
    const void *fn = kernel_for(ch, rule, W);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaFuncSetAttribute(fused)");
    void *args[] = {(void *)&map, (void *)&p};
    e = cudaLaunchKernel(fn, dim3((unsigned)pl.grid), dim3(NT), args, pl.smem, stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "launch fused kernel");
    return BNZ_OK;
}

} // namespace bnz
