// fused.cu -- the fused tile kernel for exact Sauvola / Niblack binarization.
//
// One persistent CTA walks a contiguous range of "strip rows": the image is
// cut into vertical strips of tile_w output columns, the strips are laid end
// to end (strip-major), and the total is split evenly over the grid.  For each
// run of rows it owns in a strip the CTA
//   a1  loads the strip plus its halo (W-1 columns, 16-aligned on the left)
//       row-chunk by row-chunk with 2-D TMA boxes into a shared-memory ring
//       that holds the last W + 2*chunk rows (every input byte is fetched from
//       global memory once per strip),
//   a2  for RGB input converts each chunk to gray in shared memory with the
//       integer rule of Eq. 1: f = (299 r + 587 g + 114 b + 500) / 1000,
//   a3  keeps exact integer column sums c1 = sum f, c2 = sum f^2 over the W
//       window rows in registers (4 columns per thread): add the entering row,
//       publish, subtract the leaving row -- O(1) per column per row,
//   a4  gets the horizontal window sums S1, S2 from the published column sums:
//       each lane slides over L consecutive outputs, the lanes' partial sums
//       are joined with a warp scan, and one warp-wide reduction gives the
//       first window of the row,
//   a5  takes n = W*W in the interior, the clipped count at the borders,
//   a6  decides f < t (Eq. 3) for Sauvola (Eq. 4) or Niblack with an fp32
//       filter whose error bound is proven; pixels inside the bound are
//       re-evaluated with the fp64 sequence m = S1/n, s = sqrt(V)/n, t = ...,
//       so every output equals that fp64 decision,
//   a7  writes the byte mask {0,255} or the packed 1-bit mask.
// The sums are never rounded: S1 < 2^24 and S2 < 2^32 for W <= 255, and
// V = n*S2 - S1^2 is formed in 64-bit integers.
#include <algorithm>
#include <cstdio>

#include "internal.h"
#include "ptx.cuh"

namespace bnz {
namespace {

constexpr int NT = 256;
constexpr int NWARP = NT / 32;
constexpr int MAX_DYN_SMEM = 232448 - 1024; // 227 KB opt-in limit, minus static/slack

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

// Eq. 1, integer round-half-up: q = floor(x / 1000) with x <= 255500 computed
// as the high word of x * ceil(2^32 / 1000) (exact for x < 6.1e6).
__device__ __forceinline__ uint32_t gray_of(uint32_t r, uint32_t g, uint32_t b)
{
    return __umulhi(299u * r + 587u * g + 114u * b + 500u, 4294968u);
}

// Four gray pixels from 12 interleaved bytes r0 g0 b0 r1 | g1 b1 r2 g2 | b2 r3 g3 b3.
__device__ __forceinline__ uint32_t gray4(uint32_t w0, uint32_t w1, uint32_t w2)
{
    const uint32_t p0 = gray_of(byte_of(w0, 0), byte_of(w0, 1), byte_of(w0, 2));
    const uint32_t p1 = gray_of(byte_of(w0, 3), byte_of(w1, 0), byte_of(w1, 1));
    const uint32_t p2 = gray_of(byte_of(w1, 2), byte_of(w1, 3), byte_of(w2, 0));
    const uint32_t p3 = gray_of(byte_of(w2, 1), byte_of(w2, 2), byte_of(w2, 3));
    return p0 | (p1 << 8) | (p2 << 16) | (p3 << 24);
}

// Eq. 3 with Eq. 4 (RULE 0) or Niblack (RULE 1).  fp32 filter, fp64 re-check.
template <int RULE>
__device__ __forceinline__ uint32_t decide(uint32_t f, uint32_t n, uint32_t S1, uint32_t S2, bool interior,
                                           const FusedParams &p, uint32_t &nfb, uint32_t &nties)
{
    const long long V = (long long)n * (long long)S2 - (long long)S1 * (long long)S1;
    const float sq = __fsqrt_rn(__ll2float_rn(V));
    const float S1f = __uint2float_rn(S1);
    float m, s;
    if (interior) {
        m = __fmul_rn(S1f, p.invn);
        s = __fmul_rn(sq, p.invn);
    } else {
        const float nf = __uint2float_rn(n);
        m = __fdiv_rn(S1f, nf);
        s = __fdiv_rn(sq, nf);
    }
    float t;
    if (RULE == BNZ_SAUVOLA)
        t = __fmul_rn(m, __fmaf_rn(p.kf, __fmaf_rn(s, p.invRf, -1.0f), 1.0f));
    else
        t = __fmaf_rn(p.kf, s, m);
    const float d = __fsub_rn(__uint2float_rn(f), t);
    if (fabsf(d) >= p.E)
        return d < 0.0f ? 0u : 255u;
    // Inside the fp32 margin (or t not finite): the fp64 sequence, same order
    // and roundings as the definition, no contraction.
    ++nfb;
    const double nd = (double)n;
    const double md = __ddiv_rn((double)S1, nd);
    const double sd = __ddiv_rn(__dsqrt_rn(__ll2double_rn(V)), nd);
    double td;
    if (RULE == BNZ_SAUVOLA)
        td = __dmul_rn(md, __dadd_rn(1.0, __dmul_rn(p.k, __dsub_rn(__ddiv_rn(sd, p.R), 1.0))));
    else
        td = __dadd_rn(md, __dmul_rn(p.k, sd));
    const double fd = (double)f;
    nties += fabs(__dsub_rn(fd, td)) < 1e-9 ? 1u : 0u;
    return fd < td ? 0u : 255u;
}

template <int CIN, int RULE, int PACKED, int L>
__global__ void __launch_bounds__(NT, 1) fused_kernel(const __grid_constant__ CUtensorMap tmap, const FusedParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr int PWP = PanelWidth<CIN>::PWP;
    constexpr int PWB = PWP * CIN;
    constexpr int SKS = L >= 32 ? 5 : 4; // bank skew of the column-sum rows

    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    uint8_t *ring = smem + p.off_ring;
    uint8_t *stage = smem + p.off_stage;
    uint2 *cb = reinterpret_cast<uint2 *>(smem + p.off_cb);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int CH = p.CH;
    const int W = p.W;
    const int D = (CH + W - 2) / CH; // chunks beyond the current one that a chunk of outputs needs
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

    // column-owner geometry (phase a3): 4 consecutive span columns per thread
    const bool owner = tid < ng;
    const int gcol = tid * 4;
    const int gpn = gcol / PWP, gip = gcol - gpn * PWP;

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
        const bool interior = (x0 - p.r_lo >= 0) && (x0 + p.TW - 1 + p.r_hi <= p.w - 1) && (ys >= 0) &&
                              (y0 + th_eff - 1 + p.r_hi <= p.h - 1);

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
        auto convert = [&](int j) { // RGB staging slot -> gray ring slot (a2)
            const int sslot = j % p.NSS, rslot = j % p.NS;
            const int q4 = p.SWP >> 2;
            for (int u = tid; u < CH * q4; u += NT) {
                const int r = u / q4, c = (u - r * q4) * 4;
                const int pn = c / PWP, ip = c - pn * PWP;
                const uint32_t *s32 = reinterpret_cast<const uint32_t *>(
                    stage + ((size_t)sslot * p.NPAN + pn) * CH * PWB + (size_t)r * PWB + 3 * ip);
                *reinterpret_cast<uint32_t *>(ring + (size_t)pn * p.ring_rows * PWP +
                                              (size_t)(rslot * CH + r) * PWP + ip) = gray4(s32[0], s32[1], s32[2]);
            }
        };
        // Make chunks [0, upto] available as gray rows in the ring.
        auto acquire = [&](int upto) -> bool {
            bool good = true;
            if constexpr (CIN == 1) {
                while (waited <= upto)
                    good &= wait_next();
                return !__syncthreads_or(!good);
            }
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

        // warm-up: column sums over input rows 0 .. W-2
        if (D > 0)
            ok = acquire(D - 1);
        if (ok && owner) {
            int rr = 0;
            for (int r = 0; r < W - 1; ++r) {
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

            // ---- a3: column sums, entering row i+W-1, leaving row i -------------------
            if (owner) {
                int rin = (k * CH + W - 1) % p.ring_rows, rout = (k * CH) % p.ring_rows;
                for (int ii = 0; ii < rows_k; ++ii) {
                    const uint32_t vin = *reinterpret_cast<const uint32_t *>(gbase + (size_t)rin * PWP);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint32_t b = byte_of(vin, j);
                        c1[j] += b;
                        c2[j] += b * b;
                    }
                    uint2 *row = cb + (size_t)ii * p.RS;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int c = gcol + j;
                        row[c + (c >> SKS)] = make_uint2(c1[j], c2[j]);
                    }
                    const uint32_t vout = *reinterpret_cast<const uint32_t *>(gbase + (size_t)rout * PWP);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint32_t b = byte_of(vout, j);
                        c1[j] -= b;
                        c2[j] -= b * b;
                    }
                    if (++rin == p.ring_rows)
                        rin = 0;
                    if (++rout == p.ring_rows)
                        rout = 0;
                }
            }
            __syncthreads();

            // ---- a4-a7: one warp per output row ----------------------------------------
            for (int ii = warp; ii < rows_k; ii += NWARP) {
                const int i = k * CH + ii;
                const int y = y0 + i;
                const uint2 *row = cb + (size_t)ii * p.RS;
                const int xl = lane * L;
                const int cw = xl + p.o; // span column where the window of output xl starts
                uint32_t d1[L], d2[L];
                uint32_t a1 = 0, a2 = 0;
#pragma unroll
                for (int t = 0; t < L; ++t) {
                    d1[t] = a1;
                    d2[t] = a2;
                    const int ci = cw + t + W, co = cw + t;
                    const uint2 vi = row[ci + (ci >> SKS)];
                    const uint2 vo = row[co + (co >> SKS)];
                    a1 += vi.x - vo.x;
                    a2 += vi.y - vo.y;
                }
                uint32_t s1 = 0, s2 = 0;
                for (int c = p.o + lane; c < p.o + W; c += 32) {
                    const uint2 v = row[c + (c >> SKS)];
                    s1 += v.x;
                    s2 += v.y;
                }
#pragma unroll
                for (int off = 16; off; off >>= 1) {
                    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
                    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
                }
                uint32_t i1 = a1, i2 = a2;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t t1 = __shfl_up_sync(0xffffffffu, i1, off);
                    const uint32_t t2 = __shfl_up_sync(0xffffffffu, i2, off);
                    if (lane >= off) {
                        i1 += t1;
                        i2 += t2;
                    }
                }
                const uint32_t base1 = s1 + i1 - a1, base2 = s2 + i2 - a2;

                // centre pixels f: span columns xl + o + r_lo .., ring row of input row i + r_lo
                const int rr = (i + p.r_lo) % p.ring_rows;
                const int a = xl + p.o + p.r_lo;
                const int a0 = a & ~3;
                const uint32_t sh = (uint32_t)(a & 3) * 8u;
                uint32_t fw[L / 4 + 1];
#pragma unroll
                for (int q = 0; q <= L / 4; ++q) {
                    const int c = a0 + 4 * q;
                    const int pn = c / PWP;
                    fw[q] = *reinterpret_cast<const uint32_t *>(ring + (size_t)pn * p.ring_rows * PWP +
                                                                (size_t)rr * PWP + (c - pn * PWP));
                }
#pragma unroll
                for (int q = 0; q < L / 4; ++q)
                    fw[q] = __funnelshift_r(fw[q], fw[q + 1], sh);

                int nrow = 0;
                if (!interior)
                    nrow = min(y + p.r_hi, p.h - 1) - max(y - p.r_lo, 0) + 1;
                const int xg0 = x0 + xl;
                uint32_t outw[L / 4];
#pragma unroll
                for (int q = 0; q < L / 4; ++q)
                    outw[q] = 0u;
#pragma unroll
                for (int t = 0; t < L; ++t) {
                    const int xg = xg0 + t;
                    if (xg < p.w) {
                        const uint32_t f = byte_of(fw[t >> 2], t & 3);
                        uint32_t n = (uint32_t)(W * W);
                        if (!interior)
                            n = (uint32_t)(nrow * (min(xg + p.r_hi, p.w - 1) - max(xg - p.r_lo, 0) + 1));
                        const uint32_t g =
                            decide<RULE>(f, n, base1 + d1[t], base2 + d2[t], interior, p, nfb, nties);
                        outw[t >> 2] |= g << (8 * (t & 3));
                    }
                }

                if (!PACKED) {
                    uint8_t *drow = p.dst + (size_t)y * p.dst_pitch + xg0;
                    if (p.vec_ok && xg0 + L <= p.w) {
                        if (L == 8) {
                            *reinterpret_cast<uint2 *>(drow) = make_uint2(outw[0], outw[1]);
                        } else {
#pragma unroll
                            for (int q = 0; q < L / 4; q += 4)
                                *reinterpret_cast<uint4 *>(drow + 4 * q) =
                                    make_uint4(outw[q], outw[q + 1], outw[q + 2], outw[q + 3]);
                        }
                    } else {
#pragma unroll
                        for (int t = 0; t < L; ++t)
                            if (xg0 + t < p.w)
                                drow[t] = (uint8_t)byte_of(outw[t >> 2], t & 3);
                    }
                } else {
                    uint8_t *drow = p.dst + (size_t)y * p.dst_pitch + (xg0 >> 3);
                    const int nbytes_row = (p.w + 7) >> 3;
#pragma unroll
                    for (int b = 0; b < L / 8; ++b) {
                        uint32_t bits = 0;
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            bits |= (byte_of(outw[(8 * b + j) >> 2], (8 * b + j) & 3) & 1u) << j;
                        if ((xg0 >> 3) + b < nbytes_row)
                            drow[b] = (uint8_t)bits;
                    }
                }
            }
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

template <int CIN, int RULE, int PACKED>
const void *pick_kernel(int L)
{
    switch (L) {
    case 8:
        return reinterpret_cast<const void *>(&fused_kernel<CIN, RULE, PACKED, 8>);
    case 16:
        return reinterpret_cast<const void *>(&fused_kernel<CIN, RULE, PACKED, 16>);
    default:
        return nullptr;
    }
}

const void *kernel_for(int ch, int rule, int packed, int L)
{
    if (ch == 1) {
        if (rule == BNZ_SAUVOLA)
            return packed ? pick_kernel<1, 0, 1>(L) : pick_kernel<1, 0, 0>(L);
        return packed ? pick_kernel<1, 1, 1>(L) : pick_kernel<1, 1, 0>(L);
    }
    if (rule == BNZ_SAUVOLA)
        return packed ? pick_kernel<3, 0, 1>(L) : pick_kernel<3, 0, 0>(L);
    return packed ? pick_kernel<3, 1, 1>(L) : pick_kernel<3, 1, 0>(L);
}

size_t round128(size_t v) { return (v + 127) & ~size_t(127); }

// Shared-memory layout for one (L, CH, NSS) choice; false if it does not fit.
bool layout(int ch, int W, int L, int CH, int NSS, FusedPlan *pl)
{
    const int r_lo = W / 2;
    const int PWP = ch == 1 ? PanelWidth<1>::PWP : PanelWidth<3>::PWP;
    const int PWB = PWP * ch;
    pl->L = L;
    pl->TW = 32 * L;
    pl->CH = CH;
    pl->o = (16 - (r_lo % 16)) % 16;
    pl->PWP = PWP;
    const int need = pl->o + pl->TW + W + 4; // window columns of every output, +4 for word reads
    pl->NPAN = (need + PWP - 1) / PWP;
    pl->SWP = pl->NPAN * PWP;
    if (pl->SWP / 4 > NT)
        return false;
    const int sks = L >= 32 ? 5 : 4;
    pl->RS = pl->SWP + (pl->SWP >> sks) + 1;
    const int D = (CH + W - 2) / CH;
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
    pl->off_cb = (uint32_t)off;
    off += (size_t)CH * pl->RS * sizeof(uint2);
    pl->smem = off;
    return off <= (size_t)MAX_DYN_SMEM;
}

} // namespace

float decision_margin(int rule, double k, double R)
{
    // |t32 - t| <= u m (5 + |k| (13.5 s/R + 8))  (Sauvola)  or  u (3 m + 6.5 |k| s)  (Niblack),
    // u = 2^-24, m <= 255, s <= 127.5; doubled, plus 1e-6 absolute slack.
    const double u = 1.0 / 16777216.0;
    const double ak = std::fabs(k);
    double e;
    if (rule == BNZ_SAUVOLA)
        e = u * 255.0 * (5.0 + ak * (13.5 * 127.5 / R + 8.0));
    else
        e = u * (3.0 * 255.0 + 6.5 * ak * 127.5);
    e = 2.0 * e + 1e-6;
    if (!(e < 1e30))
        e = 1e30;
    return (float)e;
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
    if (want_tw && want_tw != 256 && want_tw != 512)
        return fail(BNZ_EINVAL, "bnz_tile.tile_w must be 0, 256 or 512 (got %d)", want_tw);
    const int Ls[2] = {16, 8};
    bool found = false;
    for (int li = 0; li < 2 && !found; ++li) {
        const int L = Ls[li];
        if (want_tw && 32 * L != want_tw)
            continue;
        if (!want_tw && L == 16 && w <= 256)
            continue; // narrow pages: the 256-wide tile wastes less
        for (int nss = 3; nss >= 2 && !found; --nss)
            found = layout(ch, W, L, want_ch, nss, pl);
    }
    if (!found)
        return fail(BNZ_EINVAL, "no tile shape fits shared memory for W=%d (max %d)", W, BNZ_MAX_W);
    pl->tiles_x = (w + pl->TW - 1) / pl->TW;
    // persistent grid: one CTA per SM slot, but at least ~2W rows of work per CTA
    const int occ = std::max(1, std::min(NT == 256 ? 8 : 4, (int)(233472 / (pl->smem + 1024))));
    const long long T = (long long)pl->tiles_x * h;
    const long long min_rows = std::max(2 * W, 32);
    long long G = std::min<long long>((long long)sms * occ, (T + min_rows - 1) / min_rows);
    if (tile && tile->tile_h > 0)
        G = std::max<long long>(1, (T + tile->tile_h - 1) / tile->tile_h);
    G = std::max<long long>(1, std::min<long long>(G, 1 << 30));
    pl->tiles_y = (int)G; // grid size (CTAs)
    pl->TH = (int)((T + G - 1) / G);
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
    p.RS = pl.RS;
    p.ring_rows = pl.ring_rows;
    p.tiles_x = pl.tiles_x;
    p.off_ring = pl.off_ring;
    p.off_stage = pl.off_stage;
    p.off_cb = pl.off_cb;
    p.k = k;
    p.R = R;
    p.kf = (float)k;
    p.invRf = (float)(1.0 / R);
    p.E = decision_margin(rule, k, R);
    p.invn = (float)(1.0 / ((double)W * (double)W));
    p.vec_ok = ((reinterpret_cast<uintptr_t>(d_dst) | dst_pitch) & 15u) == 0 ? 1 : 0;
    p.timeout_cycles = 4000000000ll; // ~2 s at 2 GHz
    const void *fn = kernel_for(ch, rule, packed, pl.L);
    if (!fn)
        return fail(BNZ_EINVAL, "no kernel instance for L=%d", pl.L);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaFuncSetAttribute(fused)");
    void *args[] = {(void *)&map, (void *)&p};
    e = cudaLaunchKernel(fn, dim3((unsigned)pl.tiles_y), dim3(NT), args, pl.smem, stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "launch fused kernel");
    return BNZ_OK;
}

} // namespace bnz
