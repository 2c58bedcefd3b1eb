// otsu.cu -- global binarization (Eq. 2) with Otsu's threshold.
//
// Sec. 1 names Otsu's method as the best global technique and Eq. 2 applies
// one threshold T to every pixel: g = 0 if f < T, else 255.  T follows Otsu's
// published definition: over the 256-bin histogram of the gray page (Eq. 1),
// T in [1, 255] splits the levels into [0, T-1] and [T, 255] (counts n0, n1,
// level sums s0, s1; N, S the totals) and maximises the between-class
// variance w0 w1 (mu0 - mu1)^2 = D^2 / (N^2 n0 n1) with D = N s0 - S n0.
// D is exact (128-bit products; |D| <= 255 N^2 / 4 < 2^63 for N <= 2^28), the
// criterion is q = (d * d) / (a * b) in fp64 with d = D, a = n0, b = n1
// converted once each, and the smallest T with the largest q wins (T = 0,
// every pixel 255, when no T leaves both classes non-empty).
//
// Two launches (and a memset of the scratch) on the caller's stream, no host
// round trip:
//   otsu_hist    the histogram: four 256-bin tables per warp in shared memory
//                (lanes j, j+4, ...), merged into the caller's scratch with
//                64-bit atomics; each thread takes 16 pixels per step (128-bit
//                loads); each CTA adds its counts into one of 16 partial tables
//                in the scratch (CTA i into table i mod 16: 16 times fewer
//                atomic additions per global counter than one shared table).
//                The last CTA to finish sums the partial tables into the
//                histogram and picks T (select_T): a
//                block scan gives every thread t the exact prefixes n0, s0 of
//                the levels below t, thread t evaluates q(t), a block reduction
//                takes the argmax and stores T in the scratch;
//   otsu_mask    Eq. 2 with T read from the scratch: byte or packed mask,
//                16 pixels per thread and step.
// Both passes over the page are HBM streams (1 or 3 B/px read each, 1 B/px or
// 1/8 B/px written by the second).
#include <algorithm>
#include <cstdint>

#include "segment.cuh" // gray1 / gray4: the Eq. 1 rule of the fused kernel

namespace bnz {
namespace {

constexpr int kOtsuThreads = 256;
constexpr int kHistOffset = 0;    // uint64[256] in the scratch
constexpr int kTOffset = 2048;    // int32 T in the scratch
constexpr int kDoneOffset = 2052; // uint32 count of histogram CTAs done (the last one picks T)
constexpr int kPartOffset = 4096; // uint32[kParts][256]: the CTAs' partial histograms
constexpr int kParts = 16;
static_assert(kPartOffset + kParts * 256 * 4 <= BNZ_OTSU_SCRATCH_BYTES, "Otsu scratch too small");
constexpr int kCopies = 4;        // shared histogram tables per warp

// Gray values of the 16 pixels starting at column x of row `row` (x a
// multiple of 16, x + 16 <= w): 16 bytes (gray) or 48 bytes (RGB), 128-bit
// loads from a 16-byte aligned row start.
template <int CIN>
__device__ __forceinline__ void load16(const uint8_t *row, int x, uint32_t (&g)[4])
{
    if (CIN == 1) {
        const uint4 v = *reinterpret_cast<const uint4 *>(row + x);
        g[0] = v.x;
        g[1] = v.y;
        g[2] = v.z;
        g[3] = v.w;
    } else {
        const uint4 *p = reinterpret_cast<const uint4 *>(row + 3 * x);
        const uint4 a = p[0], b = p[1], c = p[2];
        g[0] = gray4(a.x, a.y, a.z);
        g[1] = gray4(a.w, b.x, b.y);
        g[2] = gray4(b.z, b.w, c.x);
        g[3] = gray4(c.y, c.z, c.w);
    }
}

// The raw 16 or 48 bytes of a 16-pixel group (loads only: converted later, so
// the next group's loads are in flight while this one is counted)
template <int CIN>
__device__ __forceinline__ void load16_raw(const uint8_t *row, int x, uint4 (&r)[CIN])
{
    const uint4 *p = reinterpret_cast<const uint4 *>(row + CIN * x);
#pragma unroll
    for (int i = 0; i < CIN; ++i)
        r[i] = p[i];
}

template <int CIN>
__device__ __forceinline__ void gray16(const uint4 (&r)[CIN], uint32_t (&g)[4])
{
    if (CIN == 1) {
        g[0] = r[0].x;
        g[1] = r[0].y;
        g[2] = r[0].z;
        g[3] = r[0].w;
    } else {
        const uint4 a = r[0], b = r[1 % CIN], c = r[2 % CIN];
        g[0] = gray4(a.x, a.y, a.z);
        g[1] = gray4(a.w, b.x, b.y);
        g[2] = gray4(b.z, b.w, c.x);
        g[3] = gray4(c.y, c.z, c.w);
    }
}

template <int CIN>
__device__ __forceinline__ uint32_t gray_at(const uint8_t *row, int x)
{
    if (CIN == 1)
        return row[x];
    const uint8_t *px = row + 3 * x;
    return gray1((uint32_t)px[0] | ((uint32_t)px[1] << 8) | ((uint32_t)px[2] << 16));
}

// Otsu's T from the complete histogram, by one CTA of kOtsuThreads = 256
// threads (one level each; c = the count of level threadIdx.x).
__device__ void select_T(unsigned long long c, int *T_out)
{
    __shared__ unsigned long long wn[kOtsuThreads / 32], ws[kOtsuThreads / 32], tot[2];
    __shared__ double sq[kOtsuThreads / 32];
    __shared__ int st[kOtsuThreads / 32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const unsigned long long v = c * (unsigned long long)t;
    // inclusive block scan of (count, level sum), exact 64-bit (N <= 2^28)
    unsigned long long cn = c, cs = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long a = __shfl_up_sync(0xffffffffu, cn, off);
        const unsigned long long b = __shfl_up_sync(0xffffffffu, cs, off);
        if (lane >= off) {
            cn += a;
            cs += b;
        }
    }
    if (lane == 31) {
        wn[wid] = cn;
        ws[wid] = cs;
    }
    __syncthreads();
    if (t == 0) { // exclusive offsets of the 8 warps, and the totals
        unsigned long long an = 0, as = 0;
        for (int k = 0; k < kOtsuThreads / 32; ++k) {
            const unsigned long long xn = wn[k], xs = ws[k];
            wn[k] = an;
            ws[k] = as;
            an += xn;
            as += xs;
        }
        tot[0] = an;
        tot[1] = as;
    }
    __syncthreads();
    const unsigned long long N = tot[0], S = tot[1];
    const unsigned long long n0 = cn + wn[wid] - c, s0 = cs + ws[wid] - v; // levels 0 .. t-1
    const unsigned long long n1 = N - n0;
    double q = -1.0; // t = 0 and splits with an empty class take no part
    if (t > 0 && n0 > 0 && n1 > 0) {
        const __int128 D = (__int128)N * (__int128)s0 - (__int128)S * (__int128)n0;
        const double d = (double)(long long)D; // |D| < 2^63: one rounding, as the definition's
        const double a = (double)n0, b = (double)n1;
        q = __ddiv_rn(__dmul_rn(d, d), __dmul_rn(a, b));
    }
    // argmax, the smallest t among equal q
    int bt = t;
    double bq = q;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const double oq = __shfl_down_sync(0xffffffffu, bq, off);
        const int ot = __shfl_down_sync(0xffffffffu, bt, off);
        if (oq > bq || (oq == bq && ot < bt)) {
            bq = oq;
            bt = ot;
        }
    }
    if ((t & 31) == 0) {
        sq[t >> 5] = bq;
        st[t >> 5] = bt;
    }
    __syncthreads();
    if (t == 0) {
        for (int k = 1; k < kOtsuThreads / 32; ++k)
            if (sq[k] > bq || (sq[k] == bq && st[k] < bt)) {
                bq = sq[k];
                bt = st[k];
            }
        *T_out = bq < 0.0 ? 0 : bt;
    }
}

template <int CIN>
__global__ void __launch_bounds__(kOtsuThreads)
    otsu_hist(const uint8_t *src, long long pitch, int h, int w, unsigned long long *hist, uint32_t *parts,
              unsigned int *done, int *T_out)
{
    // four tables per warp (lanes j, j+4, ...): a page's few dominant levels
    // would otherwise serialize all 32 lanes of a warp on one shared counter
    __shared__ uint32_t sh[kOtsuThreads / 32 * kCopies][256];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (kOtsuThreads / 32) * kCopies * 256; i += kOtsuThreads)
        (&sh[0][0])[i] = 0;
    __syncthreads();
    uint32_t *mine = sh[warp * kCopies + (threadIdx.x & (kCopies - 1))];
    const int groups = (w + 15) / 16; // 16-pixel groups per row
    const long long total = (long long)groups * h;
    // (row, group) of the thread's index, carried by the stride's quotient and
    // remainder: no 64-bit division per step
    const long long stride = (long long)gridDim.x * kOtsuThreads;
    const int sq = (int)(stride / groups), sr = (int)(stride - (long long)sq * groups);
    const long long g0 = (long long)blockIdx.x * kOtsuThreads + threadIdx.x;
    int y = (int)(g0 / groups), gx = (int)(g0 - (long long)y * groups);
    // software pipeline: the raw bytes of the thread's next full group are
    // loaded before the current one is counted
    uint4 cur[CIN];
    bool have = false;
    auto full = [&](int yy, int xx) { return xx + 16 <= w && yy < h; };
    if (g0 < total && full(y, gx * 16)) {
        load16_raw<CIN>(src + (long long)y * pitch, gx * 16, cur);
        have = true;
    }
    for (long long gi = g0; gi < total; gi += stride) {
        const int x = gx * 16;
        const uint8_t *row = src + (long long)y * pitch;
        int ny = y + sq, ngx = gx + sr;
        if (ngx >= groups) {
            ngx -= groups;
            ++ny;
        }
        uint4 nxt[CIN];
        const bool nfull = gi + stride < total && full(ny, ngx * 16);
        if (nfull)
            load16_raw<CIN>(src + (long long)ny * pitch, ngx * 16, nxt);
        if (have) {
            uint32_t g[4];
            gray16<CIN>(cur, g);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    atomicAdd(&mine[(g[q] >> (8 * j)) & 0xffu], 1u);
        } else {
            for (int xx = x; xx < w; ++xx)
                atomicAdd(&mine[gray_at<CIN>(row, xx)], 1u);
        }
        if (nfull) {
#pragma unroll
            for (int i = 0; i < CIN; ++i)
                cur[i] = nxt[i];
        }
        have = nfull;
        gx = ngx;
        y = ny;
    }
    __syncthreads();
    uint32_t *part = parts + (blockIdx.x % kParts) * 256;
    for (int b = threadIdx.x; b < 256; b += kOtsuThreads) {
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < kOtsuThreads / 32 * kCopies; ++k)
            c += sh[k][b];
        if (c)
            atomicAdd(&part[b], c); // < 2^28 pixels: a partial table's counts fit 32 bits
    }
    // the last CTA to finish picks T (the histogram is complete once every
    // CTA's additions are visible: each fences before it counts itself)
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        unsigned long long c = 0; // kOtsuThreads = 256: thread t sums level t over the partial tables
#pragma unroll
        for (int k = 0; k < kParts; ++k)
            c += __ldcg(parts + k * 256 + threadIdx.x);
        hist[threadIdx.x] = c;
        select_T(c, T_out);
        if (threadIdx.x == 0)
            *done = 0u; // ready for the next call on this scratch
    }
}

template <int CIN>
__global__ void __launch_bounds__(kOtsuThreads)
    otsu_mask(const uint8_t *src, long long pitch, int h, int w, const int *T_in, uint8_t *dst, long long dst_pitch,
              int packed, int vec_ok)
{
    const uint32_t T = (uint32_t)*T_in;
    // byte-wise f >= T for four packed gray values: __vcmpgeu4 gives 0xFF / 0x00 per byte
    const uint32_t T4 = T > 255u ? 0u : T * 0x01010101u;
    const int groups = (w + 15) / 16;
    const long long total = (long long)groups * h;
    // (row, group) of the thread's index, carried by the stride's quotient and
    // remainder: no 64-bit division per step
    const long long stride = (long long)gridDim.x * kOtsuThreads;
    const int sq = (int)(stride / groups), sr = (int)(stride - (long long)sq * groups);
    const long long g0 = (long long)blockIdx.x * kOtsuThreads + threadIdx.x;
    int y = (int)(g0 / groups), gx = (int)(g0 - (long long)y * groups);
    for (long long gi = g0; gi < total; gi += stride) {
        const int x = gx * 16;
        const uint8_t *row = src + (long long)y * pitch;
        uint8_t *drow = dst + (long long)y * dst_pitch;
        if (x + 16 <= w) {
            uint32_t g[4], m[4];
            load16<CIN>(row, x, g);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                m[q] = T == 0u ? 0xffffffffu : __vcmpgeu4(g[q], T4);
            if (packed) {
                uint32_t bits = 0; // bit j <-> pixel x + j: the msb of each byte
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    bits |= ((((m[q] >> 7) & 0x01010101u) * 0x01020408u) >> 24) << (4 * q);
                drow[x >> 3] = (uint8_t)bits;
                drow[(x >> 3) + 1] = (uint8_t)(bits >> 8);
            } else if (vec_ok) {
                *reinterpret_cast<uint4 *>(drow + x) = make_uint4(m[0], m[1], m[2], m[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    drow[x + j] = (uint8_t)(m[j >> 2] >> (8 * (j & 3)));
            }
        } else {
            uint32_t bits = 0;
            for (int xx = x; xx < w; ++xx) {
                const uint32_t f = gray_at<CIN>(row, xx);
                if (packed)
                    bits |= (f >= T ? 1u : 0u) << (xx - x);
                else
                    drow[xx] = f >= T ? 255 : 0;
            }
            if (packed) {
                drow[x >> 3] = (uint8_t)bits;
                if (w - x > 8)
                    drow[(x >> 3) + 1] = (uint8_t)(bits >> 8);
            }
        }
        gx += sr;
        y += sq;
        if (gx >= groups) {
            gx -= groups;
            ++y;
        }
    }
}

} // namespace

int launch_otsu(const uint8_t *d_src, size_t src_pitch, int h, int w, int ch, uint8_t *d_dst, size_t dst_pitch,
                int packed, void *d_scratch, cudaStream_t stream)
{
    int sms = 0;
    int rc = device_sm_count(&sms);
    if (rc != BNZ_OK)
        return rc;
    auto *hist = reinterpret_cast<unsigned long long *>(static_cast<uint8_t *>(d_scratch) + kHistOffset);
    int *T = reinterpret_cast<int *>(static_cast<uint8_t *>(d_scratch) + kTOffset);
    auto *done = reinterpret_cast<unsigned int *>(static_cast<uint8_t *>(d_scratch) + kDoneOffset);
    auto *parts = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(d_scratch) + kPartOffset);
    // the histogram, T, the CTA counter and the partial tables, from offset 0
    cudaError_t e = cudaMemsetAsync(d_scratch, 0, kPartOffset + kParts * 256 * sizeof(uint32_t), stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "clear histogram");
    const long long groups = (long long)((w + 15) / 16) * h;
    // a few CTAs per SM, grid-stride: every CTA merges one set of 256 bins
    const int grid = (int)std::max<long long>(1, std::min<long long>((long long)sms * 4,
                                                                      (groups + kOtsuThreads - 1) / kOtsuThreads));
    if (ch == 1)
        otsu_hist<1><<<grid, kOtsuThreads, 0, stream>>>(d_src, (long long)src_pitch, h, w, hist, parts, done, T);
    else
        otsu_hist<3><<<grid, kOtsuThreads, 0, stream>>>(d_src, (long long)src_pitch, h, w, hist, parts, done, T);
    const int vec_ok = ((reinterpret_cast<uintptr_t>(d_dst) | dst_pitch) & 15u) == 0 ? 1 : 0;
    if (ch == 1)
        otsu_mask<1><<<grid, kOtsuThreads, 0, stream>>>(d_src, (long long)src_pitch, h, w, T, d_dst,
                                                         (long long)dst_pitch, packed, vec_ok);
    else
        otsu_mask<3><<<grid, kOtsuThreads, 0, stream>>>(d_src, (long long)src_pitch, h, w, T, d_dst,
                                                         (long long)dst_pitch, packed, vec_ok);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "launch Otsu kernels");
    return BNZ_OK;
}

} // namespace bnz
