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
// Three launches on the caller's stream, no host round trip:
//   otsu_hist    the histogram: 8 warp-private 256-bin tables in shared memory
//                per CTA, merged into the caller's scratch with 64-bit atomics;
//                each thread takes 16 pixels per step (128-bit loads);
//   otsu_select  one CTA of 256 threads: a block scan gives every thread t the
//                exact prefixes n0, s0 of the levels below t, thread t
//                evaluates q(t), a block reduction takes the argmax and stores
//                T in the scratch;
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

template <int CIN>
__device__ __forceinline__ uint32_t gray_at(const uint8_t *row, int x)
{
    if (CIN == 1)
        return row[x];
    const uint8_t *px = row + 3 * x;
    return gray1((uint32_t)px[0] | ((uint32_t)px[1] << 8) | ((uint32_t)px[2] << 16));
}

template <int CIN>
__global__ void __launch_bounds__(kOtsuThreads)
    otsu_hist(const uint8_t *src, long long pitch, int h, int w, unsigned long long *hist)
{
    __shared__ uint32_t sh[kOtsuThreads / 32][256];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (kOtsuThreads / 32) * 256; i += kOtsuThreads)
        (&sh[0][0])[i] = 0;
    __syncthreads();
    uint32_t *mine = sh[warp];
    const int groups = (w + 15) / 16; // 16-pixel groups per row
    const long long total = (long long)groups * h;
    for (long long gi = (long long)blockIdx.x * kOtsuThreads + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * kOtsuThreads) {
        const int y = (int)(gi / groups);
        const int x = (int)(gi - (long long)y * groups) * 16;
        const uint8_t *row = src + (long long)y * pitch;
        if (x + 16 <= w) {
            uint32_t g[4];
            load16<CIN>(row, x, g);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    atomicAdd(&mine[(g[q] >> (8 * j)) & 0xffu], 1u);
        } else {
            for (int xx = x; xx < w; ++xx)
                atomicAdd(&mine[gray_at<CIN>(row, xx)], 1u);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += kOtsuThreads) {
        unsigned long long c = 0;
#pragma unroll
        for (int k = 0; k < kOtsuThreads / 32; ++k)
            c += sh[k][b];
        if (c)
            atomicAdd(&hist[b], c);
    }
}

__global__ void __launch_bounds__(kOtsuThreads) otsu_select(const unsigned long long *hist, int *T_out)
{
    __shared__ unsigned long long wn[kOtsuThreads / 32], ws[kOtsuThreads / 32], tot[2];
    __shared__ double sq[kOtsuThreads / 32];
    __shared__ int st[kOtsuThreads / 32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const unsigned long long c = hist[t], v = c * (unsigned long long)t;
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
    otsu_mask(const uint8_t *src, long long pitch, int h, int w, const int *T_in, uint8_t *dst, long long dst_pitch,
              int packed, int vec_ok)
{
    const uint32_t T = (uint32_t)*T_in;
    // byte-wise f >= T for four packed gray values: __vcmpgeu4 gives 0xFF / 0x00 per byte
    const uint32_t T4 = T > 255u ? 0u : T * 0x01010101u;
    const int groups = (w + 15) / 16;
    const long long total = (long long)groups * h;
    for (long long gi = (long long)blockIdx.x * kOtsuThreads + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * kOtsuThreads) {
        const int y = (int)(gi / groups);
        const int x = (int)(gi - (long long)y * groups) * 16;
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
    cudaError_t e = cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned long long), stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "clear histogram");
    const long long groups = (long long)((w + 15) / 16) * h;
    // a few CTAs per SM, grid-stride: every CTA merges one set of 256 bins
    const int grid = (int)std::max<long long>(1, std::min<long long>((long long)sms * 4,
                                                                      (groups + kOtsuThreads - 1) / kOtsuThreads));
    if (ch == 1)
        otsu_hist<1><<<grid, kOtsuThreads, 0, stream>>>(d_src, (long long)src_pitch, h, w, hist);
    else
        otsu_hist<3><<<grid, kOtsuThreads, 0, stream>>>(d_src, (long long)src_pitch, h, w, hist);
    otsu_select<<<1, kOtsuThreads, 0, stream>>>(hist, T);
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
