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
//   otsu_select  one CTA of 256 threads, thread t evaluates q(t); a block
//                reduction takes the argmax and stores T in the scratch;
//   otsu_mask    Eq. 2 with T read from the scratch: byte or packed mask.
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

// Gray values of the 8 pixels starting at column x of row `row` (x + 8 <= w):
// 8 bytes (gray) or 24 bytes (RGB) from a 16-byte aligned row start.
template <int CIN>
__device__ __forceinline__ void load8(const uint8_t *row, int x, uint32_t &g0, uint32_t &g1)
{
    if (CIN == 1) {
        const uint2 v = *reinterpret_cast<const uint2 *>(row + x);
        g0 = v.x;
        g1 = v.y;
    } else {
        const uint32_t *p = reinterpret_cast<const uint32_t *>(row + 3 * x);
        g0 = gray4(p[0], p[1], p[2]);
        g1 = gray4(p[3], p[4], p[5]);
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
    const int groups = (w + 7) / 8; // 8-pixel groups per row
    const long long total = (long long)groups * h;
    for (long long gi = (long long)blockIdx.x * kOtsuThreads + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * kOtsuThreads) {
        const int y = (int)(gi / groups);
        const int x = (int)(gi - (long long)y * groups) * 8;
        const uint8_t *row = src + (long long)y * pitch;
        if (x + 8 <= w) {
            uint32_t g0, g1;
            load8<CIN>(row, x, g0, g1);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                atomicAdd(&mine[(g0 >> (8 * j)) & 0xffu], 1u);
                atomicAdd(&mine[(g1 >> (8 * j)) & 0xffu], 1u);
            }
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
    __shared__ unsigned long long sn[256], ss[256];
    __shared__ double sq[kOtsuThreads / 32];
    __shared__ int st[kOtsuThreads / 32];
    const int t = threadIdx.x;
    sn[t] = hist[t];
    ss[t] = hist[t] * (unsigned long long)t;
    __syncthreads();
    // totals and the prefixes below t (levels 0 .. t-1), 64-bit exact (N <= 2^28)
    unsigned long long N = 0, S = 0, n0 = 0, s0 = 0;
    for (int i = 0; i < 256; ++i) {
        N += sn[i];
        S += ss[i];
        if (i < t) {
            n0 += sn[i];
            s0 += ss[i];
        }
    }
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
    const int groups = (w + 7) / 8;
    const long long total = (long long)groups * h;
    for (long long gi = (long long)blockIdx.x * kOtsuThreads + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * kOtsuThreads) {
        const int y = (int)(gi / groups);
        const int x = (int)(gi - (long long)y * groups) * 8;
        const uint8_t *row = src + (long long)y * pitch;
        uint8_t *drow = dst + (long long)y * dst_pitch;
        if (x + 8 <= w) {
            uint32_t g0, g1;
            load8<CIN>(row, x, g0, g1);
            uint32_t bits = 0; // bit j <-> pixel x + j, 1 <-> 255 (Eq. 2: f >= T)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                bits |= (((g0 >> (8 * j)) & 0xffu) >= T ? 1u : 0u) << j;
                bits |= (((g1 >> (8 * j)) & 0xffu) >= T ? 1u : 0u) << (j + 4);
            }
            if (packed) {
                drow[x >> 3] = (uint8_t)bits;
            } else {
                // bit j -> byte j of 0x00 / 0xFF
                const uint32_t lo = ((bits & 15u) * 0x00204081u & 0x01010101u) * 0xffu;
                const uint32_t hi = ((bits >> 4) * 0x00204081u & 0x01010101u) * 0xffu;
                if (vec_ok) {
                    *reinterpret_cast<uint2 *>(drow + x) = make_uint2(lo, hi);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        drow[x + j] = (uint8_t)(lo >> (8 * j));
                        drow[x + 4 + j] = (uint8_t)(hi >> (8 * j));
                    }
                }
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
            if (packed)
                drow[x >> 3] = (uint8_t)bits;
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
    const long long groups = (long long)((w + 7) / 8) * h;
    // a few CTAs per SM, grid-stride: every CTA merges one set of 256 bins
    const int grid = (int)std::max<long long>(1, std::min<long long>((long long)sms * 4,
                                                                      (groups + kOtsuThreads - 1) / kOtsuThreads));
    if (ch == 1)
        otsu_hist<1><<<grid, kOtsuThreads, 0, stream>>>(d_src, (long long)src_pitch, h, w, hist);
    else
        otsu_hist<3><<<grid, kOtsuThreads, 0, stream>>>(d_src, (long long)src_pitch, h, w, hist);
    otsu_select<<<1, kOtsuThreads, 0, stream>>>(hist, T);
    const int vec_ok = ((reinterpret_cast<uintptr_t>(d_dst) | dst_pitch) & 7u) == 0 ? 1 : 0;
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
