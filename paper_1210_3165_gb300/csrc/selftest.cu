// selftest.cu -- device checks of the hardware approximations the fused
// kernel's error bound relies on (the relative errors of sqrt.approx.f32 and
// rcp.approx.f32), of its bounded wait, and of its Eq. 1 conversion.
#include <cstring>

#include "internal.h"
#include "ptx.cuh"
#include "segment.cuh"

namespace bnz {
namespace {

__global__ void sqrt_approx_err_kernel(uint32_t first_bits, uint64_t count, unsigned int *max_err_bits)
{
    float worst = 0.0f;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const float x = __uint_as_float(first_bits + (uint32_t)i);
        float a;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(a) : "f"(x));
        // r is the correctly rounded root (|r - sqrt(x)| <= 2^-24 r); the caller adds 2^-24
        const float r = __fsqrt_rn(x);
        worst = fmaxf(worst, __fdiv_rn(fabsf(a - r), r));
    }
    for (int off = 16; off; off >>= 1)
        worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, off));
    if ((threadIdx.x & 31) == 0)
        atomicMax(max_err_bits, __float_as_uint(worst)); // non-negative floats order like their bits
}

// Eq. 1 exactly as the fused kernel's producers apply it: four pixels (12
// interleaved bytes) per gray4 call, a last partial group through gray1.
__global__ void gray_kernel(const uint8_t *rgb, size_t npix, uint8_t *gray)
{
    const size_t groups = npix / 4;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += stride) {
        const uint8_t *s = rgb + 12 * g;
        const uint32_t w0 = s[0] | (s[1] << 8) | (s[2] << 16) | ((uint32_t)s[3] << 24);
        const uint32_t w1 = s[4] | (s[5] << 8) | (s[6] << 16) | ((uint32_t)s[7] << 24);
        const uint32_t w2 = s[8] | (s[9] << 8) | (s[10] << 16) | ((uint32_t)s[11] << 24);
        const uint32_t q = gray4(w0, w1, w2);
        gray[4 * g] = (uint8_t)q;
        gray[4 * g + 1] = (uint8_t)(q >> 8);
        gray[4 * g + 2] = (uint8_t)(q >> 16);
        gray[4 * g + 3] = (uint8_t)(q >> 24);
    }
    if (blockIdx.x == 0 && threadIdx.x < npix - 4 * groups) {
        const size_t i = 4 * groups + threadIdx.x;
        const uint8_t *s = rgb + 3 * i;
        gray[i] = (uint8_t)gray1(s[0] | (s[1] << 8) | (s[2] << 16));
    }
}

__global__ void rcp_approx_err_kernel(uint32_t n_lo, uint32_t n_hi, unsigned int *max_err_bits)
{
    float worst = 0.0f;
    for (uint32_t n = n_lo + blockIdx.x * blockDim.x + threadIdx.x; n < n_hi; n += gridDim.x * blockDim.x) {
        const float x = __uint2float_rn(n); // exact for n < 2^24
        float a;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(a) : "f"(x));
        const float r = __frcp_rn(x); // correctly rounded 1/n
        worst = fmaxf(worst, __fdiv_rn(fabsf(a - r), r));
    }
    for (int off = 16; off; off >>= 1)
        worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, off));
    if ((threadIdx.x & 31) == 0)
        atomicMax(max_err_bits, __float_as_uint(worst));
}

// One thread waits, with the kernels' bounded wait, for the first phase of an
// mbarrier that expects one arrival; when `arrive` is 0 nothing ever arrives.
// out[0] = 1 if the wait gave up, out[1] = cycles spent waiting.
__global__ void wait_timeout_kernel(long long limit, int arrive, long long *out)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (arrive)
            mbar_arrive(&bar);
        const long long t0 = clock64();
        const bool ok = mbar_wait_bounded(&bar, 0u, limit);
        out[1] = clock64() - t0;
        out[0] = ok ? 0 : 1;
    }
}

} // namespace
} // namespace bnz

extern "C" BNZ_API int bnz_selftest_wait_timeout(long long limit_cycles, int arrive, int *timed_out,
                                                 long long *waited_cycles)
{
    using namespace bnz;
    if (!timed_out || limit_cycles < 0 || limit_cycles > 4000000000ll)
        return fail(BNZ_EINVAL, "need 0 <= limit_cycles <= 4e9 and a result pointer");
    long long *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * sizeof(long long));
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(selftest)");
    long long h[2] = {-1, -1};
    do {
        wait_timeout_kernel<<<1, 32>>>(limit_cycles, arrive ? 1 : 0, d);
        if ((e = cudaGetLastError()) != cudaSuccess)
            break;
        if ((e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost)) != cudaSuccess)
            break;
    } while (0);
    cudaFree(d);
    if (e != cudaSuccess)
        return cuda_fail(e, "wait self-test");
    *timed_out = (int)h[0];
    if (waited_cycles)
        *waited_cycles = h[1];
    return BNZ_OK;
}

extern "C" BNZ_API int bnz_selftest_rcp_approx(unsigned int n_lo, unsigned int n_hi, double *max_rel_err)
{
    using namespace bnz;
    if (!max_rel_err || n_lo < 1 || n_hi <= n_lo || n_hi > (1u << 24))
        return fail(BNZ_EINVAL, "need 1 <= n_lo < n_hi <= 2^24 and a result pointer");
    unsigned int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned int));
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(selftest)");
    unsigned int h = 0;
    do {
        if ((e = cudaMemset(d, 0, sizeof(unsigned int))) != cudaSuccess)
            break;
        rcp_approx_err_kernel<<<304, 256>>>(n_lo, n_hi, d);
        if ((e = cudaGetLastError()) != cudaSuccess)
            break;
        if ((e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost)) != cudaSuccess)
            break;
    } while (0);
    cudaFree(d);
    if (e != cudaSuccess)
        return cuda_fail(e, "rcp.approx self-test");
    float f;
    memcpy(&f, &h, 4);
    *max_rel_err = (double)f * (1.0 + 1e-6) + 1.0 / 16777216.0; // bound vs the exact reciprocal
    return BNZ_OK;
}

extern "C" BNZ_API int bnz_selftest_sqrt_approx(float lo, float hi, double *max_rel_err)
{
    using namespace bnz;
    if (!max_rel_err || !(lo > 0.0f) || !(hi > lo))
        return fail(BNZ_EINVAL, "need 0 < lo < hi and a result pointer");
    unsigned int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned int));
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(selftest)");
    unsigned int h = 0;
    do {
        if ((e = cudaMemset(d, 0, sizeof(unsigned int))) != cudaSuccess)
            break;
        uint32_t a, b;
        memcpy(&a, &lo, 4);
        memcpy(&b, &hi, 4);
        sqrt_approx_err_kernel<<<1216, 256>>>(a, (uint64_t)(b - a), d);
        if ((e = cudaGetLastError()) != cudaSuccess)
            break;
        if ((e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost)) != cudaSuccess)
            break;
    } while (0);
    cudaFree(d);
    if (e != cudaSuccess)
        return cuda_fail(e, "sqrt.approx self-test");
    float f;
    memcpy(&f, &h, 4);
    *max_rel_err = (double)f * (1.0 + 1e-6) + 1.0 / 16777216.0; // bound vs the exact root
    return BNZ_OK;
}

extern "C" BNZ_API int bnz_selftest_gray(const uint8_t *d_rgb, size_t npix, uint8_t *d_gray, void *stream)
{
    using namespace bnz;
    if (!d_rgb || !d_gray || npix == 0)
        return fail(BNZ_EINVAL, "bnz_selftest_gray: null pointer or no pixels");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(BNZ_ENODEV, "no CUDA device available; this library has no CPU path");
    }
    gray_kernel<<<1216, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_rgb, npix, d_gray);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "gray self-test");
    return BNZ_OK;
}

// The fused kernel's abort path, made to run: every wait of the producers and
// of the TMA issuer gives up as soon as its phase is not already complete
// (so the first wait for a copy still in flight gives up), while the issuer's
// final wait for its copies in flight keeps the normal limit, so no CTA exits
// with a copy outstanding.  The CTAs that gave up count themselves in
// d_stats[2] (and the library's error word); the call synchronizes `stream`
// and returns BNZ_ETIMEOUT if any did, as the host-pointer calls do.
extern "C" BNZ_API int bnz_selftest_fused_timeout(const uint8_t *d_src, size_t src_pitch, int height, int width,
                                                  int channels, int W, int rule, double k, double R, uint8_t *d_dst,
                                                  size_t dst_pitch, void *stream, unsigned long long *d_stats)
{
    using namespace bnz;
    int rc = check_common(d_src, src_pitch, height, width, channels, W, rule, k, R, d_dst, dst_pitch, 0);
    if (rc != BNZ_OK)
        return rc;
    if (!d_stats)
        return fail(BNZ_EINVAL, "bnz_selftest_fused_timeout: d_stats is required");
    if ((reinterpret_cast<uintptr_t>(d_src) & 15u) || (src_pitch & 15u))
        return fail(BNZ_EINVAL, "d_src must be 16-byte aligned with src_pitch a multiple of 16 (TMA)");
    unsigned int *err = nullptr;
    rc = device_err_flag(&err);
    if (rc != BNZ_OK)
        return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = launch_fused(d_src, src_pitch, height, width, channels, W, rule, k, rule == BNZ_NIBLACK ? 1.0 : R,
                      d_dst, dst_pitch, 0, nullptr, s, d_stats, err, 0, -1, true, 0);
    if (rc != BNZ_OK)
        return rc;
    unsigned long long st[4] = {0, 0, 0, 0};
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
        e = cudaMemcpy(st, d_stats, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(e, "fused timeout self-test");
    if (st[BNZ_STATS_TIMEOUTS])
        return fail(BNZ_ETIMEOUT, "%llu CTAs gave up a wait (self-test of the abort path)", st[BNZ_STATS_TIMEOUTS]);
    return BNZ_OK;
}
