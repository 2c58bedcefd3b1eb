// decide.cuh -- per-pixel decision of Eq. 3 shared by the fused and the
// integral-image kernels: an fp32 filter whose error is bounded by
// decision_margin(), and the exact fp64 re-evaluation for pixels inside it.
#pragma once
#include <cstdint>

#include "internal.h"

namespace bnz {

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

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// V (< 2^48) as float: high word exact, low word rounded, one more rounding in
// the fma -- relative error <= 2u (u = 2^-24).  A 64-bit integer conversion
// would run on the fp64 pipe.
__device__ __forceinline__ float v_to_float(unsigned long long V)
{
    return __fmaf_rn(__uint2float_rn((uint32_t)(V >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)V));
}

// fp32 filter d ~ f - t, n = W*W (constants from the host in double, rounded once)
template <int RULE>
__device__ __forceinline__ float filter_int(float ff, float S1f, float sq, const FusedParams &p)
{
    if (RULE == BNZ_SAUVOLA)
        return __fmaf_rn(-S1f, __fmaf_rn(p.kRn2, sq, p.omkn), ff);
    return __fmaf_rn(-p.kn, sq, __fmaf_rn(-p.invn, S1f, ff));
}

// fp32 filter d ~ f - t for a pixel with its own n (invn ~ 1/n from rcp.approx)
template <int RULE>
__device__ __forceinline__ float filter_n(float ff, float S1f, float sq, float invn, const FusedParams &p)
{
    if (RULE == BNZ_SAUVOLA)
        return __fmaf_rn(-S1f, __fmaf_rn(__fmul_rn(__fmul_rn(p.kR, invn), invn), sq, __fmul_rn(p.omk, invn)), ff);
    return __fmaf_rn(-__fmul_rn(p.kf, invn), sq, __fmaf_rn(-invn, S1f, ff));
}

// The fp64 sequence of the definition, same order, no contraction.
// Returns g | 0x200 if |f - t| < 1e-9 (a tie).
template <int RULE>
__device__ __noinline__ uint32_t decide_fp64(uint32_t f, uint32_t n, uint32_t S1, uint32_t S2, const FusedParams &p)
{
    const unsigned long long V = (unsigned long long)n * S2 - (unsigned long long)S1 * S1;
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
    return (fd < td ? 0u : 255u) | tie;
}

} // namespace bnz

namespace bnz {

// Eq. 3 for one pixel with exact window sums: fp32 filter, fp64 when inside
// the margin.  Counts fp64 evaluations and ties.
template <int RULE>
__device__ __forceinline__ uint32_t decide_pixel(uint32_t f, uint32_t n, uint32_t S1, uint32_t S2,
                                                 const FusedParams &p, uint32_t &nfb, uint32_t &nties)
{
    const unsigned long long V = (unsigned long long)n * S2 - (unsigned long long)S1 * S1;
    const float sq = sqrt_approx(v_to_float(V));
    const float ff = __uint2float_rn(f), S1f = __uint2float_rn(S1);
    const float d = (n == p.nW) ? filter_int<RULE>(ff, S1f, sq, p)
                                : filter_n<RULE>(ff, S1f, sq, rcp_approx(__uint2float_rn(n)), p);
    if (fabsf(d) >= p.E)
        return d < 0.0f ? 0u : 255u;
    const uint32_t r = decide_fp64<RULE>(f, n, S1, S2, p);
    ++nfb;
    nties += (r >> 9) & 1u;
    return r & 0xffu;
}

// Eq. 1, integer round-half-up, for one pixel at p[0..2] = r, g, b.
__device__ __forceinline__ uint32_t gray_rgb(const uint8_t *px)
{
    return (299u * px[0] + 587u * px[1] + 114u * px[2] + 500u) / 1000u;
}

} // namespace bnz
