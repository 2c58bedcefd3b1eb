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

// ---- double-float (two fp32 words, value = hi + lo) helpers ------------------
// Explicit round-to-nearest intrinsics throughout: contraction into fma would
// change the error terms.  u = 2^-24.

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) // exact: a + b = s + e
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) // exact when |a| >= |b| or a == 0
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add(df a, df b) // relative error <= 4u^2 (no cancellation assumed)
{
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_mul(df a, df b) // relative error <= 6u^2
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p); // exact product error
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return fast_two_sum(p, e);
}

// x / n for exact fp32 x and integer n < 2^24: q = RN(x/n), the remainder
// x - q n is exact (fma), the correction is rounded once (relative u^2 error)
__device__ __forceinline__ df df_div_int(df x, float nf)
{
    const float q = __fdiv_rn(x.hi, nf);
    const float r = __fmaf_rn(-q, nf, x.hi);
    return fast_two_sum(q, __fdiv_rn(__fadd_rn(r, x.lo), nf));
}

// sqrt(V) for 0 <= V < 2^48 (V = hi 2^32 + lo): V in double-float from three
// exact pieces, then one Newton correction of the rounded root
__device__ __forceinline__ df df_sqrt_v(unsigned long long V)
{
    const uint32_t h = (uint32_t)(V >> 32), lo = (uint32_t)V;
    const df a = two_sum(__fmul_rn(__uint2float_rn(h), 4294967296.0f), __uint2float_rn(lo >> 16) * 65536.0f);
    const df v = fast_two_sum(a.hi, __fadd_rn(a.lo, __uint2float_rn(lo & 0xffffu)));
    if (v.hi == 0.0f)
        return {0.0f, 0.0f};
    const float sh = __fsqrt_rn(v.hi);
    const float p = __fmul_rn(sh, sh);
    const float pe = __fmaf_rn(sh, sh, -p);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(v.hi, p), pe), v.lo); // V - sh^2, to rounding
    return fast_two_sum(sh, __fdiv_rn(r, __fmul_rn(2.0f, sh)));
}

// Eq. 3 for a pixel the fp32 filter could not decide.  f - t in double-float
// (Niblack t = m + k s; Sauvola t = m (1-k) + m s (k/R), m = S1/n, s = sqrt(V)/n),
// whose absolute error the host bounds from k and R (double_float_error; below
// 1e-10 for the usual |k| <= 1, R >= 64).  When it is farther than p.Tdf =
// 1e-9 + that bound + the fp64 definition's own error from zero, the fp64
// definition sees no tie and the same sign, so the sign decides; otherwise the
// fp64 sequence of the definition decides (and counts the tie).
template <int RULE>
__device__ uint32_t decide_exact(uint32_t f, uint32_t n, uint32_t S1, uint32_t S2, const FusedParams &p)
{
    const unsigned long long V = (unsigned long long)n * S2 - (unsigned long long)S1 * S1;
    const float nf = __uint2float_rn(n);
    const df m = df_div_int({__uint2float_rn(S1), 0.0f}, nf);
    const df sv = df_sqrt_v(V);
    const df sd = df_div_int(sv, nf);
    df t;
    if (RULE == BNZ_SAUVOLA)
        t = df_add(df_mul(m, {p.c1h, p.c1l}), df_mul(df_mul(m, sd), {p.c2h, p.c2l}));
    else
        t = df_add(m, df_mul({p.kh, p.kl}, sd));
    const df d = df_add({__uint2float_rn(f), 0.0f}, {-t.hi, -t.lo});
    const float dv = __fadd_rn(d.hi, d.lo);
    if (fabsf(dv) > p.Tdf)
        return dv < 0.0f ? 0u : 255u;
    return decide_fp64<RULE>(f, n, S1, S2, p);
}

// Eq. 3 for a pixel inside the fp32 filter's margin.  Niblack first tries a
// tighter fp32 evaluation of X = n (f - t) = (n f - S1) - k sqrt(V):
//   A = n f - S1 is an exact integer below 2^24 in magnitude, so exact in fp32;
//   r = RN(sqrt(RN2(V))) = sqrt(V) (1 + d), |d| <= 2.001u (V to fp32 within 2u,
//   halved by the root, then the root's own rounding); C = RN(RN(k) r) =
//   k sqrt(V) (1 + e), |e| <= 4.01u; D = RN(A - C), so |D - X| <= 4.01u |k| sqrt(V)
//   (1 + u) + u |X|.  With tau = 1e-9 + the fp64 definition's error, |D| > 4.5u
//   |k| r + 1.01 tau n (p.rk, p.rt) gives |f - t| = |X| / n > tau: no tie in the
//   definition and the sign of D.  The rest (and every Sauvola pixel, whose t =
//   m (1 - k + k s / R) scales with m |k| and leaves no such gain) take the
//   double-float and fp64 stages.
template <int RULE>
__device__ __forceinline__ uint32_t decide_refine(uint32_t f, uint32_t n, uint32_t S1, uint32_t S2,
                                                  const FusedParams &p)
{
    if (RULE == BNZ_NIBLACK) {
        const int A = (int)(n * f) - (int)S1;
        const unsigned long long V = (unsigned long long)n * S2 - (unsigned long long)S1 * S1;
        const float r = __fsqrt_rn(v_to_float(V));
        const float D = __fsub_rn(__int2float_rn(A), __fmul_rn(p.kf, r));
        const float bnd = __fmaf_rn(p.rk, r, __fmul_rn(p.rt, __uint2float_rn(n)));
        if (fabsf(D) > bnd)
            return D < 0.0f ? 0u : 255u;
    }
    return decide_exact<RULE>(f, n, S1, S2, p);
}

} // namespace bnz

namespace bnz {

// Eq. 3 for one pixel with exact window sums: fp32 filter, double-float and
// then fp64 when inside the margin.  Counts re-evaluated pixels and ties.
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
    const uint32_t r = decide_exact<RULE>(f, n, S1, S2, p);
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
