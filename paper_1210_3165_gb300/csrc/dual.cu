// dual.cu -- both threshold rules from one pass over the window sums.
//
// Sauvola (Eq. 4) and Niblack share everything up to the threshold: the gray
// page f (Eq. 1), the exact window sums S1 = sum f, S2 = sum f^2 and V =
// n*S2 - S1^2, hence m and s.  A caller that wants both masks of a page for one
// W (as when the two rules are compared) gets them here for one read of the
// page and one set of sums: the producers are the fused kernel's own
// (produce<CIN>), the consumers form the horizontal sums as in the fused kernel
// and then take the Eq. 3 decision twice, with each rule's fp32 filter, margin
// and exact re-evaluation.  Each mask equals, bit for bit, the one the
// single-rule kernel writes.
#include <cmath>

#include "segment.cuh"

namespace bnz {
namespace {

// The lane's 16 fp32 filters of one rule in the pixels whose |d| lies inside
// the rule's margin: the exact decision (double-float, then fp64 near ties)
// for those pixels, patched into the lane's output words.  Counts re-evaluated
// pixels and ties.
template <int RULE, int KO, int KI>
__device__ __forceinline__ void fix_margin(const FusedParams &p, const uint32_t *C1, const uint32_t *C2, int ao,
                                           int ai, uint32_t base1, uint32_t base2, const uint32_t (&fw)[4], int y,
                                           int xg0, uint32_t (&outw)[4], uint32_t &nfb, uint32_t &nties)
{
    const int nr = min(y + p.r_hi, p.h - 1) - max(y - p.r_lo, 0) + 1;
    uint32_t e1[L], e2[L], t1, t2;
    lane_deltas<KO, KI>(C1, C2, ao, ai, e1, e2, t1, t2);
    uint32_t amask = 0;
#pragma unroll
    for (int t = 0; t < L; ++t) {
        const int xg = xg0 + t;
        const int nc = min(xg + p.r_hi, p.w - 1) - max(xg - p.r_lo, 0) + 1;
        const uint32_t n = (uint32_t)(nr * nc);
        const uint32_t S1 = base1 + e1[t], S2 = base2 + e2[t];
        const unsigned long long V = (unsigned long long)n * S2 - (unsigned long long)S1 * S1;
        const float ff = byte_float(fw[t >> 2], t & 3);
        const float sq = sqrt_approx(v_to_float(V));
        const float d = (n == p.nW) ? filter_int<RULE>(ff, __uint2float_rn(S1), sq, p)
                                    : filter_n<RULE>(ff, __uint2float_rn(S1), sq, rcp_approx(__uint2float_rn(n)), p);
        if (xg < p.w && fabsf(d) < p.E)
            amask |= 1u << t;
    }
    uint32_t white = 0;
    for (uint32_t m = amask; m; m &= m - 1) {
        const int t = __ffs(m) - 1;
        uint32_t S1 = base1, S2 = base2, word = fw[0];
#pragma unroll
        for (int u = 0; u < L; ++u)
            if (u == t) {
                S1 += e1[u];
                S2 += e2[u];
            }
#pragma unroll
        for (int qq = 1; qq < 4; ++qq)
            if ((t >> 2) == qq)
                word = fw[qq];
        const uint32_t f = (word >> (8 * (t & 3))) & 0xffu;
        const int xg = xg0 + t;
        const int nc = min(xg + p.r_hi, p.w - 1) - max(xg - p.r_lo, 0) + 1;
        const uint32_t r = decide_exact<RULE>(f, (uint32_t)(nr * nc), S1, S2, p);
        ++nfb;
        nties += (r >> 9) & 1u;
        white |= (r & 1u) << t;
    }
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
        const uint32_t mm = ((((amask >> (4 * qq)) & 15u) * 0x00204081u) & 0x01010101u) * 0xffu;
        const uint32_t vv = ((((white >> (4 * qq)) & 15u) * 0x00204081u) & 0x01010101u) * 0xffu;
        outw[qq] = (outw[qq] & ~mm) | (vv & mm);
    }
}

// The lane's 16 outputs of row y into p.dst: byte mask or packed bits.
__device__ __forceinline__ void store_lane(const FusedParams &p, int y, int xg0, const uint32_t (&outw)[4])
{
    if (!p.packed) {
        uint8_t *drow = p.dst + (size_t)y * p.dst_pitch + xg0;
        if (p.vec_ok && xg0 + L <= p.w) {
            *reinterpret_cast<uint4 *>(drow) = make_uint4(outw[0], outw[1], outw[2], outw[3]);
        } else {
#pragma unroll
            for (int t = 0; t < L; ++t)
                if (xg0 + t < p.w)
                    drow[t] = (uint8_t)byte_dyn(outw[t >> 2], t & 3);
        }
    } else {
        uint32_t bits = 0; // bit t <-> pixel xg0 + t: the msb of each byte
#pragma unroll
        for (int qq = 0; qq < 4; ++qq)
            bits |= ((((outw[qq] >> 7) & 0x01010101u) * 0x01020408u) >> 24) << (4 * qq);
        const int valid = p.w - xg0;
        if (valid < L)
            bits &= (1u << valid) - 1u;
        uint8_t *drow = p.dst + (size_t)y * p.dst_pitch + (xg0 >> 3);
        drow[0] = (uint8_t)(bits & 0xffu);
        if (valid > 8)
            drow[1] = (uint8_t)(bits >> 8);
    }
}

// byte = 0xFF where d >= +0, 0x00 where d < 0 (sign bit replicated)
__device__ __forceinline__ uint32_t mask_word(const float (&dd)[4])
{
    const uint32_t lo = prmt(__float_as_uint(dd[0]), __float_as_uint(dd[1]), 0xFBu);
    const uint32_t hi = prmt(__float_as_uint(dd[2]), __float_as_uint(dd[3]), 0xFBu);
    return ~prmt(lo, hi, 0x5410u);
}

// Consumers of the dual kernel: horizontal sums as in consume(), then the
// Sauvola decision (constants in ps, mask to ps.dst) and the Niblack one
// (pn, mask to pn.dst).
template <int CIN, int WM8>
__device__ __forceinline__ void consume_dual(const FusedParams &ps, const FusedParams &pn, const Segment &sg,
                                             uint8_t *smem, uint32_t &nfb, uint32_t &nties_s, uint32_t &nties_n,
                                             volatile int *s_abort)
{
    const FusedParams &p = ps; // geometry, shared by both rules
    const int SWP = p.SWP;
    constexpr int KO = (4 - ((WM8 >> 1) & 3)) & 3;
    constexpr int KI = (KO + WM8) & 3;
    const uint8_t *ring = smem + p.off_ring;
    const uint32_t *cb = reinterpret_cast<const uint32_t *>(smem + p.off_cb);
    const int q = threadIdx.x - NTP;
    const int lane = q & 31, ii = q >> 5;
    const int W = p.W;
    const bool active = lane * L < p.TW;
    const int fcol = active ? lane * L + p.o + p.r_lo : 0;
    const uint8_t *fbase = ring + fcol;
    const int xg0 = sg.x0 + lane * L;
    const bool xclip = xg0 < p.r_lo || xg0 + L - 1 + p.r_hi > p.w - 1;

    int rc = (ii + p.r_lo) % p.ring_rows;
    for (int k = 0; k < sg.nk; ++k, rc = (rc + CH < p.ring_rows) ? rc + CH : rc + CH - p.ring_rows) {
        const int b = k & 1;
        bar_sync(BAR_FULL + b, NTX);
        const int rows_k = min(CH, sg.th_eff - k * CH);
        if (ii < rows_k && !*s_abort) {
            const int y = sg.y0 + k * CH + ii;
            const uint32_t *C1 = cb + (size_t)(2 * b) * CH * p.RSW + ii * p.RSW;
            const uint32_t *C2 = C1 + (size_t)CH * p.RSW;
            const int cw = lane * L + p.o;
            const int ao = cw >> 2, ai = (cw + W) >> 2;

            uint32_t d1[L], d2[L];
            uint32_t a1 = 0, a2 = 0;
            if (active) {
                lane_deltas<KO, KI>(C1, C2, ao, ai, d1, d2, a1, a2);
            } else {
#pragma unroll
                for (int t = 0; t < L; ++t)
                    d1[t] = d2[t] = 0u;
            }
            uint32_t s1 = 0, s2 = 0;
            for (int c = p.o + lane; c < p.o + W; c += 32) {
                const int qc = cpos(c);
                s1 += C1[qc];
                s2 += C2[qc];
            }
            s1 = __reduce_add_sync(0xffffffffu, s1);
            s2 = __reduce_add_sync(0xffffffffu, s2);
            uint32_t x1 = a1, x2 = a2;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t t1 = __shfl_up_sync(0xffffffffu, x1, off);
                const uint32_t t2 = __shfl_up_sync(0xffffffffu, x2, off);
                if (lane >= off) {
                    x1 += t1;
                    x2 += t2;
                }
            }
            const uint32_t base1 = s1 + x1 - a1, base2 = s2 + x2 - a2;

            const uint4 fv = *reinterpret_cast<const uint4 *>(fbase + (size_t)rc * SWP);
            const uint32_t fw[4] = {fv.x, fv.y, fv.z, fv.w};
            const bool yclip = (y < p.r_lo) || (y + p.r_hi > p.h - 1);
            const bool lane_clip = active && xg0 < p.w && (yclip || xclip);
            uint32_t outs[4], outn[4];
            float mns = INFINITY, mnn = INFINITY;
            if (!__any_sync(0xffffffffu, lane_clip)) {
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    float ds[4], dn[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int t = 4 * qq + e;
                        const uint32_t S1 = base1 + d1[t];
                        const uint32_t S2 = base2 + d2[t];
                        const unsigned long long V =
                            (unsigned long long)p.nW * S2 - (unsigned long long)S1 * S1;
                        const float ff = byte_float(fw[qq], e);
                        const float S1f = __uint2float_rn(S1);
                        const float sq = sqrt_approx(v_to_float(V));
                        ds[e] = filter_int<BNZ_SAUVOLA>(ff, S1f, sq, ps);
                        dn[e] = filter_int<BNZ_NIBLACK>(ff, S1f, sq, pn);
                        mns = fminf(mns, fabsf(ds[e]));
                        mnn = fminf(mnn, fabsf(dn[e]));
                    }
                    outs[qq] = mask_word(ds);
                    outn[qq] = mask_word(dn);
                }
            } else {
                const int nr = min(y + p.r_hi, p.h - 1) - max(y - p.r_lo, 0) + 1;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    float ds[4], dn[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int t = 4 * qq + e;
                        const int xg = xg0 + t;
                        const int nc = min(xg + p.r_hi, p.w - 1) - max(xg - p.r_lo, 0) + 1;
                        const uint32_t n = (uint32_t)(nr * nc);
                        const uint32_t S1 = base1 + d1[t], S2 = base2 + d2[t];
                        const unsigned long long V = (unsigned long long)n * S2 - (unsigned long long)S1 * S1;
                        const float ff = byte_float(fw[qq], e);
                        const float S1f = __uint2float_rn(S1);
                        const float invn = rcp_approx(__uint2float_rn(n));
                        const float sq = sqrt_approx(v_to_float(V));
                        ds[e] = filter_n<BNZ_SAUVOLA>(ff, S1f, sq, invn, ps);
                        dn[e] = filter_n<BNZ_NIBLACK>(ff, S1f, sq, invn, pn);
                        mns = fminf(mns, xg < p.w ? fabsf(ds[e]) : INFINITY);
                        mnn = fminf(mnn, xg < p.w ? fabsf(dn[e]) : INFINITY);
                    }
                    outs[qq] = mask_word(ds);
                    outn[qq] = mask_word(dn);
                }
            }
            // rare: values inside a rule's fp32 margin take that rule's exact path
            if (mns < ps.E && active)
                fix_margin<BNZ_SAUVOLA, KO, KI>(ps, C1, C2, ao, ai, base1, base2, fw, y, xg0, outs, nfb, nties_s);
            if (mnn < pn.E && active)
                fix_margin<BNZ_NIBLACK, KO, KI>(pn, C1, C2, ao, ai, base1, base2, fw, y, xg0, outn, nfb, nties_n);
            if (active && xg0 < p.w) {
                store_lane(ps, y, xg0, outs);
                store_lane(pn, y, xg0, outn);
            }
        }
        if (k + 2 < sg.nk)
            bar_arrive(BAR_EMPTY + b, NTX);
    }
}

template <int CIN, int WM8>
__global__ void __launch_bounds__(NT, 1)
    dual_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ FusedParams ps,
                const __grid_constant__ FusedParams pn)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        init_barriers(smem, CIN == 1 ? ps.NS : ps.NSS);
        prefetch_tmap(&tmap);
        s_abort = 0;
    }
    __syncthreads();
    uint64_t phase = 0, ephase = 0, eused = 0;
    uint32_t nfb = 0, nties_s = 0, nties_n = 0;
    const long long T = (long long)ps.tiles_x * (ps.y_hi - ps.y_lo);
    const long long L0 = T * blockIdx.x / gridDim.x, L1 = T * (blockIdx.x + 1) / gridDim.x;
    for (long long cur = L0; cur < L1;) {
        const Segment sg = make_segment(ps, cur, L1);
        cur += sg.th_eff;
        if (threadIdx.x < NTP)
            produce<CIN>(&tmap, ps, sg, smem, phase, ephase, eused, &s_abort);
        else
            consume_dual<CIN, WM8>(ps, pn, sg, smem, nfb, nties_s, nties_n, &s_abort);
        __syncthreads();
        if (s_abort)
            break;
    }
    report(ps.stats, ps.err_flag, nfb, nties_s, s_abort != 0);
    // the Niblack mask's ties in the fourth counter
#pragma unroll
    for (int off = 16; off; off >>= 1)
        nties_n += __shfl_xor_sync(0xffffffffu, nties_n, off);
    if ((threadIdx.x & 31) == 0 && ps.stats && nties_n)
        atomicAdd(&ps.stats[BNZ_STATS_TIES_NIBLACK], (unsigned long long)nties_n);
}

template <int CIN>
const void *pick_dual(int wm8)
{
    switch (wm8) {
    case 0: return reinterpret_cast<const void *>(&dual_kernel<CIN, 0>);
    case 1: return reinterpret_cast<const void *>(&dual_kernel<CIN, 1>);
    case 2: return reinterpret_cast<const void *>(&dual_kernel<CIN, 2>);
    case 3: return reinterpret_cast<const void *>(&dual_kernel<CIN, 3>);
    case 4: return reinterpret_cast<const void *>(&dual_kernel<CIN, 4>);
    case 5: return reinterpret_cast<const void *>(&dual_kernel<CIN, 5>);
    case 6: return reinterpret_cast<const void *>(&dual_kernel<CIN, 6>);
    default: return reinterpret_cast<const void *>(&dual_kernel<CIN, 7>);
    }
}

} // namespace

int launch_dual(const uint8_t *d_src, size_t src_pitch, int h, int w, int ch, int W, double ks, double R, double kn,
                uint8_t *d_dst_s, uint8_t *d_dst_n, size_t dst_pitch, int packed, const bnz_tile *tile,
                cudaStream_t stream, unsigned long long *d_stats, unsigned int *d_err)
{
    FusedPlan pl;
    int rc = plan_fused(h, w, ch, W, tile, &pl);
    if (rc != BNZ_OK)
        return rc;
    CUtensorMap map;
    rc = encode_span_map(&map, d_src, (uint64_t)w * ch, (uint64_t)h, (uint64_t)src_pitch,
                         (uint32_t)(pl.SWP * ch), (uint32_t)pl.CH);
    if (rc != BNZ_OK)
        return rc;
    FusedParams ps, pn, dn;
    fill_fused_params(&ps, pl, h, w, W, BNZ_SAUVOLA, ks, R, d_dst_s, dst_pitch, packed, d_stats, d_err);
    // the Niblack parameters: the same geometry, that rule's constants and mask
    fill_decision_params(&dn, h, w, W, BNZ_NIBLACK, kn, 1.0);
    pn = ps;
    pn.k = dn.k;
    pn.R = dn.R;
    pn.omkn = dn.omkn;
    pn.kRn2 = dn.kRn2;
    pn.invn = dn.invn;
    pn.kn = dn.kn;
    pn.kf = dn.kf;
    pn.omk = dn.omk;
    pn.kR = dn.kR;
    pn.E = dn.E;
    pn.kh = dn.kh;
    pn.kl = dn.kl;
    pn.c1h = dn.c1h;
    pn.c1l = dn.c1l;
    pn.c2h = dn.c2h;
    pn.c2l = dn.c2l;
    pn.dst = d_dst_n;
    pn.vec_ok = ((reinterpret_cast<uintptr_t>(d_dst_n) | dst_pitch) & 15u) == 0 ? 1 : 0;
    const void *fn = ch == 1 ? pick_dual<1>(W & 7) : pick_dual<3>(W & 7);
    rc = ensure_smem_optin(fn);
    if (rc != BNZ_OK)
        return rc;
    void *args[] = {(void *)&map, (void *)&ps, (void *)&pn};
    const cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)pl.grid), dim3(NT), args, pl.smem, stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "launch dual kernel");
    return BNZ_OK;
}

} // namespace bnz
