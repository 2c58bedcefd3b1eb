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

// Fast decision of both rules for the lane's 16 pixels when every window of the
// warp is W x W: the sums, V, sqrt(V), S1 and the pixel values are formed
// once, then each rule's fp32 filter gives its own mask word and margin.
template <bool SMALL>
__device__ __forceinline__ void decide_lane_int_dual(const FusedParams &ps, const FusedParams &pn, uint32_t base1,
                                                     uint32_t base2, const uint32_t (&d1)[L], const uint32_t (&d2)[L],
                                                     const uint32_t (&fw)[4], uint32_t (&outs)[4], uint32_t (&outn)[4],
                                                     float &mns, float &mnn)
{
    const long long NB2 = (long long)((unsigned long long)ps.nW * base2);
    const int nb1 = -(int)base1;
    const int nW = (int)ps.nW;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
        float2 nf01, nf23;
        neg_bytes(fw[qq], nf01, nf23);
        float s[4], q[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            stats_int<SMALL>(base1, nb1, NB2, nW, d1[4 * qq + e], d2[4 * qq + e], s[e], q[e]);
        const float2 s01 = make_float2(s[0], s[1]), s23 = make_float2(s[2], s[3]);
        const float2 q01 = make_float2(q[0], q[1]), q23 = make_float2(q[2], q[3]);
        const float2 a = filter2_int<BNZ_SAUVOLA>(s01, q01, nf01, ps);
        const float2 c = filter2_int<BNZ_SAUVOLA>(s23, q23, nf23, ps);
        const float2 an = filter2_int<BNZ_NIBLACK>(s01, q01, nf01, pn);
        const float2 cn = filter2_int<BNZ_NIBLACK>(s23, q23, nf23, pn);
        mns = fminf(mns, fminf(fminf(fabsf(a.x), fabsf(a.y)), fminf(fabsf(c.x), fabsf(c.y))));
        mnn = fminf(mnn, fminf(fminf(fabsf(an.x), fabsf(an.y)), fminf(fabsf(cn.x), fabsf(cn.y))));
        outs[qq] = sign_bytes(a.x, a.y, c.x, c.y);
        outn[qq] = sign_bytes(an.x, an.y, cn.x, cn.y);
    }
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
    constexpr int KO = Align<WM8>::KO, KI = Align<WM8>::KI;
    const int SWP = p.SWP;
    const uint8_t *ring = smem + p.off_ring;
    const uint32_t *cb = reinterpret_cast<const uint32_t *>(smem + p.off_cb);
    const LaneGeo g = lane_geo<KO>(p, sg);
    const uint8_t *fbase = ring + g.fcol;

    int rc = (g.ii + p.r_lo) % p.ring_rows;
    for (int k = 0; k < sg.nk; ++k, rc = (rc + CH < p.ring_rows) ? rc + CH : rc + CH - p.ring_rows) {
        const int b = k & 1;
        bar_sync(BAR_FULL + b, NTX);
        const int rows_k = min(CH, sg.th_eff - k * CH);
        if (g.ii < rows_k && !*s_abort) {
            const int y = sg.y0 + k * CH + g.ii;
            const uint32_t *C1 = cb + (size_t)(2 * b) * C2O + g.ii * RS;
            uint32_t d1[L], d2[L], base1, base2;
            row_sums<KO, KI, WM8>(p, g, C1, d1, d2, base1, base2);

            const uint4 fv = *reinterpret_cast<const uint4 *>(fbase + (size_t)rc * SWP);
            const uint32_t fw[4] = {fv.x, fv.y, fv.z, fv.w};
            const bool yclip = (y < p.r_lo) || (y + p.r_hi > p.h - 1);
            const bool lane_clip = g.active && g.xg0 < p.w && (yclip || g.xclip);
            uint32_t outs[4], outn[4];
            float mns = INFINITY, mnn = INFINITY;
            const bool sm = small_window(p);
            if (!__any_sync(0xffffffffu, lane_clip)) {
                if (sm)
                    decide_lane_int_dual<true>(ps, pn, base1, base2, d1, d2, fw, outs, outn, mns, mnn);
                else
                    decide_lane_int_dual<false>(ps, pn, base1, base2, d1, d2, fw, outs, outn, mns, mnn);
            } else {
                const float2 *tab = reinterpret_cast<const float2 *>(smem + kTabOffset);
                if (sm) {
                    decide_lane_border<BNZ_SAUVOLA, true>(ps, tab, y, g.xg0, base1, base2, d1, d2, fw, outs, mns);
                    decide_lane_border<BNZ_NIBLACK, true>(pn, tab, y, g.xg0, base1, base2, d1, d2, fw, outn, mnn);
                } else {
                    decide_lane_border<BNZ_SAUVOLA, false>(ps, tab, y, g.xg0, base1, base2, d1, d2, fw, outs, mns);
                    decide_lane_border<BNZ_NIBLACK, false>(pn, tab, y, g.xg0, base1, base2, d1, d2, fw, outn, mnn);
                }
            }
            // rare: values inside a rule's fp32 margin take that rule's exact path
            if ((mns < ps.E || mnn < pn.E) && g.active) {
                uint32_t e1[L], e2[L];
                lane_sums_again<KO, KI, WM8>(p, g, C1, e1, e2);
                if (mns < ps.E)
                    fix_margin<BNZ_SAUVOLA>(ps, y, g.xg0, base1, base2, e1, e2, fw, outs, nfb, nties_s);
                if (mnn < pn.E)
                    fix_margin<BNZ_NIBLACK>(pn, y, g.xg0, base1, base2, e1, e2, fw, outn, nfb, nties_n);
            }
            if (g.active && g.xg0 < p.w) {
                store_lane(ps, y, g.xg0, outs);
                store_lane(pn, y, g.xg0, outn);
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
    init_recip_table(smem);
    __syncthreads();
    uint64_t phase = 0, ephase = 0, eused = 0;
    uint32_t nfb = 0, nties_s = 0, nties_n = 0;
    long long L0, L1;
    cta_range(ps, L0, L1);
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
    pn.Eint = dn.Eint;
    pn.Tdf = dn.Tdf;
    pn.rk = dn.rk;
    pn.rt = dn.rt;
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
