// fused.cu -- the fused tile kernel for exact Sauvola / Niblack binarization.
//
// One persistent CTA of 16 warps walks a contiguous range of "strip rows":
// the image is cut into vertical strips of 512 output columns (256 for very
// large W), the strips are laid end to end (strip-major) and the total is
// split evenly over the grid.  Warps 0-7 (producers) and 8-15 (consumers)
// work on consecutive row chunks at the same time, handing over column sums
// through two shared-memory buffers guarded by named barriers.
//
// Producers, for each chunk of rows of a strip segment:
//   a1  load the strip plus its halo (W-1 columns, 16-aligned on the left)
//       chunk by chunk with 2-D TMA boxes into a shared-memory ring holding
//       the last W + 3 chunks of rows, so each input byte comes from global
//       memory once per strip;
//   a2  for RGB input convert each chunk to gray in shared memory with the
//       integer rule of Eq. 1, f = (299 r + 587 g + 114 b + 500) / 1000
//       (two byte dot products and a multiply-high per pixel);
//   a3  keep exact column sums c1 = sum f and c2 = sum f^2 over the W window
//       rows in registers (4 columns per thread), publish them for each row
//       of the chunk, adding the entering row and dropping the leaving one.
// Consumers, one output row per warp:
//   a4  form the horizontal window sums S1, S2: each lane slides over 16
//       consecutive outputs (128-bit loads realigned at compile time), the
//       lanes' partial sums are joined by a warp scan, and a warp reduction
//       gives the row's first window;
//   a5  use n = W*W, or, in warps that touch the image border, the clipped
//       count of each pixel;
//   a6  decide f < t (Eq. 3) for Sauvola (Eq. 4) or Niblack with an fp32
//       filter whose error is bounded (decision_margin); pixels inside the
//       bound re-run the fp64 sequence m = S1/n, s = sqrt(V)/n, t = ..., so
//       every output equals that fp64 decision;
//   a7  write the byte mask {0,255} or the packed 1-bit mask.
// The sums are exact: S1 < 2^24 and S2 < 2^32 for W <= 255, and
// V = n*S2 - S1^2 is formed in 64-bit integers.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <set>
#include <utility>

#include "segment.cuh"

namespace bnz {
namespace {

template <int CIN, int RULE, int WM8>
__global__ void __launch_bounds__(NT, 1)
    fused_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ FusedParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        init_barriers(smem, CIN == 1 ? p.NS : p.NSS);
        prefetch_tmap(&tmap);
        s_abort = 0;
    }
    init_recip_table(smem);
    __syncthreads();
    uint64_t phase = 0;             // bit i: parity of the next completion of full barrier i
    uint64_t ephase = 0, eused = 0; // TMA issuer: free-signal parity, slots ever loaded
    uint32_t nfb = 0, nties = 0;
    long long L0, L1;
    cta_range(p, L0, L1);
    for (long long cur = L0; cur < L1;) {
        const Segment sg = make_segment(p, cur, L1);
        cur += sg.th_eff;
        run_segment<CIN, RULE, WM8>(&tmap, p, sg, smem, phase, ephase, eused, nfb, nties, &s_abort);
        __syncthreads(); // the next segment reuses the ring from slot 0
        if (s_abort)
            break;
    }
    report(p.stats, p.err_flag, nfb, nties, s_abort != 0);
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

// Shared-memory layout for one (strip width, staging) choice.  The span of a
// strip (its outputs plus the window halo, 16-aligned on the left, plus the
// 128-bit over-read of the consumers' streams) is one TMA box per chunk of
// rows: at most 256 elements of 8 bytes.
bool layout(int ch, int W, int tw, int NSS, FusedPlan *pl)
{
    const int r_lo = W / 2;
    pl->TW = tw;
    pl->CH = CH;
    pl->o = (16 - (r_lo % 16)) % 16;
    const int need = pl->o + tw + W + 4;
    pl->SWP = (need + 15) / 16 * 16;
    if (pl->SWP * ch > 256 * 8)
        return false;
    // column-sum groups read by the consumers: leaving streams 4j + i, entering
    // streams 4j + wq + i (i <= 4, j < tw/16), first window below wq
    pl->o4 = pl->o >> 2;
    pl->wq = (W + (pl->o & 3)) >> 2;
    pl->ngo = tw / 4 + pl->wq + 1;
    if (pl->ngo > NTPW || pl->ngo > 4 * QG)
        return false;
    const int D = (CH + W - 1) / CH;
    // ring: chunks in use (D + 1), one more because producers run a chunk ahead
    // of the consumers' centre rows, and for gray the chunks loaded ahead
    pl->NS = D + 2 + (ch == 1 ? kLeadGray : 1);
    pl->NSS = ch == 3 ? NSS : 0;
    pl->ring_rows = pl->NS * CH;
    const int nbar = std::max(pl->NS, pl->NSS);
    if (2 * nbar > kMaxBarriers)
        return false;
    size_t off = round128((size_t)kTabOffset + kTabBytes); // barriers and reciprocal table, as in every kernel
    pl->off_ring = (uint32_t)off;
    off = round128(off + (size_t)pl->ring_rows * pl->SWP);
    pl->off_stage = (uint32_t)off;
    off = round128(off + (size_t)pl->NSS * CH * pl->SWP * ch);
    pl->off_cb = (uint32_t)off;
    off += (size_t)4 * C2O * 4; // 2 buffers x {c1, c2} x CH rows x RS words
    pl->smem = off;
    return off <= (size_t)MAX_DYN_SMEM;
}

} // namespace

// Error bound of the fp32 filter (u = 2^-24, e = relative error of sqrt.approx,
// r = relative error of rcp.approx = 4u).  V reaches fp32 with relative error
// <= 2u, so sqrt(V) carries <= u + e.
//   Sauvola, d32 = f - S1 * (a + b * sqrt(V)), a ~ (1-k)/n, b ~ k/(R n^2):
//     constants from the host carry <= u; per-pixel ones from rcp carry
//     a: <= r + 2u = 6u, b: <= 2r + 3u = 11u;
//     |d32 - (f - t)| <= 6u m|1-k| + m|k| (s/R) (12u + e) + u T + u (255 + T),
//     T = m (|1-k| + |k| s/R) >= |t|.
//   Niblack, d32 = f - S1 * invn - (k invn) sqrt(V), invn ~ 1/n within 4u:
//     |d32 - (f - t)| <= 4u m + 510 u + |k| s (7u + e) + u (510 + |k| s).
// With m <= 255 and s <= 127.5 this gives Emax; E = 2 Emax + 1e-6, which also
// covers the fp64 definition's own rounding (< 1e-12) and keeps every pixel
// with |f - t| < 1e-9 inside the margin, so ties are decided in fp64.
float decision_margin(int rule, double k, double R)
{
    const double u = 1.0 / 16777216.0;
    const double e = kSqrtApproxRelErr;
    const double ak = std::fabs(k);
    const double m = 255.0, smax = 127.5;
    double em;
    if (rule == BNZ_SAUVOLA) {
        const double T = m * (std::fabs(1.0 - k) + ak * smax / R);
        em = 6.0 * u * m * std::fabs(1.0 - k) + m * ak * (smax / R) * (12.0 * u + e) + u * T + u * (255.0 + T);
    } else {
        em = 4.0 * u * m + u * 510.0 + ak * smax * (7.0 * u + e) + u * (510.0 + ak * smax);
    }
    double E = 2.0 * em + 1e-6 + 2.0 * fp64_definition_error(rule, k, R);
    if (!(E < 1e30))
        E = 1e30;
    return (float)E;
}

// The unclipped-window filter (n = W*W; constants rounded once on the host,
// u each) is tighter.  Niblack, nd = RN(x), x = S1 RN(1/n) + RN(RN(k/n) sq - f),
// sq = sqrt.approx(V to fp32 within 2u) = sqrt(V) (1 + e + 1.01u):
//   S1 RN(1/n) = m (1 + u)                      -> u m
//   RN(k/n) sq = k s (1 + e + 2.02u)            -> |k| s (e + 2.02u)
//   rounding of k s - f                         -> u (1.01 |k| s + 255)
// so |x - (t - f)| <= em = u (510 + 1.01 |k| s) + |k| s (e + 2.02u), s <= 127.5.
// The last rounding keeps the sign of x and |x| >= |nd| / (1 + u), so
// |nd| >= E_int = 2 em + 1e-6 + 2 (the fp64 definition's error) gives the sign of
// t - f and no tie.  A lane with a pixel below E_int is re-evaluated with the
// general filter (margin E): a pixel it leaves alone has |t - f| > E/2, beyond
// the interior filter's whole error (em + u (255 + |k| s + 1) <= E/2), so its
// fast result stands.  Sauvola keeps E (its margin pixels are rare).
float decision_margin_interior(int rule, double k, double R)
{
    const float E = decision_margin(rule, k, R);
    if (rule != BNZ_NIBLACK)
        return E;
    const double u = 1.0 / 16777216.0;
    const double e = kSqrtApproxRelErr;
    const double ks = std::fabs(k) * 127.5;
    const double em = u * (510.0 + 1.01 * ks) + ks * (e + 2.02 * u);
    const double Ei = 2.0 * em + 1e-6 + 2.0 * fp64_definition_error(rule, k, R);
    return Ei < (double)E ? (float)Ei : E;
}

// Absolute error of the fp64 sequence of the definition (m = S1/n, s =
// sqrt(V)/n, then the rule left to right; V exact) against exact arithmetic:
// each correctly rounded operation adds at most w = 2^-53 of its result, and
// the results are bounded by 255 (m), 127.5 (s), T (t).  Counted generously.
double fp64_definition_error(int rule, double k, double R)
{
    const double w = 1.0 / 9007199254740992.0;
    const double m = 255.0, s = 127.5, ak = std::fabs(k);
    if (rule == BNZ_SAUVOLA)
        return 16.0 * w * (m + m * std::fabs(1.0 - k) + m * ak * (s / R + 1.0));
    return 8.0 * w * (m + ak * s);
}

// Absolute error of decide_exact's double-float f - t (pairs of fp32, u^2 =
// 2^-48 per operation): m = S1/n and sqrt(V)/n within 1 and 6 u^2 relative,
// the constants 1-k, k, k/R within 1.1 u^2 relative, each product adds 6 u^2,
// each sum 3 u^2 of its operands' magnitudes (cancellation allowed):
//   Sauvola |t~ - t| <= 12 u^2 m|1-k| + 24 u^2 m s |k|/R
//   Niblack |t~ - t| <= 4 u^2 m + 17 u^2 |k| s
// plus 3 u^2 (255 + T) for f - t; doubled for the final rounding and margin.
double double_float_error(int rule, double k, double R)
{
    const double u2 = 1.0 / 281474976710656.0;
    const double m = 255.0, s = 127.5, ak = std::fabs(k);
    double et, T;
    if (rule == BNZ_SAUVOLA) {
        et = 12.0 * u2 * m * std::fabs(1.0 - k) + 24.0 * u2 * m * s * ak / R;
        T = m * std::fabs(1.0 - k) + m * s * ak / R;
    } else {
        et = 4.0 * u2 * m + 17.0 * u2 * ak * s;
        T = m + ak * s;
    }
    return 2.0 * (et + 3.0 * u2 * (255.0 + T));
}

// A pixel whose double-float |f - t| exceeds 1e-9 + both error bounds is no tie
// of the fp64 definition and has the same sign there; the others run the fp64
// sequence.  Never below 1.2e-9; rounded up to fp32.
float double_float_cut(int rule, double k, double R)
{
    double c = 1e-9 + double_float_error(rule, k, R) + fp64_definition_error(rule, k, R);
    c = std::max(c, 1.2e-9) * (1.0 + 1e-6);
    if (!(c < 1e30))
        c = 1e30;
    return (float)c;
}

void fill_decision_params(FusedParams *p, int h, int w, int W, int rule, double k, double R)
{
    *p = FusedParams{};
    p->h = h;
    p->y_lo = 0;
    p->y_hi = h;
    p->w = w;
    p->W = W;
    p->r_lo = W / 2;
    p->r_hi = W - 1 - W / 2;
    p->nW = (uint32_t)(W * W);
    p->k = k;
    p->R = R;
    const double n = (double)W * (double)W;
    p->omkn = (float)((1.0 - k) / n);
    p->kRn2 = (float)(k / (R * n * n));
    p->invn = (float)(1.0 / n);
    p->kn = (float)(k / n);
    p->kf = (float)k;
    p->omk = (float)(1.0 - k);
    p->kR = (float)(k / R);
    p->E = decision_margin(rule, k, R);
    p->Eint = decision_margin_interior(rule, k, R);
    p->Tdf = double_float_cut(rule, k, R);
    {
        const double u = 1.0 / 16777216.0;
        p->rk = (float)(4.5 * u * std::fabs(k));
        p->rt = (float)(1.01 * (1e-9 + fp64_definition_error(rule, k, R)));
    }
    auto split = [](double x, float *hi, float *lo) {
        *hi = (float)x;
        *lo = (float)(x - (double)*hi);
    };
    split(k, &p->kh, &p->kl);
    split(1.0 - k, &p->c1h, &p->c1l);
    split(k / R, &p->c2h, &p->c2l);
}

int plan_shape(int h, int w, int ch, int W, int want_tw, FusedPlan *pl)
{
    if (want_tw && want_tw != TW && want_tw != TW / 2 && want_tw != TW / 4)
        return fail(BNZ_EINVAL, "tile width must be 0, 128, 256 or 512 (got %d)", want_tw);
    // widest strip first (least halo work), then fewer staging slots, then narrower strips
    bool found = false;
    for (int tw = TW; tw >= TW / 4 && !found; tw /= 2) {
        if (want_tw && tw != want_tw)
            continue;
        for (int nss = 3; nss >= 2 && !found; --nss)
            found = layout(ch, W, tw, nss, pl);
    }
    if (!found)
        return fail(BNZ_EINVAL, "no tile shape fits shared memory for W=%d%s", W,
                    want_tw ? " with the requested tile width" : "");
    pl->tiles_x = (w + pl->TW - 1) / pl->TW;
    (void)h;
    return BNZ_OK;
}

// The opt-in to the largest dynamic shared memory any plan uses, once per
// device and kernel (a per-launch cudaFuncSetAttribute costs microseconds).
int ensure_smem_optin(const void *fn)
{
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> g(mu);
        if (done.count({dev, fn}))
            return BNZ_OK;
    }
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaFuncSetAttribute(dynamic shared memory)");
    std::lock_guard<std::mutex> g(mu);
    done.insert({dev, fn});
    return BNZ_OK;
}

int plan_fused(int h, int w, int ch, int W, const bnz_tile *tile, FusedPlan *pl, int rows)
{
    if (rows < 0)
        rows = h;
    int sms = 0;
    int rc = device_sm_count(&sms);
    if (rc != BNZ_OK)
        return rc;
    if (tile && tile->chunk && tile->chunk != CH)
        return fail(BNZ_EINVAL, "bnz_tile.chunk must be 0 or %d (got %d)", CH, tile->chunk);
    rc = plan_shape(h, w, ch, W, tile ? tile->tile_w : 0, pl);
    if (rc != BNZ_OK)
        return rc;
    // one CTA per SM: 512 threads with up to 128 registers each take the whole register file
    const int occ = 1;
    // persistent grid: one CTA per resident slot, but at least ~2W rows of work per CTA
    const long long T = (long long)pl->tiles_x * rows;
    const long long min_rows = std::max(2 * W, 32);
    long long G = std::min<long long>((long long)sms * occ, (T + min_rows - 1) / min_rows);
    if (tile && tile->tile_h > 0)
        G = (T + tile->tile_h - 1) / tile->tile_h;
    G = std::max<long long>(1, std::min<long long>(G, 1 << 30));
    // whole CTAs per strip when every strip gets at least two: the first and
    // last strips get edge_weight/16 times an inner strip's share
    const int S = pl->tiles_x;
    const int ew = (tile && tile->edge_weight > 0) ? tile->edge_weight : kEdgeWeight;
    pl->n_edge = 0;
    pl->edge_w = ew;
    if (S >= 2 && G >= 2 * S && rows >= 2) {
        if (S == 2) {
            G &= ~1ll;
            pl->n_edge = (int)(G / 2);
        } else {
            const double tot = 2.0 * ew + 16.0 * (S - 2);
            long long ne = std::llround((double)G * ew / tot);
            pl->n_edge = (int)std::max<long long>(1, std::min<long long>(ne, (G - (S - 2)) / 2));
        }
    }
    pl->grid = (int)G;
    pl->rows_per_cta = (int)((T + G - 1) / G);
    return BNZ_OK;
}

void fill_fused_params(FusedParams *p, const FusedPlan &pl, int h, int w, int W, int rule, double k, double R,
                       uint8_t *d_dst, size_t dst_pitch, int packed, unsigned long long *d_stats, unsigned int *d_err)
{
    fill_decision_params(p, h, w, W, rule, k, R);
    p->dst = d_dst;
    p->dst_pitch = (long long)dst_pitch;
    p->stats = d_stats;
    p->err_flag = d_err;
    p->o = pl.o;
    p->TW = pl.TW;
    p->CH = pl.CH;
    p->NS = pl.NS;
    p->NSS = pl.NSS;
    p->SWP = pl.SWP;
    p->o4 = pl.o4;
    p->wq = pl.wq;
    p->ngo = pl.ngo;
    p->ring_rows = pl.ring_rows;
    p->tiles_x = pl.tiles_x;
    p->n_edge = pl.n_edge;
    p->edge_w = pl.edge_w;
    p->off_ring = pl.off_ring;
    p->off_stage = pl.off_stage;
    p->off_cb = pl.off_cb;
    p->packed = packed ? 1 : 0;
    p->vec_ok = ((reinterpret_cast<uintptr_t>(d_dst) | dst_pitch) & 15u) == 0 ? 1 : 0;
    p->timeout_cycles = 4000000000ll; // ~2 s at 2 GHz
    p->drain_cycles = 4000000000ll;
}

int launch_fused(const uint8_t *d_src, size_t src_pitch, int h, int w, int ch, int W, int rule, double k, double R,
                 uint8_t *d_dst, size_t dst_pitch, int packed, const bnz_tile *tile, cudaStream_t stream,
                 unsigned long long *d_stats, unsigned int *d_err, int y_lo, int y_hi, bool force_wait,
                 long long wait_cycles)
{
    if (y_hi < 0)
        y_hi = h;
    if (y_lo < 0 || y_lo >= y_hi || y_hi > h)
        return fail(BNZ_EINVAL, "row range [%d, %d) outside [0, %d)", y_lo, y_hi, h);
    FusedPlan pl;
    int rc = plan_fused(h, w, ch, W, tile, &pl, y_hi - y_lo);
    if (rc != BNZ_OK)
        return rc;
    CUtensorMap map;
    rc = encode_span_map(&map, d_src, (uint64_t)w * ch, (uint64_t)h, (uint64_t)src_pitch,
                         (uint32_t)(pl.SWP * ch), (uint32_t)pl.CH);
    if (rc != BNZ_OK)
        return rc;
    FusedParams p;
    fill_fused_params(&p, pl, h, w, W, rule, k, R, d_dst, dst_pitch, packed, d_stats, d_err);
    p.y_lo = y_lo;
    p.y_hi = y_hi;
    if (force_wait)
        p.timeout_cycles = wait_cycles;
    const void *fn = kernel_for(ch, rule, W);
    rc = ensure_smem_optin(fn);
    if (rc != BNZ_OK)
        return rc;
    void *args[] = {(void *)&map, (void *)&p};
    cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)pl.grid), dim3(NT), args, pl.smem, stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "launch fused kernel");
    return BNZ_OK;
}

} // namespace bnz
