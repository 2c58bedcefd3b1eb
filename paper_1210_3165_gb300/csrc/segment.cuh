// segment.cuh -- device code of the fused tile kernel shared by the
// single-page launch (fused.cu), the batched persistent launch (batch.cu) and
// the two-rule launch (dual.cu): one strip segment processed by 8 producer and
// 8 consumer warps.
#pragma once
#include <cstdint>

#include "decide.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace bnz {

constexpr int NTP = 256;            // producer threads (warps 0-7)
constexpr int NTPW = NTP - 32;      // column-sum producers (warps 0-6); warp 7 issues the TMA loads
constexpr int NTQ = 256;            // consumer threads (warps 8-15), one row each
constexpr int NT = NTP + NTQ;
constexpr int NTX = NTPW + NTQ;     // threads of the producer/consumer hand-over barriers
constexpr int kEmpty = 48;          // mbarriers [0, 48): slot full; [48, 96): slot free again
constexpr int L = 16;               // outputs per consumer lane per row
constexpr int TW = 32 * L;          // widest strip; 256 is used when the ring would not fit
constexpr int BAR_FULL = 1;         // named barriers 1,2: column-sum buffer b is ready
constexpr int BAR_EMPTY = 3;        // named barriers 3,4: column-sum buffer b may be refilled
constexpr int BAR_PROD = 5;         // producers only
constexpr int CH = 8;               // rows per chunk (TMA box height, one consumer warp per row)
constexpr int kLeadGray = 3;        // gray: chunks loaded ahead of the ones in use
constexpr int MAX_DYN_SMEM = 232448 - 1024; // 227 KB opt-in limit, minus slack

// Column-sum rows.  Column c of a strip's span belongs to the 4-column group
// g = (c >> 2) - o4, counted from the group holding the first column of the
// leaving stream (span column o).  Group g is stored at group position
// (g & 3) * QG + (g >> 2): four interleaved quarters of QG groups, so that
//   - the consumers' 128-bit loads (lane j reads groups 4j + i, the same i in
//     every lane) hit consecutive positions: no bank conflict, and every
//     offset is a compile-time constant plus 16 bytes per lane;
//   - the producers' 128-bit stores (thread g writes group g) fall on eight
//     distinct 16-byte bank groups per phase, because QG = 2 (mod 4);
//   - column c + 32 sits 8 words after column c (first-window loop).
constexpr int QG = 42;              // groups per quarter; QG % 4 == 2
constexpr int RS = 16 * QG;         // words per column-sum row
constexpr int C2O = CH * RS;        // words from the c1 rows of a buffer to its c2 rows

__device__ __forceinline__ void bar_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ void bar_arrive(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// byte J of w, zero-extended (one permute)
template <int J>
__device__ __forceinline__ uint32_t byte_at(uint32_t w)
{
    return __byte_perm(w, 0u, 0x4440u | J);
}

__device__ __forceinline__ uint32_t byte_dyn(uint32_t w, int j)
{
    return (w >> (8 * j)) & 0xffu;
}

// Minus byte J of w as a float, exactly: one permute forms the bit pattern
// 0xCB0000bb (= -(2^23 + b)); adding 2^23 (paired, two pixels per
// instruction) leaves -b.
template <int J>
__device__ __forceinline__ float neg_byte_pattern(uint32_t w)
{
    return __uint_as_float(prmt(w, 0xCB000000u, 0x7440u + J));
}

// Eq. 1 for one pixel, x = 299 r + 587 g + 114 b + 500 formed by two 16x8-bit
// dot products over the bytes where r, g, b sit, then q = floor(x / 1000) as
// the high word of x * ceil(2^32 / 1000): division by a constant through a
// multiply-high reciprocal (Granlund and Montgomery), exact because
// x * (1000 * ceil(2^32/1000) - 2^32) < 2^32 for x < 6.1e6 (x <= 255500 here).
__device__ __forceinline__ uint32_t div1000(uint32_t x)
{
    return __umulhi(x, 4294968u);
}

// Eq. 1 for one pixel whose r, g, b are bytes 0..2 of px (byte 3 ignored).
__device__ __forceinline__ uint32_t gray1(uint32_t px)
{
    return div1000(__dp2a_hi(0x00000072u, px, __dp2a_lo(0x024B012Bu, px, 500u)));
}

// Four gray pixels from 12 interleaved bytes r0 g0 b0 r1 | g1 b1 r2 g2 | b2 r3 g3 b3,
// packed into one word (pixel i in byte i).  Each pixel's three bytes are
// reached where they lie, by the low or high byte pair of a word, so no
// realignment is needed.
__device__ __forceinline__ uint32_t gray4(uint32_t w0, uint32_t w1, uint32_t w2)
{
    const uint32_t x0 = __dp2a_hi(0x00000072u, w0, __dp2a_lo(0x024B012Bu, w0, 500u));  // r0 g0 | b0
    const uint32_t x1 = __dp2a_lo(0x0072024Bu, w1, __dp2a_hi(0x012B0000u, w0, 500u));  // r1 | g1 b1
    const uint32_t x2 = __dp2a_lo(0x00000072u, w2, __dp2a_hi(0x024B012Bu, w1, 500u));  // r2 g2 | b2
    const uint32_t x3 = __dp2a_hi(0x0072024Bu, w2, __dp2a_lo(0x012B0000u, w2, 500u));  // r3 | g3 b3
    const uint32_t lo = prmt(div1000(x0), div1000(x1), 0x0040u);
    const uint32_t hi = prmt(div1000(x2), div1000(x3), 0x0040u);
    return prmt(lo, hi, 0x5410u);
}

struct Segment {
    int x0, y0, th_eff, xs, ys, nchk, nk;
};

// The segment starting at strip-row `cur` (strip-major over the launch's output
// rows: cur = strip * (y_hi - y_lo) + row - y_lo) of page p, ending no later
// than strip-row `end`.
__device__ __forceinline__ Segment make_segment(const FusedParams &p, long long cur, long long end)
{
    Segment sg;
    const int nr = p.y_hi - p.y_lo;
    const int tx = (int)(cur / nr);
    sg.y0 = p.y_lo + (int)(cur - (long long)tx * nr);
    sg.th_eff = (int)min((long long)(p.y_hi - sg.y0), end - cur);
    sg.x0 = tx * p.TW;
    sg.xs = sg.x0 - p.r_lo - p.o; // span start column (multiple of 16, may be < 0)
    sg.ys = sg.y0 - p.r_lo;       // first input row (may be < 0: zero-filled)
    sg.nchk = (sg.th_eff + p.W - 1 + CH - 1) / CH;
    sg.nk = (sg.th_eff + CH - 1) / CH;
    return sg;
}

// The strip-rows [L0, L1) of this CTA.  n_edge > 0: whole CTAs per strip, so
// that no CTA starts a second segment (each segment first sums its window's
// rows): n_edge CTAs on the first and on the last strip (their windows clip
// at the page's sides, the slower path), the others dealt evenly over the
// inner strips; each CTA takes an even share of its strip's rows.
__device__ __forceinline__ void cta_range(const FusedParams &p, long long &L0, long long &L1)
{
    const int nr = p.y_hi - p.y_lo;
    const int G = (int)gridDim.x, i = (int)blockIdx.x;
    if (p.n_edge <= 0) {
        const long long T = (long long)p.tiles_x * nr;
        L0 = T * i / G;
        L1 = T * (i + 1) / G;
        return;
    }
    const int S = p.tiles_x, ne = p.n_edge;
    int s, j, n;
    if (i < ne) {
        s = 0, j = i, n = ne;
    } else if (i >= G - ne) {
        s = S - 1, j = i - (G - ne), n = ne;
    } else {
        const int m = S - 2, R = G - 2 * ne, q = R / m, rem = R % m, k = i - ne;
        if (k < rem * (q + 1)) {
            s = 1 + k / (q + 1), j = k % (q + 1), n = q + 1;
        } else {
            const int k2 = k - rem * (q + 1);
            s = 1 + rem + k2 / q, j = k2 % q, n = q;
        }
    }
    if (s == 0 || s == S - 1 || p.edge_w <= 16) { // every row of an edge strip takes the border path
        L0 = (long long)s * nr + (long long)nr * j / n;
        L1 = (long long)s * nr + (long long)nr * (j + 1) / n;
        return;
    }
    // inner strip: the rows whose windows clip at the page's top or bottom also
    // take the border path and weigh edge_w / 16 as much
    const int top = min(max(p.r_lo - p.y_lo, 0), nr);
    const int bot = min(max(p.y_hi - (p.h - p.r_hi), 0), nr - top);
    const long long ew = p.edge_w, mid = nr - top - bot;
    const long long tot = (top + bot) * ew + mid * 16;
    auto row_at = [&](long long c) -> long long { // first row whose cost prefix reaches c
        if (c <= top * ew)
            return (c + ew - 1) / ew;
        c -= top * ew;
        if (c <= mid * 16)
            return top + (c + 15) / 16;
        c -= mid * 16;
        return top + mid + (c + ew - 1) / ew;
    };
    L0 = (long long)s * nr + row_at(tot * j / n);
    L1 = (long long)s * nr + row_at(tot * (j + 1) / n);
}

// ---------------------------------------------------------------------------
// producers: TMA ring, RGB->gray, column sums (a1-a3)
// ---------------------------------------------------------------------------
template <int CIN>
__device__ __forceinline__ void produce(const CUtensorMap *tmap, const FusedParams &p, const Segment &sg,
                                        uint8_t *smem, uint64_t &phase, uint64_t &ephase, uint64_t &eused,
                                        volatile int *s_abort)
{
    const int SWP = p.SWP;
    const int SWB = SWP * CIN;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + kEmpty;
    uint8_t *ring = smem + p.off_ring;
    uint8_t *stage = smem + p.off_stage;
    uint32_t *cb = reinterpret_cast<uint32_t *>(smem + p.off_cb);
    const int tid = threadIdx.x; // 0..NTP-1
    const int W = p.W;
    const int D = (CH + W - 1) / CH;
    const int nbar = CIN == 1 ? p.NS : p.NSS; // TMA targets: gray ring slots or RGB staging slots
    const uint32_t chunk_bytes = (uint32_t)(CH * SWB);

    // ---- warp 7: the TMA issuer (lane 0).  It runs ahead of the column-sum
    // producers, limited only by free slots: a slot is refilled once the
    // producers signal (empty barrier) that its previous chunk is consumed.
    // Its own state, kept across segments: `phase` bit s = parity of the next
    // completion of full[s], `ephase` bit s = parity of the next free signal
    // of slot s, `eused` bit s = slot s was ever loaded.
    if (tid >= NTPW) {
        if (tid != NTPW)
            return;
        const int x = sg.xs * CIN / 8; // element coordinate, 16-byte aligned (xs is a multiple of 16)
        int j = 0, slot = 0; // slot = j mod nbar, kept by increment (no division)
        for (; j < sg.nchk && !*s_abort; ++j, slot = (slot + 1 == nbar) ? 0 : slot + 1) {
            if ((eused >> slot) & 1ull) {
                if (!mbar_wait_bounded(&empty[slot], (uint32_t)((ephase >> slot) & 1ull), p.timeout_cycles)) {
                    *s_abort = 1;
                    break;
                }
                ephase ^= 1ull << slot;
            }
            eused |= 1ull << slot;
            uint8_t *dst = (CIN == 1 ? ring : stage) + (size_t)slot * chunk_bytes;
            mbar_arrive_expect_tx(&full[slot], chunk_bytes);
            tma_load_2d(dst, tmap, x, sg.ys + j * CH, &full[slot]);
            phase ^= 1ull << slot;
        }
        // no copy may be in flight when the segment ends: wait (bounded) for
        // the last load of each slot (earlier ones completed before its reuse)
        const int q0 = max(0, j - nbar);
        for (int q = q0, qs = q0 % nbar; q < j; ++q, qs = (qs + 1 == nbar) ? 0 : qs + 1)
            (void)mbar_wait_bounded(&full[qs], (uint32_t)(((phase >> qs) & 1ull) ^ 1ull), p.drain_cycles);
        return;
    }

    // ---- warps 0-6: RGB->gray (a2) and column sums (a3) of one 4-column
    // group per thread: group g = tid, span columns scol .. scol + 3.
    const bool owner = tid < p.ngo;
    const int scol = 4 * (tid + p.o4);
    const int gofs = 4 * ((tid & 3) * QG + (tid >> 2)); // word offset of the group in a column-sum row
    uint8_t *gbase = ring + scol;              // this thread's 4 columns, ring row 0
    const uint8_t *sbase = stage + 3 * scol;   // the same columns in staging slot 0
    const int ring_bytes = p.ring_rows * SWP;
    // columns at or right of the image edge must read as zero; the last 8-byte
    // element of a row may carry up to 7 padding bytes past the edge
    const int xg = sg.xs + scol;
    uint32_t keep = 0xffffffffu;
    if (xg + 4 > p.w)
        keep = xg >= p.w ? 0u : (0xffffffffu >> (8 * (4 - (p.w - xg))));
    const bool fix = owner && keep != 0xffffffffu && xg < ((p.w * CIN + 7) / 8 * 8 + CIN - 1) / CIN;

    // chunk counters and their slots, kept by increment (a run-time modulo costs
    // about twenty instructions and every producer thread would pay it per chunk)
    int waited = 0, freed = 0;
    int wslot = 0, fslot = 0, last = 0; // slots (mod nbar) of chunk `waited`, of chunk `freed`, of the last wait
    int gslot = 0;                      // RGB: gray ring slot (mod NS) of the next chunk converted
    bool good = !*s_abort;
    // every producer waits for itself; a wait that gives up flags the CTA
    // (the barrier protocol goes on, so no thread is left waiting)
    auto wait_one = [&]() {
        const int slot = wslot;
        last = slot;
        wslot = (wslot + 1 == nbar) ? 0 : wslot + 1;
        if (!mbar_wait_bounded(&full[slot], (uint32_t)((phase >> slot) & 1ull), p.timeout_cycles)) {
            good = false;
            *s_abort = 1;
        }
        phase ^= 1ull << slot;
        if (CIN == 1 && fix && good) { // gray: clear the padding bytes in this thread's columns
            uint8_t *r0 = gbase + (size_t)slot * CH * SWP;
            for (int r = 0; r < CH; ++r)
                *reinterpret_cast<uint32_t *>(r0 + r * SWP) &= keep;
            fence_proxy_async_smem(); // these writes precede the slot's next TMA load
        }
        ++waited;
    };
    // one producer frees the slots whose chunks no producer or consumer reads again
    auto release_to = [&](int upto) {
        for (; freed < upto; ++freed) {
            if (tid == 0)
                mbar_arrive(&empty[fslot]);
            fslot = (fslot + 1 == nbar) ? 0 : fslot + 1;
        }
    };
    // RGB: this thread's 4 columns of the chunk just waited for (staging slot
    // `last`), into the next gray ring slot (Eq. 1); chunks are converted in order
    auto convert = [&]() {
        const int gs = gslot;
        gslot = (gslot + 1 == p.NS) ? 0 : gslot + 1;
        if (!owner)
            return;
        const uint8_t *src = sbase + (size_t)last * CH * SWB;
        uint8_t *dst = gbase + (size_t)gs * CH * SWP;
        uint32_t wv[CH][3];
#pragma unroll
        for (int r = 0; r < CH; ++r) {
            const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src + r * SWB);
            wv[r][0] = s32[0];
            wv[r][1] = s32[1];
            wv[r][2] = s32[2];
        }
#pragma unroll
        for (int r = 0; r < CH; ++r)
            *reinterpret_cast<uint32_t *>(dst + r * SWP) = gray4(wv[r][0], wv[r][1], wv[r][2]) & keep;
    };

    // warm-up: chunks 0..D-1 hold rows 0..W-1, the window of the segment's first output row
    for (int j = 0; j < D; ++j) {
        if (good)
            wait_one();
        if (CIN == 3) {
            if (good)
                convert();
            bar_sync(BAR_PROD, NTPW); // staging slot j is free
            release_to(j + 1);
        }
    }
    uint32_t c1[4] = {0u, 0u, 0u, 0u}, c2[4] = {0u, 0u, 0u, 0u};
    if (good && owner) {
        int off = 0;
        for (int r = 0; r < W; ++r) {
            const uint32_t v = *reinterpret_cast<const uint32_t *>(gbase + off);
            c1[0] += byte_at<0>(v);
            c1[1] += byte_at<1>(v);
            c1[2] += byte_at<2>(v);
            c1[3] += byte_at<3>(v);
            c2[0] += byte_at<0>(v) * byte_at<0>(v);
            c2[1] += byte_at<1>(v) * byte_at<1>(v);
            c2[2] += byte_at<2>(v) * byte_at<2>(v);
            c2[3] += byte_at<3>(v) * byte_at<3>(v);
            off += SWP;
            if (off == ring_bytes)
                off = 0;
        }
    }
    int off_in = (W % p.ring_rows) * SWP; // ring offset of row i + W (entering for output row i + 1)
    int off_out = 0;                      // ring offset of row i (leaving), chunk-aligned

    for (int k = 0; k < sg.nk; ++k) {
        const int b = k & 1;
        if (k >= 2) {
            bar_sync(BAR_EMPTY + b, NTX); // consumers are done with chunk k-2
            if (CIN == 1)
                release_to(k - 1);        // gray: chunk k-2 was last read as leaving / centre rows
        }
        const int need = min(k + D, sg.nchk - 1);
        while (good && waited <= need) {
            wait_one();
            if (CIN == 3 && good)
                convert(); // own columns only: no barrier before the column sums
        }
        const int rows_k = min(CH, sg.th_eff - k * CH);
        if (good && owner) {
            const bool last = (k + 1 == sg.nk);
            uint32_t *C1 = cb + (size_t)(2 * b) * C2O + gofs;
            uint32_t vi[CH], vo[CH];
#pragma unroll
            for (int r = 0; r < CH; ++r) { // load first, then add: no smem latency per row
                int oi = off_in + r * SWP;
                if (oi >= ring_bytes)
                    oi -= ring_bytes;
                vi[r] = *reinterpret_cast<const uint32_t *>(gbase + oi);
                vo[r] = *reinterpret_cast<const uint32_t *>(gbase + off_out + r * SWP);
            }
#pragma unroll
            for (int r = 0; r < CH; ++r) {
                if (r < rows_k) {
                    *reinterpret_cast<uint4 *>(C1 + r * RS) = make_uint4(c1[0], c1[1], c1[2], c1[3]);
                    *reinterpret_cast<uint4 *>(C1 + C2O + r * RS) = make_uint4(c2[0], c2[1], c2[2], c2[3]);
                    if (!(last && r + 1 == rows_k)) { // slide to the next row
                        const uint32_t a = vi[r], o = vo[r];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint32_t aj = __byte_perm(a, 0u, 0x4440u | j);
                            const uint32_t oj = __byte_perm(o, 0u, 0x4440u | j);
                            c1[j] = c1[j] + aj - oj;
                            c2[j] = c2[j] + aj * aj - oj * oj;
                        }
                    }
                }
            }
        }
        off_in += CH * SWP;
        if (off_in >= ring_bytes)
            off_in -= ring_bytes;
        off_out += CH * SWP;
        if (off_out >= ring_bytes)
            off_out -= ring_bytes;
        bar_arrive(BAR_FULL + b, NTX); // always, so consumers never wait forever
        if (CIN == 3) {
            bar_sync(BAR_PROD, NTPW); // every producer is past the conversions of this step
            release_to(waited);       // their staging slots may be refilled
        }
    }
    // every chunk of the segment is consumed: free the remaining slots so the
    // issuer's count of free signals per slot matches its count of loads
    if (good)
        release_to(sg.nchk);
}

// ---------------------------------------------------------------------------
// consumers: horizontal sums (a4)
// ---------------------------------------------------------------------------

// A lane's 16 outputs: running offsets d[t] = S(x0 + t) - S(x0) of the window
// sums and their total a = S(x0 + 16) - S(x0), from the leaving stream (groups
// 4j + i of the lane, Lb = the c1 row + 4j words) and the entering stream
// (groups 4j + wq + i, Eb = the c1 row + 4(j + (wq >> 2)) words, WR = wq & 3),
// realigned at compile time by KO and KI (first column within its group).
template <int KO, int KI, int WR>
__device__ __forceinline__ void lane_deltas(const uint32_t *Lb, const uint32_t *Eb, uint32_t (&d1)[L],
                                            uint32_t (&d2)[L], uint32_t &a1, uint32_t &a2)
{
    auto lo = [&](int i, int arr) {
        return *reinterpret_cast<const uint4 *>(Lb + arr * C2O + 4 * ((i & 3) * QG + (i >> 2)));
    };
    auto li = [&](int i, int arr) {
        return *reinterpret_cast<const uint4 *>(Eb + arr * C2O + 4 * (((WR + i) & 3) * QG + ((WR + i) >> 2)));
    };
    a1 = 0;
    a2 = 0;
    uint4 o1 = lo(0, 0), o2 = lo(0, 1);
    uint4 i1 = li(0, 0), i2 = li(0, 1);
#pragma unroll
    for (int j = 0; j < L / 4; ++j) {
        uint4 o1n = make_uint4(0, 0, 0, 0), o2n = o1n, i1n = o1n, i2n = o1n;
        if (KO != 0 || j + 1 < L / 4) {
            o1n = lo(j + 1, 0);
            o2n = lo(j + 1, 1);
        }
        if (KI != 0 || j + 1 < L / 4) {
            i1n = li(j + 1, 0);
            i2n = li(j + 1, 1);
        }
        const uint32_t vo1[8] = {o1.x, o1.y, o1.z, o1.w, o1n.x, o1n.y, o1n.z, o1n.w};
        const uint32_t vo2[8] = {o2.x, o2.y, o2.z, o2.w, o2n.x, o2n.y, o2n.z, o2n.w};
        const uint32_t vi1[8] = {i1.x, i1.y, i1.z, i1.w, i1n.x, i1n.y, i1n.z, i1n.w};
        const uint32_t vi2[8] = {i2.x, i2.y, i2.z, i2.w, i2n.x, i2n.y, i2n.z, i2n.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            d1[4 * j + e] = a1;
            d2[4 * j + e] = a2;
            a1 = a1 + vi1[e + KI] - vo1[e + KO];
            a2 = a2 + vi2[e + KI] - vo2[e + KO];
        }
        o1 = o1n;
        o2 = o2n;
        i1 = i1n;
        i2 = i2n;
    }
}

// Geometry of a consumer lane that stays fixed over a segment.
struct LaneGeo {
    int lane, ii;       // lane, and this warp's row within each chunk
    bool active;        // lane * 16 < strip width (256-wide strips leave lanes 16..31 idle)
    int xg0;            // image column of the lane's first output
    bool xclip;         // some window of the lane leaves the image horizontally
    int fo;             // word offset of first-window column KO + lane in a column-sum row
    int fcol;           // span column of the lane's first centre pixel (a multiple of 16)
};

template <int KO>
__device__ __forceinline__ LaneGeo lane_geo(const FusedParams &p, const Segment &sg)
{
    LaneGeo g;
    const int q = threadIdx.x - NTP;
    g.lane = q & 31;
    g.ii = q >> 5;
    g.active = g.lane * L < p.TW;
    g.xg0 = sg.x0 + g.lane * L;
    g.xclip = g.xg0 < p.r_lo || g.xg0 + L - 1 + p.r_hi > p.w - 1;
    const int c = KO + g.lane; // first-window column relative to the group origin
    g.fo = 4 * (((c >> 2) & 3) * QG + (c >> 4)) + (c & 3);
    g.fcol = g.active ? g.lane * L + p.o + p.r_lo : 0;
    return g;
}

// Exact window sums of the lane's 16 pixels in one output row: S1 = base1 +
// d1[t], S2 = base2 + d2[t] (mod 2^32; S1 < 2^24 and S2 < 2^32 for W <= 255).
// C1 = the row's c1 column sums (c2 at C1 + C2O).
template <int KO, int KI, int WM8>
__device__ __forceinline__ void row_sums(const FusedParams &p, const LaneGeo &g, const uint32_t *C1,
                                         uint32_t (&d1)[L], uint32_t (&d2)[L], uint32_t &base1, uint32_t &base2)
{
    // wq = (W + KO) >> 2; for a given W mod 8 its low two bits take one of two
    // values, chosen by bit 3 of W
    constexpr int WR0 = ((WM8 + KO) >> 2) & 3;
    constexpr int WR1 = (WR0 + 2) & 3;
    uint32_t a1 = 0, a2 = 0;
    if (g.active) {
        const uint32_t *Lb = C1 + 4 * g.lane;
        const uint32_t *Eb = Lb + 4 * (p.wq >> 2);
        if (p.W & 8)
            lane_deltas<KO, KI, WR1>(Lb, Eb, d1, d2, a1, a2);
        else
            lane_deltas<KO, KI, WR0>(Lb, Eb, d1, d2, a1, a2);
    } else {
#pragma unroll
        for (int t = 0; t < L; ++t)
            d1[t] = d2[t] = 0u;
    }
    // the window of the strip's first output: relative columns [KO, KO + W)
    uint32_t s1 = 0, s2 = 0;
    for (int c = g.lane, off = g.fo; c < p.W; c += 32, off += 8) {
        s1 += C1[off];
        s2 += C1[C2O + off];
    }
    s1 = __reduce_add_sync(0xffffffffu, s1);
    s2 = __reduce_add_sync(0xffffffffu, s2);
    uint32_t x1 = a1, x2 = a2;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t1 = __shfl_up_sync(0xffffffffu, x1, off);
        const uint32_t t2 = __shfl_up_sync(0xffffffffu, x2, off);
        if (g.lane >= off) {
            x1 += t1;
            x2 += t2;
        }
    }
    base1 = s1 + x1 - a1;
    base2 = s2 + x2 - a2;
}

// The same sums again (after the fast decision let go of them), for the rare
// lanes with pixels inside the fp32 margin.
template <int KO, int KI, int WM8>
__device__ __forceinline__ void lane_sums_again(const FusedParams &p, const LaneGeo &g, const uint32_t *C1,
                                                uint32_t (&e1)[L], uint32_t (&e2)[L])
{
    constexpr int WR0 = ((WM8 + KO) >> 2) & 3;
    constexpr int WR1 = (WR0 + 2) & 3;
    uint32_t t1, t2;
    const uint32_t *Lb = C1 + 4 * g.lane;
    const uint32_t *Eb = Lb + 4 * (p.wq >> 2);
    if (p.W & 8)
        lane_deltas<KO, KI, WR1>(Lb, Eb, e1, e2, t1, t2);
    else
        lane_deltas<KO, KI, WR0>(Lb, Eb, e1, e2, t1, t2);
}

// ---------------------------------------------------------------------------
// consumers: m, s, t and Eq. 3 (a5, a6)
// ---------------------------------------------------------------------------

// Per-pixel statistics of the fp32 filter for an unclipped window (n = W*W):
// sqrt(V) by sqrt.approx from V = n*S2 - S1^2, exact in 64 bits and rounded to
// fp32 (hi word exact, lo word rounded, one more rounding in the fma: relative
// error <= 2u), and S1 as fp32 (exact, S1 < 2^24).
// With SMALL (W <= 22, so V <= n^2 * 127.5^2 < 2^32) V is exact in 32 bits
// (modular arithmetic gives the exact value) and rounds to fp32 once.
template <bool SMALL>
__device__ __forceinline__ void stats_int(uint32_t base1, int nb1, long long NB2, int nW, uint32_t d1, uint32_t d2,
                                          float &s1f, float &sq)
{
    const uint32_t S1 = base1 + d1;
    float vf;
    if (SMALL) {
        const uint32_t V = (uint32_t)NB2 + (uint32_t)nW * d2 - S1 * S1;
        vf = __uint2float_rn(V);
    } else {
        const int nS1 = nb1 - (int)d1;                              // -S1
        const long long P = NB2 + (long long)nW * (int)d2;          // n * S2
        const long long V = P + (long long)(int)S1 * nS1;           // n * S2 - S1^2 >= 0
        vf = __fmaf_rn(__uint2float_rn((uint32_t)((unsigned long long)V >> 32)), 4294967296.0f,
                       __uint2float_rn((uint32_t)V));
    }
    sq = sqrt_approx(vf);
    s1f = __uint2float_rn(S1);
}

// W <= 22: the window variance fits 32 bits
__device__ __forceinline__ bool small_window(const FusedParams &p)
{
    return p.W <= 22;
}

// Two pixels' fp32 filters, nd ~ t - f (= -d), for an unclipped window:
//   Sauvola nd = S1 * (omkn + kRn2 * sqrt(V)) - f
//   Niblack nd = S1 * invn + (kn * sqrt(V) - f)
template <int RULE>
__device__ __forceinline__ float2 filter2_int(float2 s1f, float2 sq, float2 nff, const FusedParams &p)
{
    if (RULE == BNZ_SAUVOLA) {
        const float2 x = __ffma2_rn(make_float2(p.kRn2, p.kRn2), sq, make_float2(p.omkn, p.omkn));
        return __ffma2_rn(s1f, x, nff);
    }
    const float2 y = __ffma2_rn(make_float2(p.kn, p.kn), sq, nff);
    return __ffma2_rn(s1f, make_float2(p.invn, p.invn), y);
}

// Byte i of the result = 0xFF where nd[i] has its sign bit set (t < f: white),
// 0x00 otherwise; nd = +-0 lies inside every margin and is re-decided.
__device__ __forceinline__ uint32_t sign_bytes(float n0, float n1, float n2, float n3)
{
    const uint32_t lo = prmt(__float_as_uint(n0), __float_as_uint(n1), 0xFBu);
    const uint32_t hi = prmt(__float_as_uint(n2), __float_as_uint(n3), 0xFBu);
    return prmt(lo, hi, 0x5410u);
}

// -b as fp32 for the four bytes of w, paired
__device__ __forceinline__ void neg_bytes(uint32_t w, float2 &n01, float2 &n23)
{
    const float2 bias = make_float2(8388608.0f, 8388608.0f);
    n01 = __fadd2_rn(make_float2(neg_byte_pattern<0>(w), neg_byte_pattern<1>(w)), bias);
    n23 = __fadd2_rn(make_float2(neg_byte_pattern<2>(w), neg_byte_pattern<3>(w)), bias);
}

// Fast decision of the lane's 16 pixels when every window of the warp is W x W.
// outw: byte t of word t/4 = 255 (white) or 0; mn: smallest |nd|.
template <int RULE, bool SMALL>
__device__ __forceinline__ void decide_lane_int(const FusedParams &p, uint32_t base1, uint32_t base2,
                                                const uint32_t (&d1)[L], const uint32_t (&d2)[L],
                                                const uint32_t (&fw)[4], uint32_t (&outw)[4], float &mn)
{
    const long long NB2 = (long long)((unsigned long long)p.nW * base2);
    const int nb1 = -(int)base1;
    const int nW = (int)p.nW;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
        float2 nf01, nf23;
        neg_bytes(fw[qq], nf01, nf23);
        float s[4], q[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            stats_int<SMALL>(base1, nb1, NB2, nW, d1[4 * qq + e], d2[4 * qq + e], s[e], q[e]);
        const float2 a = filter2_int<RULE>(make_float2(s[0], s[1]), make_float2(q[0], q[1]), nf01, p);
        const float2 c = filter2_int<RULE>(make_float2(s[2], s[3]), make_float2(q[2], q[3]), nf23, p);
        mn = fminf(mn, fminf(fminf(fabsf(a.x), fabsf(a.y)), fminf(fabsf(c.x), fabsf(c.y))));
        outw[qq] = sign_bytes(a.x, a.y, c.x, c.y);
    }
}

// The general filter for one pixel with its own (clipped) count n, as nd = -d.
template <int RULE>
__device__ __forceinline__ float filter_general(uint32_t f, uint32_t n, uint32_t S1, uint32_t S2,
                                                const FusedParams &p)
{
    const unsigned long long V = (unsigned long long)n * S2 - (unsigned long long)S1 * S1;
    const float sq = sqrt_approx(v_to_float(V));
    const float ff = __uint2float_rn(f), S1f = __uint2float_rn(S1);
    const float d = (n == p.nW) ? filter_int<RULE>(ff, S1f, sq, p)
                                : filter_n<RULE>(ff, S1f, sq, rcp_approx(__uint2float_rn(n)), p);
    return -d;
}

// Clipped count of the window around column xg: n = nr * nc.
__device__ __forceinline__ uint32_t clipped_n(const FusedParams &p, int nr, int xg)
{
    const int nc = min(xg + p.r_hi, p.w - 1) - max(xg - p.r_lo, 0) + 1;
    return (uint32_t)(nr * nc);
}

__device__ __forceinline__ int clipped_rows(const FusedParams &p, int y)
{
    return min(y + p.r_hi, p.h - 1) - max(y - p.r_lo, 0) + 1;
}

// Table of 1/j and 1/j^2 (fp32, correctly rounded) for j = 1..BNZ_MAX_W, at
// the start of shared memory after the barriers: the clipped windows' constants
// come from it instead of a reciprocal per pixel.
constexpr int kTabOffset = kMaxBarriers * 8;
constexpr int kTabBytes = (BNZ_MAX_W + 1) * 8;

__device__ __forceinline__ void init_recip_table(uint8_t *smem)
{
    float2 *tab = reinterpret_cast<float2 *>(smem + kTabOffset);
    for (int j = threadIdx.x; j <= BNZ_MAX_W; j += blockDim.x)
        tab[j] = j ? make_float2(__fdiv_rn(1.0f, (float)j), __fdiv_rn(1.0f, (float)(j * j))) : make_float2(0.f, 0.f);
}

// Fast decision of the lane's 16 pixels in a warp that touches the image
// border: each pixel with its own clipped count n = nr * nc, and its
// constants from the reciprocal table:
//   Sauvola c0 = ((1-k)/nr)(1/nc), c1 = (k/(R nr^2))(1/nc^2)   nd = S1 (c0 + c1 sqrt(V)) - f
//   Niblack c0 = (1/nr)(1/nc),     c1 = (k/nr)(1/nc)          nd = S1 c0 + (c1 sqrt(V) - f)
// Each constant is within 5u of its value (u = 2^-24), inside the error
// budget decision_margin allows a clipped window.
template <int RULE, bool SMALL>
__device__ __forceinline__ void decide_lane_border(const FusedParams &p, const float2 *tab, int y, int xg0,
                                                   uint32_t base1, uint32_t base2, const uint32_t (&d1)[L],
                                                   const uint32_t (&d2)[L], const uint32_t (&fw)[4],
                                                   uint32_t (&outw)[4], float &mn)
{
    const int nr = clipped_rows(p, y);
    const float2 tr = tab[nr];
    const float r0 = RULE == BNZ_SAUVOLA ? __fmul_rn(p.omk, tr.x) : tr.x;
    const float r1 = RULE == BNZ_SAUVOLA ? __fmul_rn(p.kR, tr.y) : __fmul_rn(p.kf, tr.x);
    const int a = xg0 + p.r_hi, bl = xg0 - p.r_lo;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
        float2 nf01, nf23;
        neg_bytes(fw[qq], nf01, nf23);
        float s[4], q[4], c0[4], c1[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int t = 4 * qq + e;
            // pixels past the image's right edge (results discarded) would give nc <= 0: keep the
            // table index in [1, W]
            const int nc = max(min(a + t, p.w - 1) - max(bl + t, 0) + 1, 1);
            const uint32_t n = (uint32_t)(nr * nc);
            const float2 tc = tab[nc];
            c0[e] = __fmul_rn(r0, tc.x);
            c1[e] = __fmul_rn(r1, RULE == BNZ_SAUVOLA ? tc.y : tc.x);
            const uint32_t S1 = base1 + d1[t], S2 = base2 + d2[t];
            float vf;
            if (SMALL) {
                vf = __uint2float_rn(n * S2 - S1 * S1);
            } else {
                const long long V = (long long)((unsigned long long)n * S2) + (long long)(int)S1 * -(int)S1;
                vf = __fmaf_rn(__uint2float_rn((uint32_t)((unsigned long long)V >> 32)), 4294967296.0f,
                               __uint2float_rn((uint32_t)V));
            }
            q[e] = sqrt_approx(vf);
            s[e] = __uint2float_rn(S1);
        }
        float2 nd01, nd23;
        if (RULE == BNZ_SAUVOLA) {
            nd01 = __ffma2_rn(make_float2(s[0], s[1]),
                              __ffma2_rn(make_float2(c1[0], c1[1]), make_float2(q[0], q[1]), make_float2(c0[0], c0[1])),
                              nf01);
            nd23 = __ffma2_rn(make_float2(s[2], s[3]),
                              __ffma2_rn(make_float2(c1[2], c1[3]), make_float2(q[2], q[3]), make_float2(c0[2], c0[3])),
                              nf23);
        } else {
            nd01 = __ffma2_rn(make_float2(s[0], s[1]), make_float2(c0[0], c0[1]),
                              __ffma2_rn(make_float2(c1[0], c1[1]), make_float2(q[0], q[1]), nf01));
            nd23 = __ffma2_rn(make_float2(s[2], s[3]), make_float2(c0[2], c0[3]),
                              __ffma2_rn(make_float2(c1[2], c1[3]), make_float2(q[2], q[3]), nf23));
        }
        const float nd[4] = {nd01.x, nd01.y, nd23.x, nd23.y};
#pragma unroll
        for (int e = 0; e < 4; ++e)
            mn = fminf(mn, xg0 + 4 * qq + e < p.w ? fabsf(nd[e]) : INFINITY);
        outw[qq] = sign_bytes(nd[0], nd[1], nd[2], nd[3]);
    }
}

// The pixels of the lane inside the fp32 margin, decided exactly (double-float,
// then fp64 near ties) and patched into outw.  Any pixel whose true |f - t| is
// at most the filters' error bound has |nd| < E = 2 * bound + 1e-6 in every
// filter, so this general recomputation flags every pixel the fast filter
// might have decided wrongly, whichever fast filter ran.
template <int RULE>
__device__ __forceinline__ void fix_margin(const FusedParams &p, int y, int xg0, uint32_t base1, uint32_t base2,
                                           const uint32_t (&e1)[L], const uint32_t (&e2)[L],
                                           const uint32_t (&fw)[4], uint32_t (&outw)[4], uint32_t &nfb,
                                           uint32_t &nties)
{
    const int nr = clipped_rows(p, y);
    uint32_t amask = 0;
#pragma unroll
    for (int t = 0; t < L; ++t) {
        const int xg = xg0 + t;
        const float nd = filter_general<RULE>(byte_dyn(fw[t >> 2], t & 3), clipped_n(p, nr, xg), base1 + e1[t],
                                              base2 + e2[t], p);
        if (xg < p.w && fabsf(nd) < p.E)
            amask |= 1u << t;
    }
    uint32_t white = 0; // bit t: the exact decision of pixel t is 255
    for (uint32_t m = amask; m; m &= m - 1) {
        const int t = __ffs(m) - 1;
        // register arrays are indexed with compile-time constants only
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
        const uint32_t r = decide_refine<RULE>(byte_dyn(word, t & 3), clipped_n(p, nr, xg0 + t), S1, S2, p);
        ++nfb;
        nties += (r >> 9) & 1u;
        white |= (r & 1u) << t;
    }
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) { // bits 4qq..4qq+3 -> bytes 0..3 of word qq
        const uint32_t mm = ((((amask >> (4 * qq)) & 15u) * 0x00204081u) & 0x01010101u) * 0xffu;
        const uint32_t vv = ((((white >> (4 * qq)) & 15u) * 0x00204081u) & 0x01010101u) * 0xffu;
        outw[qq] = (outw[qq] & ~mm) | (vv & mm);
    }
}

// ---------------------------------------------------------------------------
// consumers: output (a7)
// ---------------------------------------------------------------------------

// The lane's 16 outputs of row y into p.dst: byte mask or packed bits.
__device__ __forceinline__ void store_lane(const FusedParams &p, int y, int xg0, const uint32_t (&outw)[4])
{
    if (!p.packed) {
        uint8_t *drow = p.dst + (size_t)y * p.dst_pitch + xg0;
        if (p.vec_ok && xg0 + L <= p.w) {
            *reinterpret_cast<uint4 *>(drow) = make_uint4(outw[0], outw[1], outw[2], outw[3]);
        } else {
            for (int t = 0; t < L && xg0 + t < p.w; ++t)
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

// Compile-time alignment of the two horizontal streams.  o = (-r_lo) mod 16
// and r_lo = W/2: the leaving stream starts KO columns into its group and the
// entering stream (W columns later) KI columns into its group.
template <int WM8>
struct Align {
    static constexpr int KO = (4 - ((WM8 >> 1) & 3)) & 3;
    static constexpr int KI = (KO + WM8) & 3;
};

template <int CIN, int RULE, int WM8>
__device__ __forceinline__ void consume(const FusedParams &p, const Segment &sg, uint8_t *smem, uint32_t &nfb,
                                        uint32_t &nties, volatile int *s_abort)
{
    constexpr int KO = Align<WM8>::KO, KI = Align<WM8>::KI;
    const int SWP = p.SWP;
    const uint8_t *ring = smem + p.off_ring;
    const uint32_t *cb = reinterpret_cast<const uint32_t *>(smem + p.off_cb);
    const LaneGeo g = lane_geo<KO>(p, sg);
    const uint8_t *fbase = ring + g.fcol;

    int rc = (g.ii + p.r_lo) % p.ring_rows; // ring row of this warp's centre row in chunk k
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
            uint32_t outw[4];
            float mn = INFINITY; // smallest |nd| of the lane's pixels inside the image
            const bool sm = small_window(p);
            float Eq = p.E; // the margin of the filter that ran
            if (!__any_sync(0xffffffffu, lane_clip)) {
                if (sm)
                    decide_lane_int<RULE, true>(p, base1, base2, d1, d2, fw, outw, mn);
                else
                    decide_lane_int<RULE, false>(p, base1, base2, d1, d2, fw, outw, mn);
                Eq = p.Eint;
            } else {
                const float2 *tab = reinterpret_cast<const float2 *>(smem + kTabOffset);
                if (sm)
                    decide_lane_border<RULE, true>(p, tab, y, g.xg0, base1, base2, d1, d2, fw, outw, mn);
                else
                    decide_lane_border<RULE, false>(p, tab, y, g.xg0, base1, base2, d1, d2, fw, outw, mn);
            }
            if (mn < Eq && g.active) { // rare: a value inside the fp32 margin
                uint32_t e1[L], e2[L];
                lane_sums_again<KO, KI, WM8>(p, g, C1, e1, e2);
                fix_margin<RULE>(p, y, g.xg0, base1, base2, e1, e2, fw, outw, nfb, nties);
            }
            if (g.active && g.xg0 < p.w)
                store_lane(p, y, g.xg0, outw);
        }
        if (k + 2 < sg.nk)
            bar_arrive(BAR_EMPTY + b, NTX);
    }
}

template <int CIN, int RULE, int WM8>
__device__ __forceinline__ void run_segment(const CUtensorMap *tmap, const FusedParams &p, const Segment &sg,
                                            uint8_t *smem, uint64_t &phase, uint64_t &ephase, uint64_t &eused,
                                            uint32_t &nfb, uint32_t &nties, volatile int *s_abort)
{
    if (threadIdx.x < NTP)
        produce<CIN>(tmap, p, sg, smem, phase, ephase, eused, s_abort);
    else
        consume<CIN, RULE, WM8>(p, sg, smem, nfb, nties, s_abort);
}

// Kernel prologue: full and empty barriers for up to `nbar` ring/staging slots.
__device__ __forceinline__ void init_barriers(uint8_t *smem, int nbar)
{
    // (thread 0 only; the reciprocal table is filled by all threads, init_recip_table)
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    for (int i = 0; i < nbar; ++i) {
        mbar_init(&bars[i], 1);
        mbar_init(&bars[kEmpty + i], 1);
    }
    fence_mbar_init();
    fence_proxy_async_smem();
}

// Warp-aggregated statistics and the timeout report at kernel end.
__device__ __forceinline__ void report(unsigned long long *stats, unsigned int *err_flag, uint32_t nfb,
                                       uint32_t nties, bool aborted)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        nfb += __shfl_xor_sync(0xffffffffu, nfb, off);
        nties += __shfl_xor_sync(0xffffffffu, nties, off);
    }
    if ((threadIdx.x & 31) == 0 && stats && (nfb | nties)) {
        atomicAdd(&stats[BNZ_STATS_FALLBACKS], (unsigned long long)nfb);
        atomicAdd(&stats[BNZ_STATS_TIES], (unsigned long long)nties);
    }
    if (aborted && threadIdx.x == 0) {
        if (stats)
            atomicAdd(&stats[BNZ_STATS_TIMEOUTS], 1ull);
        if (err_flag)
            atomicAdd(err_flag, 1u);
    }
}

} // namespace bnz
