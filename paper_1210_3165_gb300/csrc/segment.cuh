// segment.cuh -- device code of the fused tile kernel shared by the
// single-page launch (fused.cu) and the batched persistent launch (batch.cu):
// one strip segment processed by 8 producer and 8 consumer warps.
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

// Shared memory holds rows row-major: the gray ring (ring_rows x SWP bytes)
// and, for RGB, the staging slots (CH x 3*SWP bytes each), each chunk of rows
// one TMA box of 8-byte elements.

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

// Byte j of w as a float, exactly: one permute forms the bit pattern
// 0x4B0000bb (= 2^23 + b) and one subtraction removes 2^23, instead of a
// byte extract and an integer-to-float conversion.
__device__ __forceinline__ float byte_float(uint32_t w, int j)
{
    return __fsub_rn(__uint_as_float(prmt(w, 0x4B000000u, 0x7440u + (uint32_t)j)), 8388608.0f);
}

// Word offset of 4-column group g in a column-sum row.  The groups are
// XOR-swizzled within aligned blocks of four, g ^ ((g >> 3) & 3), so that
// both access patterns hit eight distinct 16-byte bank groups per phase: the
// producers' 128-bit stores (consecutive groups, one per thread) and the
// consumers' 128-bit loads (groups four apart, one per lane, any offset).
__device__ __forceinline__ int gpos(int g)
{
    return 4 * (g ^ ((g >> 3) & 3));
}

// Word offset of span column c.
__device__ __forceinline__ int cpos(int c)
{
    return gpos(c >> 2) + (c & 3);
}

__device__ __forceinline__ uint4 ld_group(const uint32_t *C, int a) // columns 4a..4a+3
{
    return *reinterpret_cast<const uint4 *>(C + gpos(a));
}

// Eq. 1 for one pixel whose r, g, b are bytes 0..2 of px (byte 3 ignored):
// x = 299 r + 587 g + 114 b + 500 = (43 r + 75 g + 114 b) + 256 (r + 2 g) + 500,
// q = floor(x / 1000) = high word of x * ceil(2^32 / 1000) (exact for x < 6.1e6).
__device__ __forceinline__ uint32_t gray1(uint32_t px)
{
    const uint32_t hi = __dp4a(px, 0x00000201u, 0u);
    const uint32_t x = __dp4a(px, 0x00724B2Bu, hi * 256u + 500u);
    return __umulhi(x, 4294968u);
}

// Four gray pixels from 12 interleaved bytes r0 g0 b0 r1 | g1 b1 r2 g2 | b2 r3 g3 b3.
__device__ __forceinline__ uint32_t gray4(uint32_t w0, uint32_t w1, uint32_t w2)
{
    const uint32_t g0 = gray1(w0);
    const uint32_t g1 = gray1(__funnelshift_r(w0, w1, 24));
    const uint32_t g2 = gray1(__funnelshift_r(w1, w2, 16));
    const uint32_t g3 = gray1(w2 >> 8);
    return g0 | (g1 << 8) | (g2 << 16) | (g3 << 24);
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

// One segment with the 16 warps split into producers and consumers.
template <int CIN, int RULE, int WM8>
__device__ __forceinline__ void run_segment(const CUtensorMap *tmap, const FusedParams &p, const Segment &sg,
                                            uint8_t *smem, uint64_t &phase, uint64_t &ephase, uint64_t &eused,
                                            uint32_t &nfb, uint32_t &nties, volatile int *s_abort);

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
            (void)mbar_wait_bounded(&full[qs], (uint32_t)(((phase >> qs) & 1ull) ^ 1ull), p.timeout_cycles);
        return;
    }

    // ---- warps 0-6: RGB->gray (a2) and column sums (a3), 4 columns per thread
    const bool owner = tid < (SWP >> 2);
    const int gcol = tid * 4;
    const int gofs = cpos(gcol);
    uint8_t *gbase = ring + gcol;              // this thread's 4 columns, ring row 0
    const uint8_t *sbase = stage + 3 * gcol;   // the same columns in staging slot 0
    const int ring_bytes = p.ring_rows * SWP;
    // columns at or right of the image edge must read as zero; the last 8-byte
    // element of a row may carry up to 7 padding bytes past the edge
    const int xg = sg.xs + gcol;
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
            uint32_t *C1 = cb + (size_t)(2 * b) * CH * p.RSW + gofs;
            uint32_t *C2 = C1 + (size_t)CH * p.RSW;
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
                    *reinterpret_cast<uint4 *>(C1 + r * p.RSW) = make_uint4(c1[0], c1[1], c1[2], c1[3]);
                    *reinterpret_cast<uint4 *>(C2 + r * p.RSW) = make_uint4(c2[0], c2[1], c2[2], c2[3]);
                    if (!(last && r + 1 == rows_k)) { // slide to the next row
                        const uint32_t a = vi[r], o = vo[r];
                        c1[0] = c1[0] + byte_at<0>(a) - byte_at<0>(o);
                        c1[1] = c1[1] + byte_at<1>(a) - byte_at<1>(o);
                        c1[2] = c1[2] + byte_at<2>(a) - byte_at<2>(o);
                        c1[3] = c1[3] + byte_at<3>(a) - byte_at<3>(o);
                        c2[0] = c2[0] + byte_at<0>(a) * byte_at<0>(a) - byte_at<0>(o) * byte_at<0>(o);
                        c2[1] = c2[1] + byte_at<1>(a) * byte_at<1>(a) - byte_at<1>(o) * byte_at<1>(o);
                        c2[2] = c2[2] + byte_at<2>(a) * byte_at<2>(a) - byte_at<2>(o) * byte_at<2>(o);
                        c2[3] = c2[3] + byte_at<3>(a) * byte_at<3>(a) - byte_at<3>(o) * byte_at<3>(o);
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

// A lane's 16 outputs: running offsets d[t] = S(x0 + t) - S(x0) of the window
// sums (leaving stream from column group ao, entering from ai, realigned at
// compile time by KO / KI), and their total a = S(x0 + 16) - S(x0).
template <int KO, int KI>
__device__ __forceinline__ void lane_deltas(const uint32_t *C1, const uint32_t *C2, int ao, int ai, uint32_t (&d1)[L],
                                            uint32_t (&d2)[L], uint32_t &a1, uint32_t &a2)
{
    a1 = 0;
    a2 = 0;
    uint4 o1 = ld_group(C1, ao), o2 = ld_group(C2, ao);
    uint4 i1 = ld_group(C1, ai), i2 = ld_group(C2, ai);
#pragma unroll
    for (int j = 0; j < L / 4; ++j) {
        uint4 o1n = make_uint4(0, 0, 0, 0), o2n = o1n, i1n = o1n, i2n = o1n;
        if (KO != 0 || j + 1 < L / 4) {
            o1n = ld_group(C1, ao + j + 1);
            o2n = ld_group(C2, ao + j + 1);
        }
        if (KI != 0 || j + 1 < L / 4) {
            i1n = ld_group(C1, ai + j + 1);
            i2n = ld_group(C2, ai + j + 1);
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

// ---------------------------------------------------------------------------
// consumers: horizontal sums, threshold, output (a4-a7)
// ---------------------------------------------------------------------------
template <int CIN, int RULE, int WM8>
__device__ __forceinline__ void consume(const FusedParams &p, const Segment &sg, uint8_t *smem, uint32_t &nfb,
                                        uint32_t &nties, volatile int *s_abort)
{
    const int SWP = p.SWP;
    // o = (-r_lo) mod 16 and r_lo = W/2: the misalignments of the leaving
    // (span column o + x) and entering (o + W + x) streams depend on W mod 8
    constexpr int KO = (4 - ((WM8 >> 1) & 3)) & 3;
    constexpr int KI = (KO + WM8) & 3;
    const uint8_t *ring = smem + p.off_ring;
    const uint32_t *cb = reinterpret_cast<const uint32_t *>(smem + p.off_cb);
    const int q = threadIdx.x - NTP;
    const int lane = q & 31, ii = q >> 5; // this warp's row within each chunk
    const int W = p.W;
    const bool active = lane * L < p.TW; // 256-wide strips leave lanes 16..31 idle
    // centre pixels of this lane's 16 outputs start at span column lane*16 + o + r_lo (a multiple of 16)
    const int fcol = active ? lane * L + p.o + p.r_lo : 0;
    const uint8_t *fbase = ring + fcol;
    const int xg0 = sg.x0 + lane * L;
    const bool xclip = xg0 < p.r_lo || xg0 + L - 1 + p.r_hi > p.w - 1; // some window of the lane leaves the image

    int rc = (ii + p.r_lo) % p.ring_rows; // ring row of this warp's centre row in chunk k
    for (int k = 0; k < sg.nk; ++k, rc = (rc + CH < p.ring_rows) ? rc + CH : rc + CH - p.ring_rows) {
        const int b = k & 1;
        bar_sync(BAR_FULL + b, NTX);
        const int rows_k = min(CH, sg.th_eff - k * CH);
        if (ii < rows_k && !*s_abort) {
            const int i = k * CH + ii;
            const int y = sg.y0 + i;
            const uint32_t *C1 = cb + (size_t)(2 * b) * CH * p.RSW + ii * p.RSW;
            const uint32_t *C2 = C1 + (size_t)CH * p.RSW;
            const int cw = lane * L + p.o; // leaving-stream start; entering = cw + W
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
            // the window of the strip's first output: span columns [o, o + W)
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
            uint32_t outw[4];
            float mn = INFINITY; // smallest |d| of the lane's pixels inside the image
            if (!__any_sync(0xffffffffu, lane_clip)) {
                // every window of the warp is W x W: shared constants
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    float dd[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int t = 4 * qq + e;
                        const uint32_t S1 = base1 + d1[t];
                        const uint32_t S2 = base2 + d2[t]; // exact: S2 < 2^32
                        const unsigned long long V =
                            (unsigned long long)p.nW * S2 - (unsigned long long)S1 * S1;
                        const float ff = byte_float(fw[qq], e);
                        dd[e] = filter_int<RULE>(ff, __uint2float_rn(S1), sqrt_approx(v_to_float(V)), p);
                        mn = fminf(mn, fabsf(dd[e]));
                    }
                    // byte = 0xFF where d >= +0, 0x00 where d < 0 (sign bit replicated)
                    const uint32_t lo = prmt(__float_as_uint(dd[0]), __float_as_uint(dd[1]), 0xFBu);
                    const uint32_t hi = prmt(__float_as_uint(dd[2]), __float_as_uint(dd[3]), 0xFBu);
                    outw[qq] = ~prmt(lo, hi, 0x5410u);
                }
            } else {
                // border warp: each pixel with its own clipped count n = nr * nc
                const int nr = min(y + p.r_hi, p.h - 1) - max(y - p.r_lo, 0) + 1;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    float dd[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int t = 4 * qq + e;
                        const int xg = xg0 + t;
                        const int nc = min(xg + p.r_hi, p.w - 1) - max(xg - p.r_lo, 0) + 1;
                        const uint32_t n = (uint32_t)(nr * nc);
                        const uint32_t S1 = base1 + d1[t], S2 = base2 + d2[t];
                        const unsigned long long V = (unsigned long long)n * S2 - (unsigned long long)S1 * S1;
                        const float ff = byte_float(fw[qq], e);
                        const float invn = rcp_approx(__uint2float_rn(n));
                        dd[e] = filter_n<RULE>(ff, __uint2float_rn(S1), sqrt_approx(v_to_float(V)), invn, p);
                        mn = fminf(mn, xg < p.w ? fabsf(dd[e]) : INFINITY);
                    }
                    const uint32_t lo = prmt(__float_as_uint(dd[0]), __float_as_uint(dd[1]), 0xFBu);
                    const uint32_t hi = prmt(__float_as_uint(dd[2]), __float_as_uint(dd[3]), 0xFBu);
                    outw[qq] = ~prmt(lo, hi, 0x5410u);
                }
            }
            if (mn < p.E && active) { // rare: a value inside the fp32 margin -> fp64 for those pixels
                // (1) which pixels: the 16 filters again, unrolled and independent (with
                // each pixel's own n, as the border path), into a bit mask;
                // (2) the fp64 sequence for the set bits only, typically one.  Register
                // arrays are indexed with compile-time constants only, so nothing of the
                // fast path moves to local memory.
                const int nr = min(y + p.r_hi, p.h - 1) - max(y - p.r_lo, 0) + 1;
                // the sums again from the column-sum buffer (still valid: it is released
                // after this row), so the fast path's offsets need not live until here
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
                                                : filter_n<RULE>(ff, __uint2float_rn(S1), sq,
                                                                 rcp_approx(__uint2float_rn(n)), p);
                    if (xg < p.w && fabsf(d) < p.E)
                        amask |= 1u << t;
                }
                uint32_t white = 0; // bit t: the fp64 decision of pixel t is 255
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
                for (int qq = 0; qq < 4; ++qq) { // bits 4qq..4qq+3 -> bytes 0..3 of word qq
                    const uint32_t mm = ((((amask >> (4 * qq)) & 15u) * 0x00204081u) & 0x01010101u) * 0xffu;
                    const uint32_t vv = ((((white >> (4 * qq)) & 15u) * 0x00204081u) & 0x01010101u) * 0xffu;
                    outw[qq] = (outw[qq] & ~mm) | (vv & mm);
                }
            }
            if (active && xg0 < p.w) {
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
