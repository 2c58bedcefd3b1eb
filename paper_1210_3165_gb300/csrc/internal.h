// internal.h -- declarations shared by the library's translation units
// (kernel launch parameters, tile plans, error reporting).  Not installed.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/bnz.h"

namespace bnz {

// Sets the calling thread's last-error message (printf-style) and returns rc.
int fail(int rc, const char *fmt, ...);
// Maps a CUDA runtime error to BNZ_ECUDA with a message naming `what`.
int cuda_fail(cudaError_t e, const char *what);

// Encodes a 2-D tensor map over rows of `row_bytes` bytes, `pitch` apart, in
// 8-byte elements (ceil(row_bytes/8) per row, so the last element of a row
// may take up to 7 padding bytes), with boxes of box_bytes x box_rows.
int encode_span_map(CUtensorMap *map, const void *base, uint64_t row_bytes, uint64_t rows, uint64_t pitch,
                    uint32_t box_bytes, uint32_t box_rows);

int device_sm_count(int *sms);

// Argument checks shared by the binarize entry points (BNZ_OK or BNZ_EINVAL).
int check_common(const void *src, size_t src_pitch, int height, int width, int channels, int W, int rule,
                 double k, double R, const void *dst, size_t dst_pitch, int packed);

// ---- fused tile kernel -----------------------------------------------------

// Shape of one launch of the fused kernel (host-side plan).
struct FusedPlan {
    int TW, CH;     // strip width (32 lanes x 16 outputs), rows per TMA chunk
    int NS;         // ring slots (chunks) of gray rows in shared memory
    int NSS;        // staging slots for RGB chunks (0 for gray)
    int SWP;        // span width in pixels: one TMA box of SWP*channels bytes per chunk
    int ring_rows;  // NS * CH
    int o;          // span start offset: (x0 - r_lo) - floor16(x0 - r_lo)
    int o4, wq;     // o >> 2; (W + (o & 3)) >> 2: group of the entering stream's first column
    int ngo;        // 4-column groups whose column sums the consumers read (from group o4 on)
    int tiles_x;    // strips across the image
    int grid;       // persistent CTAs
    int n_edge;     // CTAs on each of the first and last strips (0: one even split of all strip-rows)
    int edge_w;     // the edge weight used (sixteenths)
    int rows_per_cta;
    uint32_t off_ring, off_stage, off_cb; // column sums: 2 buffers x {c1, c2} x CH rows x RS words
    size_t smem;
};

struct FusedParams {
    uint8_t *dst;
    long long dst_pitch;
    unsigned long long *stats;
    unsigned int *err_flag; // library-owned device word, counts CTAs that gave up
    int h, w, W, r_lo, r_hi, o;
    int y_lo, y_hi;  // output rows [y_lo, y_hi) of this launch (the window clips at 0 and h)
    int TW, CH, NS, NSS, SWP, ring_rows, tiles_x;
    int o4, wq, ngo; // column-sum groups: origin, entering-stream offset, count (see FusedPlan)
    int n_edge;      // CTAs per edge strip, the rest dealt evenly over the inner strips (0: even split)
    int edge_w;      // cost of a row taking the border path, in sixteenths of an inner row's
    uint32_t off_ring, off_stage, off_cb;
    int packed;     // 1: one bit per pixel
    int vec_ok;     // dst and dst_pitch 16-byte aligned
    uint32_t nW;    // W*W
    double k, R;    // the caller's parameters, for the fp64 re-evaluation
    // fp32 constants of the filter for unclipped windows (n = W*W):
    //   Sauvola d = f - S1 * (omkn + kRn2 * sqrt(V)),  omkn = (1-k)/n, kRn2 = k/(R n^2)
    //   Niblack d = f - S1 * invn - kn * sqrt(V),      invn = 1/n,     kn = k/n
    float omkn, kRn2, invn, kn;
    float kf, omk, kR; // k, 1-k, k/R for windows with a per-pixel n
    float E;           // proven bound on |d32 - (f - t)|, with safety factor
    float Eint;        // the same for the unclipped-window filter (n = W*W, host constants): <= E
    // double-float constants of the second stage: k, 1-k, k/R as hi + lo
    float kh, kl, c1h, c1l, c2h, c2l;
    // the second stage decides by the sign of its f - t when |f - t| > Tdf =
    // 1e-9 + its own error bound + the fp64 definition's (double_float_cut)
    float Tdf;
    // Niblack, first re-decision of a margin pixel: X = n (f - t) = (n f - S1) - k sqrt(V) in fp32 decides
    // when |X| > rk sqrt(V) + rt n (rk = 4.5 u |k|, rt = 1.01 (1e-9 + the fp64 definition's error))
    float rk, rt;
    long long timeout_cycles; // limit of every wait but the final drain (<= 0: give up unless already complete)
    long long drain_cycles;   // limit of the TMA issuer's final wait for its copies in flight
};

// Shape of the fused kernel for one page (strip width, ring, shared-memory
// offsets); want_tw = 0 picks the widest strip that fits.
int plan_shape(int h, int w, int ch, int W, int want_tw, FusedPlan *plan);
// rows: output rows of the launch (h for a whole page), which sets the grid.
int plan_fused(int h, int w, int ch, int W, const bnz_tile *tile, FusedPlan *plan, int rows = -1);
void fill_fused_params(FusedParams *p, const FusedPlan &pl, int h, int w, int W, int rule, double k, double R,
                       uint8_t *d_dst, size_t dst_pitch, int packed, unsigned long long *d_stats,
                       unsigned int *d_err);
constexpr int kMaxBarriers = 96; // mbarriers reserved at the start of shared memory: full + empty per slot
// Default cost of an edge strip's row against an inner strip's, in sixteenths (bnz_tile.edge_weight).
constexpr int kEdgeWeight = 20; // measured best of 16..32 on 4096^2 RGB pages, W 15..101, both rules
// Raise the kernel's dynamic shared-memory limit to the largest plan, once per device.
int ensure_smem_optin(const void *fn);
// Output rows [y_lo, y_hi) of the page (0, h: all); the kernel reads input rows
// [y_lo - W/2, y_hi + W) at most, the ones past y_hi - 1 + (W - 1 - W/2) unused.
// wait_cycles > 0 (or <= 0 with force_wait) overrides the waits' limit (self-test of the abort path).
int launch_fused(const uint8_t *d_src, size_t src_pitch, int h, int w, int ch, int W, int rule, double k,
                 double R, uint8_t *d_dst, size_t dst_pitch, int packed, const bnz_tile *tile,
                 cudaStream_t stream, unsigned long long *d_stats, unsigned int *d_err, int y_lo = 0,
                 int y_hi = -1, bool force_wait = false, long long wait_cycles = 0);

// Library-owned per-device error word (allocated on first use).
int device_err_flag(unsigned int **flag);

// Relative error bounds assumed for sqrt.approx.f32 (on [1, 2^48)) and
// rcp.approx.f32 (on the integers 1..65025); both are measured on the device
// by bnz_selftest_approx in the tests.
constexpr double kSqrtApproxRelErr = 1.0 / (1 << 21);
constexpr double kRcpApproxRelErr = 1.0 / (1 << 22);

// fp32 decision margin E (see fused.cu for the derivation), and the tighter
// one of the unclipped-window filter.
float decision_margin(int rule, double k, double R);
float decision_margin_interior(int rule, double k, double R);
// Error bounds, for m <= 255 and s <= 127.5, of the double-float evaluation of
// f - t and of the fp64 definition's t; and the cut Tdf built from them.
double double_float_error(int rule, double k, double R);
double fp64_definition_error(int rule, double k, double R);
float double_float_cut(int rule, double k, double R);

// Fills the geometry and threshold constants of `p` shared by every kernel
// that takes the Eq. 3 decision (window radii, k, R, fp32 constants, margin).
void fill_decision_params(FusedParams *p, int h, int w, int W, int rule, double k, double R);

// ---- integral-image comparison variant (integral.cu) -----------------------
size_t integral_scratch_bytes(int h, int w);
int launch_integral_tables(const uint8_t *d_src, size_t src_pitch, int h, int w, int ch, void *scratch,
                           cudaStream_t stream, long long *ld_out);
int launch_integral(const uint8_t *d_src, size_t src_pitch, int h, int w, int ch, int W, int rule, double k,
                    double R, uint8_t *d_dst, size_t dst_pitch, int packed, void *scratch, cudaStream_t stream,
                    unsigned long long *d_stats);

// ---- reduced-set rule of Sec. 2 and the Eq. 6 counts (gs.cu) ---------------
int launch_gs(const uint8_t *d_src, size_t src_pitch, int h, int w, int ch, int W, int gs, int rule, double k,
              double R, uint8_t *d_dst, size_t dst_pitch, unsigned long long *d_stats, cudaStream_t stream);
int launch_confusion(const uint8_t *d_mask, size_t mask_pitch, int mask_ink, const uint8_t *d_ref, size_t ref_pitch,
                     int ref_ink, int h, int w, unsigned long long *d_counts, cudaStream_t stream);

} // namespace bnz
