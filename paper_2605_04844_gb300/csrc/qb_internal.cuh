// qb_internal.cuh -- shared device helpers and workspace layout of libquadbox.
// Method: QuadBox (arXiv 2605.04844); see include/quadbox.h for the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/quadbox.h"

namespace qb {

constexpr int kTile = 16;             // 16 x 16 pixel tiles (Sec. 2)
constexpr int kTileShift = 4;
constexpr float kAlphaMin = 1.0f / 255.0f;  // alpha_min (Sec. 3.1.1)
constexpr float kAlphaMax = 0.99f;          // opacity cap (3DGS convention)
constexpr float kTStop = 1e-4f;             // transmittance stop (3DGS convention)
constexpr float kDilation = 0.3f;           // low-pass dilation of Sigma^2D
constexpr int kDepthBits = 31;              // key = (tile << 31) | depth bits
constexpr uint32_t kErrCapacity = 1u;
constexpr uint32_t kErrTimeout = 2u;
constexpr int kMaxDigitBits = 11;
constexpr int kDepthDigitBits = 8;  // the depth-order sort: 31 bits in 4 passes (8 + 8 + 8 + 7)
constexpr int kMaxPasses = 8;              // ceil(64 / 8)

// meta bits
constexpr int kMetaVisible = 1;
constexpr int kMetaOrient = 2;
constexpr int kMetaClampShift = 2;

struct CamDev {
    float V[12];  // rows 0..2 of the world->view matrix
    float fx, fy, cx, cy;
    float limx, limy;  // 1.3 * tan_fov
    float campos[3];
    float znear;
    int W, H;
};

// Workspace offsets (bytes) of a frame; all 256-byte aligned.
struct Layout {
    size_t xy, shape, conic_o, rgbd, box, r3, meta, counts, offsets, segs;
    size_t counts_e, chunk_first;  // counts in emission order; the emit's chunk table
    size_t scan_part;
    size_t keys0, keys1, vals0, vals1;
    size_t sort_scratch, sort_scratch_bytes;
    size_t dkeys0, dkeys1, dvals0, dvals1, dsort_scratch;  // depth order of the Gaussians
    size_t ranges, tfinal, ncontrib, neval;
    size_t tile_counts;  // per-tile pair counts of the tile histogram (+ its block counter)
    size_t tile_diff;  // (tiles_y+1) x (tiles_x+1) int difference array
    size_t tile_single;  // tiles ints: pair counts of single-tile Gaussians
    size_t order_cnt;   // [2][kOrderBuckets]: the render's and the backward's tile orders (TileOrder)
    size_t order_list;  // [2][kOrderBuckets][tiles]
    size_t gscreen;  // [n][9] screen-space gradients
    size_t state;  // u64 n_pairs, u32 err_flags, padding
    size_t total;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Sets the message qb_last_error() returns on the calling thread.
void set_last_error(const char *msg);
// Counts one kernel launch of the library (qb_kernel_launches) and reports
// it to the launch hook, if one is set, just before the launch on stream s.
void note_launch(const char *kernel, cudaStream_t s);
// Raises kernel func's dynamic shared-memory limit on the current device to
// at least bytes; the limit set is remembered per (kernel, device), and the
// calls are safe from several host threads.
cudaError_t ensure_dyn_smem(const void *func, size_t bytes);

// ---- sort -------------------------------------------------------------------
// Digit geometry of an LSD radix sort on bits [0, end_bit) with digits of at
// most digit_bits: ceil(end_bit / digit_bits) passes whose widths differ by at
// most one (13 bits at 8: 7 + 6), pass p on bits [shift[p], shift[p] + bits[p]).
struct PassGeo {
    int passes;
    int shift[kMaxPasses], bits[kMaxPasses];
};

__host__ __device__ inline PassGeo pass_geo(int end_bit, int digit_bits) {
    PassGeo g;
    g.passes = end_bit > 0 ? (end_bit + digit_bits - 1) / digit_bits : 0;
    int sh = 0;
    for (int p = 0; p < kMaxPasses; ++p) {
        const int w = p < g.passes ? end_bit / g.passes + (p < end_bit % g.passes ? 1 : 0) : 0;
        g.shift[p] = sh;
        g.bits[p] = w;
        sh += w;
    }
    return g;
}

size_t sort_scratch_bytes(uint64_t n, int end_bit, int digit_bits);
// Sorts pairs on bits [0, end_bit).  n_dev: device count (<= n_max) or null
// when n_max is exact.  Returns the number of passes; result lies in the alt
// buffers when the pass count is odd.
cudaError_t sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                       uint64_t n_max, const uint64_t *n_dev, int end_bit, int digit_bits,
                       void *scratch, uint32_t *err_flags, cudaStream_t stream, int *passes_out);
// The same sort on 32-bit keys (end_bit <= 32).  With hist_ready the
// exclusive bucket offsets of every pass are already in the scratch's
// histogram table (sort_hist_table, stride sort_hist_stride per pass).
cudaError_t sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                       uint64_t n_max, const uint64_t *n_dev, int end_bit, int digit_bits,
                       void *scratch, uint32_t *err_flags, cudaStream_t stream, int *passes_out,
                       bool hist_ready = false);
uint32_t *sort_hist_table(void *scratch);
int sort_hist_stride();
// Pieces of the depth-first tile sort.  The look-back words of pass p are laid
// out for n_cap pairs; sort_clear zeroes the tile counters and look-back words
// of passes [first_pass, end_pass).
uint32_t *sort_lookback(void *scratch, uint64_t n_cap, int digit_bits, int pass);
uint32_t *sort_counter(void *scratch, int pass);
cudaError_t sort_clear(void *scratch, uint64_t n_cap, int digit_bits, int first_pass, int end_pass,
                       cudaStream_t s);
// Passes [first_pass, passes) of the tile sort on bits [0, end_bit) (pass
// widths from pass_geo): pass p writes buffer A when passes - 1 - p is even,
// else B, reading the other; the last pass writes values only (into A).
// Values are below val_bound; a two-pass sort from pass 0 whose values fit
// beside the second digit in one word carries packed words between its
// passes and leaves vB unused.
cudaError_t tile_sort_passes(uint32_t *kA, uint32_t *vA, uint32_t *kB, uint32_t *vB, uint64_t n_cap, uint64_t n_max,
                             const uint64_t *n_dev, int end_bit, int first_pass, int digit_bits, void *scratch,
                             uint32_t *err, cudaStream_t s, uint64_t val_bound);
inline bool pass_writes_a(int passes, int p) { return ((passes - 1 - p) & 1) == 0; }

// ---- device helpers -----------------------------------------------------------
// Gaussians whose stretching factor f (Eq. f-closed) has f^2 below this take
// the render's exact power form: with r = b / a = -Sigma12 / Sigma22 and
// u = dx + r dy, d^T Lambda d = a u^2 + dy^2 / Sigma22, a sum of two
// non-negative terms, where a dx^2 + 2 b dx dy + c dy^2 of a thin Gaussian
// cancels its large terms in float32 (an error of about 2^-24 (a dx^2 +
// 2 |b dx dy| + c dy^2), up to 10^5 times the result along a needle).
constexpr float kElongatedF2 = 0.01f;  // f < 0.1: aspect ratio above 10 : 1

// Exponents below this give alpha = o e^power < (1/255) e^-0.001: the 1e-3
// margin is far wider than the float32 error of the alpha test, so skipping
// them first never changes a decision of that test.
__device__ __forceinline__ float skip_threshold(float o) { return -logf(255.0f * o) - 1e-3f; }

// Whether some point of the pixel rectangle [x0, x1] x [y0, y1] can give the
// Gaussian (mu^2D, conic (a, b, c)) an exponent above t, i.e. whether the
// rectangle meets the ellipse q(d) = a dx^2 + 2 b dx dy + c dy^2 <= -2t,
// d = mu^2D - pixel.  q is convex, so its minimum over the rectangle is 0 when
// mu^2D lies inside and otherwise lies on an edge, where it is the 1D
// minimiser clamped to the edge.  The test is conservative: the radius gets a
// 1 % + 0.01 margin, far above the float32 error of q and of the kernels'
// exponents for conics whose stretching factor is above kElongatedF2, and an
// elongated or degenerate conic always meets the rectangle.
__device__ __forceinline__ bool ellipse_meets_rect(float mx, float my, float a, float b, float c, float t,
                                                   bool elongated, float x0, float y0, float x1, float y1) {
    if (elongated || !(a > 0.f && c > 0.f)) return true;
    const float r2 = fmaxf(-2.f * t, 0.f) * 1.01f + 1e-2f;
    const float ul = mx - x1, uh = mx - x0, vl = my - y1, vh = my - y0;
    if (ul <= 0.f && uh >= 0.f && vl <= 0.f && vh >= 0.f) return true;
    const float ia = 1.f / a, ic = 1.f / c;
    float best = INFINITY;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float v = e ? vh : vl;  // horizontal edge: dy fixed
        const float u = fminf(fmaxf(-b * v * ia, ul), uh);
        best = fminf(best, fmaf(a * u, u, fmaf(2.f * b * u, v, c * v * v)));
        const float u2 = e ? uh : ul;  // vertical edge: dx fixed
        const float v2 = fminf(fmaxf(-b * u2 * ic, vl), vh);
        best = fminf(best, fmaf(a * u2, u2, fmaf(2.f * b * u2, v2, c * v2 * v2)));
    }
    return best <= r2;
}

// Exponent of the 2D Gaussian at offset (dx, dy) = mu^2D - pixel,
// -(a dx^2 + 2 b dx dy + c dy^2) / 2, evaluated as a quadratic in dy:
//   A + dy (B + cc dy),  A = ca dx^2, B = cb dx,
// with (ca, cb, cc) = (-a/2, -b, -c/2), exact rescalings of the conic.  A and
// B depend on the pixel column only.  The operation sequence is spelled out
// with intrinsics so the forward and backward kernels take identical
// decisions.
__device__ __forceinline__ void power_terms(float ca, float cb, float dx, float &A, float &B) {
    A = __fmul_rn(__fmul_rn(ca, dx), dx);
    B = __fmul_rn(cb, dx);
}

__device__ __forceinline__ float power_from(float A, float B, float cc, float dy) {
    return __fmaf_rn(dy, __fmaf_rn(cc, dy, B), A);
}

struct Rect {
    int x0, y0, x1, y1;  // inclusive tile bounds; empty if x0 > x1 || y0 > y1
};

__device__ __forceinline__ bool rect_empty(const Rect &r) { return r.x0 > r.x1 || r.y0 > r.y1; }

__device__ __forceinline__ Rect empty_rect() { return Rect{1, 1, 0, 0}; }

// Closed pixel interval [lo, hi] -> tiles of the pixel centres it holds,
// clipped to [0, npx-1].  Single IEEE float operations only (no contraction
// is possible: no products), so the integers are reproducible off-device.
__device__ __forceinline__ bool tiles_of(float lo, float hi, int npx, int &t0, int &t1) {
    float p0 = fmaxf(ceilf(lo), 0.0f);
    float p1 = fminf(floorf(hi), (float)(npx - 1));
    if (!(p0 <= p1)) return false;
    t0 = ((int)p0) >> kTileShift;
    t1 = ((int)p1) >> kTileShift;
    return true;
}

__device__ __forceinline__ Rect intersect(const Rect &a, const Rect &b) {
    Rect r{max(a.x0, b.x0), max(a.y0, b.y0), min(a.x1, b.x1), min(a.y1, b.y1)};
    return rect_empty(r) ? empty_rect() : r;
}

// The per-mode tile rectangles of one Gaussian (up to four sub-boxes).
// Quadrant order I (+x,+y), II (-x,+y), III (-x,-y), IV (+x,-y); orient = 1
// when Sigma12 >= 0, i.e. the major axis runs through quadrants I and III.
// Sub-boxes share the corner mu^2D (Sec. 3.1.2).
__device__ __forceinline__ int box_rects(float mx, float my, float4 box, float r3, bool orient, int mode,
                                         bool clamp3s, int W, int H, Rect out[4]) {
    out[0] = out[1] = out[2] = out[3] = empty_rect();
    Rect r3s;
    // __fadd_rn/__fsub_rn: one rounding each, never fused with a product.
    bool ok = tiles_of(__fsub_rn(ceilf(mx), r3), __fadd_rn(floorf(mx), r3), W, r3s.x0, r3s.x1) &
              tiles_of(__fsub_rn(ceilf(my), r3), __fadd_rn(floorf(my), r3), H, r3s.y0, r3s.y1);
    if (!ok) r3s = empty_rect();
    if (mode == QB_BIN_AABB3S) {
        out[0] = r3s;
        return rect_empty(r3s) ? 0 : 1;
    }
    if (clamp3s && rect_empty(r3s)) return 0;
    if (mode == QB_BIN_ADR) {
        Rect r;
        bool oka = tiles_of(__fsub_rn(mx, box.x), __fadd_rn(mx, box.x), W, r.x0, r.x1) &
                   tiles_of(__fsub_rn(my, box.y), __fadd_rn(my, box.y), H, r.y0, r.y1);
        if (!oka) return 0;
        out[0] = clamp3s ? intersect(r, r3s) : r;
        return rect_empty(out[0]) ? 0 : 1;
    }
    int nonempty = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        bool same = (q == 0 || q == 2);
        bool major = orient ? same : !same;
        if (mode == QB_BIN_DUALBOX && !major) continue;
        float ex = major ? box.x : box.z, ey = major ? box.y : box.w;
        bool px = (q == 0 || q == 3), py = (q == 0 || q == 1);
        float xlo = px ? mx : __fsub_rn(mx, ex), xhi = px ? __fadd_rn(mx, ex) : mx;
        float ylo = py ? my : __fsub_rn(my, ey), yhi = py ? __fadd_rn(my, ey) : my;
        Rect r;
        bool okq = tiles_of(xlo, xhi, W, r.x0, r.x1) & tiles_of(ylo, yhi, H, r.y0, r.y1);
        if (!okq) continue;
        out[q] = clamp3s ? intersect(r, r3s) : r;
        nonempty += rect_empty(out[q]) ? 0 : 1;
    }
    return nonempty;
}

// QPass (Sec. 3.2): global tile range of the sub-boxes, scan lines along its
// shorter axis; per line, min/max merge of the other-axis ranges of the
// sub-boxes whose range overlaps the line.  Returns the number of lines and
// the scan geometry; line_interval() gives a line's [lo, hi].
struct QPass {
    Rect b[4];
    int s0, s1;    // scan-line range
    bool columns;  // true: lines are tile columns (x), intervals along y
};

__device__ __forceinline__ bool qpass_setup(const Rect rects[4], QPass &qp) {
    int gx0 = 1 << 30, gy0 = 1 << 30, gx1 = -1, gy1 = -1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        qp.b[q] = rects[q];
        if (rect_empty(rects[q])) continue;
        gx0 = min(gx0, rects[q].x0);
        gy0 = min(gy0, rects[q].y0);
        gx1 = max(gx1, rects[q].x1);
        gy1 = max(gy1, rects[q].y1);
    }
    if (gx1 < 0) return false;
    qp.columns = (gx1 - gx0) <= (gy1 - gy0);
    qp.s0 = qp.columns ? gx0 : gy0;
    qp.s1 = qp.columns ? gx1 : gy1;
    return true;
}

__device__ __forceinline__ void qpass_line(const QPass &qp, int s, int &lo, int &hi) {
    lo = 1 << 30;
    hi = -1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const Rect &r = qp.b[q];
        int a0 = qp.columns ? r.x0 : r.y0, a1 = qp.columns ? r.x1 : r.y1;
        int o0 = qp.columns ? r.y0 : r.x0, o1 = qp.columns ? r.y1 : r.x1;
        bool hit = (s >= a0) & (s <= a1);  // empty boxes have a0 > a1
        lo = hit ? min(lo, o0) : lo;
        hi = hit ? max(hi, o1) : hi;
    }
}

// Runs of consecutive scan lines whose merged interval is the same: the
// interval of a line changes only where a sub-box's range on the scan axis
// begins or ends, so the QPass output is a union of at most 7 disjoint
// rectangles ("segments"), each visited line by line exactly as QPass does.
struct QSeg {
    int s0, lo;   // first line, first tile on the other axis
    int nl, len;  // lines in the run, interval length
};

// The runs are found in order and stored in fixed slots (so the array stays
// in registers): slot k holds the k-th run, an empty one (no sub-box overlaps
// its lines) with nl = len = 0.  The lines [s0, s1] have at most six interior
// breakpoints (each sub-box begins or ends at most once), so seven slots hold
// every run.  Returns the number of slots used.
__device__ __forceinline__ int qpass_segments(const QPass &qp, QSeg seg[7]) {
    int used = 0;
    int cur = qp.s0;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        seg[k] = QSeg{0, 0, 0, 0};
        if (cur > qp.s1) continue;
        int next = qp.s1 + 1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Rect &r = qp.b[q];
            if (rect_empty(r)) continue;
            const int a0 = qp.columns ? r.x0 : r.y0, a1 = qp.columns ? r.x1 : r.y1;
            if (a0 > cur) next = min(next, a0);
            if (a1 + 1 > cur) next = min(next, a1 + 1);
        }
        int lo, hi;
        qpass_line(qp, cur, lo, hi);
        if (hi >= lo) seg[k] = QSeg{cur, lo, next - cur, hi - lo + 1};
        used = k + 1;
        cur = next;
    }
    return used;
}

__device__ __forceinline__ bool seg_empty(const QSeg &g) { return g.nl <= 0 || g.len <= 0; }

__device__ __forceinline__ uint32_t qpass_count(const Rect rects[4]) {
    QPass qp;
    if (!qpass_setup(rects, qp)) return 0;
    uint32_t c = 0;
    for (int s = qp.s0; s <= qp.s1; ++s) {
        int lo, hi;
        qpass_line(qp, s, lo, hi);
        c += (hi >= lo) ? (uint32_t)(hi - lo + 1) : 0u;
    }
    return c;
}

// Naive traversal (QuadBox-dagger, Table 3): nested loops over each
// sub-box's rectangle, skipping tiles held by an earlier sub-box.
__device__ __forceinline__ bool in_rect(const Rect &r, int tx, int ty) {
    return !rect_empty(r) && tx >= r.x0 && tx <= r.x1 && ty >= r.y0 && ty <= r.y1;
}

__device__ __forceinline__ uint32_t naive_count(const Rect r[4]) {
    uint32_t c = 0;
    for (int q = 0; q < 4; ++q) {
        if (rect_empty(r[q])) continue;
        for (int ty = r[q].y0; ty <= r[q].y1; ++ty)
            for (int tx = r[q].x0; tx <= r[q].x1; ++tx) {
                bool seen = false;
                for (int p = 0; p < q; ++p) seen |= in_rect(r[p], tx, ty);
                c += seen ? 0u : 1u;
            }
    }
    return c;
}

}  // namespace qb
