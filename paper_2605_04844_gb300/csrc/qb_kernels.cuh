// qb_kernels.cuh -- kernel argument blocks and launchers of libquadbox.
#pragma once

#include "qb_internal.cuh"

namespace qb {

// Cameras processed together: records of camera c live at [c * n, (c+1) * n).
constexpr int kMaxGroupCams = 16;

struct CamSet {
    int n_cams;
    CamDev cam[kMaxGroupCams];
};

struct PreArgs {
    int n;  // Gaussians (records per camera)
    const float *means, *scales, *quats, *opac, *sh;
    bool raw;
    bool sh_vec4;    // sh rows may be read as float4 (16-byte aligned)
    bool quat_vec4;  // quats may be read as float4 (16-byte aligned)
    CamSet cams;     // one grid row per camera
    int mode;
    bool clamp3s;
    float2 *xy;      // [n_cams * n] ...
    float2 *shape;   // (r, -e/2) of an elongated Gaussian's exact power form, else (0, 0)
    float4 *conic_o, *rgbd, *box;
    float *r3;
    int *meta;
    uint32_t *counts;
    int *tile_diff;    // per camera [(tiles_y+1)][(tiles_x+1)] difference array of pair counts, or null
    int *tile_single;  // per camera [tiles] pair counts of single-tile Gaussians
    uint32_t diff_off[kMaxGroupCams], single_off[kMaxGroupCams];
    uint4 *segs;       // [records][4] QPass segment records (pack_segments), or null
    uint32_t *depth_keys, *depth_vals;  // [records] depth-sort keys and record indices, or null
};

// A Gaussian's QPass traversal as at most seven segments, packed in 16 words
// (four uint4): word 0 = segment count | column flag << 3 | first tile row
// << 4 | last tile row << 18; segment k in words 1 + 2k (first line | first
// cell << 16) and 2 + 2k (lines | cells << 16).
// Only the first ceil((1 + 2 ns) / 4) uint4 are written and read.
__device__ __forceinline__ int seg_chunks(int ns) { return (1 + 2 * ns + 3) >> 2; }

// Image geometry of one camera in a set of cameras rendered together.  Tile
// ids are global over the set (camera c owns [tile_base, tile_base + tiles));
// per-pixel arrays and the planar [3][H][W] image of camera c start at pixel
// pix_base (the image at float offset 3 * pix_base).  The render reads the
// camera's sorted values at vals + vals_base (its ranges are relative to it)
// and a value v names the record rec_base + v.
struct CamTile {
    int W, H, tiles_x, tiles_y;
    uint32_t tile_base;
    uint32_t rec_base;
    uint64_t pix_base;
    uint64_t vals_base;
};

// The camera owning global tile t in a device table of n cameras ordered by
// tile_base (binary search).
__device__ __forceinline__ int camera_in_table(const CamTile *table, int n, uint32_t t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (table[mid].tile_base <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct TileSet {
    int n_cams;
    uint32_t total_tiles;
    CamTile cam[kMaxGroupCams];
};

__device__ __forceinline__ int camera_of(const TileSet &ts, uint32_t gtile) {
    int c = 0;
#pragma unroll 1
    for (int k = 1; k < ts.n_cams; ++k) c = gtile >= ts.cam[k].tile_base ? k : c;
    return c;
}

struct TileOffsets {
    uint32_t diff[kMaxGroupCams], single[kMaxGroupCams];
};

struct EmitArgs {
    int n;                 // records (cameras x Gaussians)
    int n_per_cam;         // Gaussians per camera
    const uint32_t *perm;  // emission order -> record (null: index order)
    const float2 *xy;
    const float4 *box;
    const float *r3;
    const int *meta;
    const float4 *rgbd;
    const uint32_t *counts;   // by Gaussian
    const uint32_t *offsets;  // by emission position
    const uint32_t *counts_e;     // the counts by emission position, or null (read through perm)
    const uint32_t *chunk_first;  // emission position holding output position c kEmitStride, or null
    const uint4 *segs;        // QPass segment records from the preprocess, or null (recomputed)
    uint32_t *vals;
    const uint64_t *n_pairs;
    uint64_t n_pairs_host;  // P when the host knows it, else UINT64_MAX
    uint64_t capacity;
    int mode;
    bool clamp3s;
    uint32_t *err;
    TileSet ts;  // camera of record r is r / n_per_cam
};

// Tiles filed by work into kOrderBuckets buckets, heaviest first: bucket
// j = kOrderBuckets - 1 - min(work / kOrderWidth, kOrderBuckets - 1) holds
// cnt[j] tiles at list[j * ntiles ...]; position p of the order is slot
// p - (cnt[0] + ... + cnt[j - 1]) of the bucket j that contains it.  The
// counts are zeroed before the tiles are filed, each tile exactly once.
constexpr int kOrderBuckets = 64;
constexpr uint32_t kOrderWidth = 16;  // entries of work per bucket
struct TileOrder {
    uint32_t *cnt;   // [kOrderBuckets], or null: no order
    uint32_t *list;  // [kOrderBuckets][ntiles]
};

__device__ __forceinline__ void order_file(const TileOrder &o, uint32_t ntiles, uint32_t tile, uint32_t work) {
    const uint32_t j = (uint32_t)kOrderBuckets - 1u - min(work / kOrderWidth, (uint32_t)kOrderBuckets - 1u);
    const uint32_t slot = atomicAdd(o.cnt + j, 1u);
    if (slot < ntiles) o.list[(size_t)j * ntiles + slot] = tile;
}

// The tile at position pos of the order, found by one warp (every warp of a
// block finds the same tile, with no shared memory or barrier): lane l reads
// buckets l and l + 32.  Position pos itself when no bucket holds it (never,
// when every tile was filed once).
static_assert(kOrderBuckets == 64, "order_pick reads two buckets per lane");
__device__ __forceinline__ uint32_t order_pick(const TileOrder &o, uint32_t ntiles, uint32_t pos) {
    const int lane = threadIdx.x & 31;
    const uint32_t c0 = o.cnt[lane], c1 = o.cnt[32 + lane];
    uint32_t i0 = c0, i1 = c1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u0 = __shfl_up_sync(0xffffffffu, i0, d), u1 = __shfl_up_sync(0xffffffffu, i1, d);
        if (lane >= d) i0 += u0, i1 += u1;
    }
    i1 += __shfl_sync(0xffffffffu, i0, 31);  // inclusive prefixes of buckets lane and 32 + lane
    const uint32_t e0 = i0 - c0, e1 = i1 - c1;
    const bool h0 = pos >= e0 && pos < i0 && pos - e0 < ntiles;
    const bool h1 = pos >= e1 && pos < i1 && pos - e1 < ntiles;
    uint32_t t = pos;
    if (h0) t = o.list[(size_t)lane * ntiles + (pos - e0)];
    if (h1) t = o.list[(size_t)(32 + lane) * ntiles + (pos - e1)];
    const uint32_t m0 = __ballot_sync(0xffffffffu, h0), m1 = __ballot_sync(0xffffffffu, h1);
    const int src = m0 ? __ffs(m0) - 1 : (m1 ? __ffs(m1) - 1 : 0);
    t = __shfl_sync(0xffffffffu, t, src);
    return (m0 | m1) && t < ntiles ? t : pos;
}

struct RenderArgs {
    const uint2 *ranges;  // by global tile
    const uint32_t *vals;
    const float2 *xy;
    const float2 *shape;
    const float4 *conic_o, *rgbd;
    float bg[3];
    float *img;     // packed planar images
    float *tfinal;  // per pixel (all cameras)
    int *ncontrib;
    int *neval;
    TileSet ts;
    uint32_t *queue;     // persistent launch: tile counter (zeroed); null: one block per tile
    int tiles_per_fetch;
    int blocks_per_sm;   // persistent blocks per SM (0: occupancy limit)
    unsigned long long *counts;  // measurement only (single frame): [evaluated, power test passed] or null
    const CamTile *cam_table;    // persistent launch over ts.n_cams cameras from this device table, or null (ts.cam)
    // one block per tile (single frame): with order.cnt set, block b renders
    // the tile at position b of the tiles by decreasing work (TileOrder), else
    // tile b; with order_out.cnt set, every tile is filed by its largest
    // last-contributor count (the backward's work)
    TileOrder order, order_out;
};

struct BwdArgs {
    const uint2 *ranges;
    const uint32_t *vals;
    const float2 *xy;
    const float2 *shape;
    const float4 *conic_o, *rgbd;
    float bg[3];
    const float *dL_dimg;  // packed like the images
    const float *tfinal;
    const int *ncontrib;
    double *g_screen;  // [records][9]: mu_x, mu_y, Sigma11, Sigma12, Sigma22, o, r, g, b
    TileSet ts;
    uint32_t *queue;
    int tiles_per_fetch;
    int blocks_per_sm;
    const CamTile *cam_table;  // as RenderArgs::cam_table
    TileOrder order;           // as RenderArgs::order
};

struct PreBwdArgs {
    int n;  // Gaussians
    const float *means, *scales, *quats, *opac, *sh;
    bool raw;
    CamSet cams;
    const int *meta;          // [n_cams * n]
    const double *g_screen;   // [n_cams * n][9]
    float *gm, *gs, *gq, *go, *gsh;
    bool sh_vec4, gsh_vec4;   // sh / gsh rows may be accessed as float4 (16-byte aligned)
};

cudaError_t launch_preprocess(const PreArgs &a, int deg, cudaStream_t s);
// partials: scan_partials_count(n) words of scratch (block status words and
// the block counter), cleared by the launch; a look-back that waits too long
// raises kErrTimeout in *err.
cudaError_t launch_scan(const uint32_t *counts, const uint32_t *perm, int n, uint32_t *offsets, uint64_t *partials,
                        uint64_t *n_pairs, uint32_t *err, cudaStream_t s, uint32_t *counts_e = nullptr,
                        uint32_t *chunk_first = nullptr, uint32_t chunk_cap = 0);
// Output positions per entry of the scan's chunk table (a divisor of every
// emit kernel's per-warp output range).
constexpr uint32_t kEmitStride = 256;
inline uint64_t chunk_table_size(uint64_t pair_capacity) { return pair_capacity / kEmitStride + 1; }
size_t scan_partials_count(int n);
template <typename KeyT>
cudaError_t launch_emit(const EmitArgs &a, KeyT *keys, cudaStream_t s);
// K3 fused with the first pass of the depth-first tile sort (digit bits
// [0, digit_bits) of the tile id); write_keys false when it is the only pass.
cudaError_t launch_emit_sweep(const EmitArgs &a, int digit_bits, bool write_keys, uint32_t *kout, uint32_t *vout,
                              const uint32_t *bin_off, uint32_t *lookback, uint32_t *counter, cudaStream_t s);
// Counts, scans and places the pairs (writes e.vals and the ranges).
cudaError_t launch_expand_ranges(const uint2 *ranges, int ntiles, uint32_t *out, uint64_t n_out, cudaStream_t s);
template <typename KeyT>
cudaError_t launch_ranges(const KeyT *keys, uint64_t n_max, const uint64_t *n_dev, uint2 *ranges, int ntiles,
                          cudaStream_t s);
// Ranges and every tile-sort pass's bucket offsets from the per-tile counts
// in the preprocess's difference arrays (the fused-emit frame path).
cudaError_t launch_tile_prep(int *tile_diff, const int *tile_single, const TileSet &ts,
                             const uint32_t *diff_off, const uint32_t *single_off, uint2 *ranges, uint32_t *hist,
                             int hist_stride, int digit_bits, int tile_bits, uint64_t capacity, cudaStream_t s);
// Per-tile counts of n tile ids into counts[0, ntiles) (counts and the
// block counter at counts[ntiles] zeroed here); ntiles <= kTileCountMax.
// With ranges non-null the last block also writes the ranges and every
// tile-sort pass's exclusive bucket offsets (hist, stride hist_stride).
constexpr int kTileCountMax = 24576;
cudaError_t launch_tile_count(const uint32_t *keys, uint64_t n_max, const uint64_t *n_dev, int ntiles,
                              uint32_t *counts, uint2 *ranges, uint32_t *hist, int hist_stride, int digit_bits,
                              int tile_bits, cudaStream_t s);
cudaError_t launch_render(const RenderArgs &a, int batch, cudaStream_t s);
// Files every tile of a single frame (a.ts.cam[0]) into a.order by an
// estimate of the render's work: the entries composited until four sample
// pixels of the tile stop (the whole list where one does not).
cudaError_t launch_tile_work(const RenderArgs &a, cudaStream_t s);
cudaError_t launch_l1_grad(const float *img, const float *target, float *dL, uint64_t n, float scale, double *loss,
                           cudaStream_t s);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, uint64_t n, float lr, float b1, float b2,
                        float eps, int t, cudaStream_t s);
cudaError_t launch_render_bwd(const BwdArgs &a, cudaStream_t s);
cudaError_t launch_preprocess_bwd(const PreBwdArgs &a, int deg, cudaStream_t s);

}  // namespace qb
