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
    float4 *conic_o, *rgbd, *box;
    float *r3;
    int *meta;
    uint32_t *counts;
    int *tile_diff;    // per camera [(tiles_y+1)][(tiles_x+1)] difference array of pair counts, or null
    int *tile_single;  // per camera [tiles] pair counts of single-tile Gaussians
    uint32_t diff_off[kMaxGroupCams], single_off[kMaxGroupCams];
};

// Image geometry of one camera in a set of cameras rendered together.  Tile
// ids are global over the set (camera c owns [tile_base, tile_base + tiles));
// per-pixel arrays and the planar [3][H][W] image of camera c start at pixel
// pix_base (the image at float offset 3 * pix_base).
struct CamTile {
    int W, H, tiles_x, tiles_y;
    uint32_t tile_base;
    uint64_t pix_base;
};

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
    uint32_t *vals;
    const uint64_t *n_pairs;
    uint64_t n_pairs_host;  // P when the host knows it, else UINT64_MAX
    uint64_t capacity;
    int mode;
    bool clamp3s;
    uint32_t *err;
    TileSet ts;  // camera of record r is r / n_per_cam
};

struct RenderArgs {
    const uint2 *ranges;  // by global tile
    const uint32_t *vals;
    const float2 *xy;
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
};

struct BwdArgs {
    const uint2 *ranges;
    const uint32_t *vals;
    const float2 *xy;
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
};

struct PreBwdArgs {
    int n;  // Gaussians
    const float *means, *scales, *quats, *opac, *sh;
    bool raw;
    CamSet cams;
    const int *meta;          // [n_cams * n]
    const double *g_screen;   // [n_cams * n][9]
    float *gm, *gs, *gq, *go, *gsh;
};

cudaError_t launch_preprocess(const PreArgs &a, int deg, cudaStream_t s);
cudaError_t launch_scan(const uint32_t *counts, const uint32_t *perm, int n, uint32_t *offsets, uint64_t *partials,
                        uint64_t *n_pairs, cudaStream_t s);
size_t scan_partials_count(int n);
cudaError_t launch_depth_keys(int n, const float4 *rgbd, const uint32_t *counts, uint32_t *keys, uint32_t *vals,
                              cudaStream_t s);
template <typename KeyT>
cudaError_t launch_emit(const EmitArgs &a, KeyT *keys, cudaStream_t s);
template <typename KeyT>
cudaError_t launch_ranges(const KeyT *keys, uint64_t n_max, const uint64_t *n_dev, uint2 *ranges, int ntiles,
                          cudaStream_t s);
cudaError_t launch_tile_prep(int *tile_diff, const int *tile_single, const TileSet &ts, const uint32_t *diff_off,
                             const uint32_t *single_off, uint2 *ranges, uint32_t *hist, int hist_stride,
                             int digit_bits, int passes, uint64_t capacity, cudaStream_t s);
cudaError_t launch_render(const RenderArgs &a, int batch, cudaStream_t s);
cudaError_t launch_render_bwd(const BwdArgs &a, cudaStream_t s);
cudaError_t launch_preprocess_bwd(const PreBwdArgs &a, int deg, cudaStream_t s);

}  // namespace qb
