// qb_kernels.cuh -- kernel argument blocks and launchers of libquadbox.
#pragma once

#include "qb_internal.cuh"

namespace qb {

struct PreArgs {
    int n;
    const float *means, *scales, *quats, *opac, *sh;
    bool raw;
    bool sh_vec4;    // sh rows may be read as float4 (16-byte aligned)
    bool quat_vec4;  // quats may be read as float4 (16-byte aligned)
    CamDev cam;
    int mode;
    bool clamp3s;
    float2 *xy;
    float4 *conic_o, *rgbd, *box;
    float *r3;
    int *meta;
    uint32_t *counts;
    int *tile_diff;    // [(tiles_y+1)][(tiles_x+1)] difference array of per-tile pair counts, or null
    int *tile_single;  // [tiles] pair counts of single-tile Gaussians
    int tiles_x;
};

struct EmitArgs {
    int n;
    const uint32_t *perm;  // emission order -> Gaussian (null: index order)
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
    int W, H, tiles_x;
    uint32_t *err;
};

struct RenderArgs {
    const uint2 *ranges;
    const uint32_t *vals;
    const float2 *xy;
    const float4 *conic_o, *rgbd;
    int W, H, tiles_x, tiles_y;
    float bg[3];
    float *img;     // [3][H][W]
    float *tfinal;  // [H][W]
    int *ncontrib;  // [H][W]
    int *neval;     // [H][W]
};

struct BwdArgs {
    const uint2 *ranges;
    const uint32_t *vals;
    const float2 *xy;
    const float4 *conic_o, *rgbd;
    int W, H, tiles_x, tiles_y;
    float bg[3];
    const float *dL_dimg;  // [3][H][W]
    const float *tfinal;
    const int *ncontrib;
    double *g_screen;  // [n][9]: mu_x, mu_y, Sigma11, Sigma12, Sigma22, o, r, g, b
};

struct PreBwdArgs {
    int n;
    const float *means, *scales, *quats, *opac, *sh;
    bool raw;
    CamDev cam;
    const int *meta;
    const double *g_screen;  // [n][9]
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
cudaError_t launch_tile_prep(int *tile_diff, const int *tile_single, int tiles_x, int tiles_y, uint2 *ranges,
                             uint32_t *hist, int hist_stride, int digit_bits, int passes, cudaStream_t s);
cudaError_t launch_render(const RenderArgs &a, int batch, cudaStream_t s);
cudaError_t launch_render_bwd(const BwdArgs &a, cudaStream_t s);
cudaError_t launch_preprocess_bwd(const PreBwdArgs &a, int deg, cudaStream_t s);

}  // namespace qb
