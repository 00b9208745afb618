// qb_render.cu -- K6: tile-parallel front-to-back compositing (Sec. 2
// "Render", Eq. 2), as one block per tile (single frame) or as a persistent
// kernel that takes tiles of several cameras from a global work queue.
//
// A tile is rendered by 128 threads, each owning two pixels of one column
// (rows r and r + 8).  The tile's depth-sorted Gaussian list is walked in
// batches staged in shared memory (mu^2D, the skip threshold, opacity, the
// rescaled conic and the colour).  Per entry and pixel (3DGS conventions):
//   power = -(a dx^2 + 2 b dx dy + c dy^2)/2, skip if power > 0 or if it is
//   so low that alpha is certainly below 1/255;
//   alpha = min(0.99, o e^power), skip if alpha < 1/255;
//   T' = T (1 - alpha); stop before adding once T' < 1e-4;
//   C += alpha T c; T = T'.
// The column terms of the exponent are shared by the thread's two pixels.
// A tile ends as soon as all of its pixels have stopped.
#include "qb_kernels.cuh"

namespace qb {

constexpr int kRenderThreads = 128;  // two pixels per thread

template <int BATCH>
__device__ __forceinline__ void render_tile(const RenderArgs &a, uint32_t gtile, int ci, float4 *s_m, float4 *s_c,
                                            float4 *s_rgb) {
    const CamTile &C = a.ts.cam[ci];
    const uint32_t lt = gtile - C.tile_base;
    const int tx = (int)(lt % (uint32_t)C.tiles_x), ty = (int)(lt / (uint32_t)C.tiles_x);
    const int tid = threadIdx.x;
    const int px = tx * kTile + (tid & (kTile - 1));
    const int py0 = ty * kTile + (tid >> kTileShift), py1 = py0 + 8;
    const bool in0 = px < C.W && py0 < C.H, in1 = px < C.W && py1 < C.H;
    const float pxf = (float)px, py0f = (float)py0, py1f = (float)py1;
    bool done0 = !in0, done1 = !in1;

    const uint2 range = a.ranges[gtile];
    const int total = (int)(range.y - range.x);
    float T0 = 1.f, T1 = 1.f;
    float c00 = 0.f, c01 = 0.f, c02 = 0.f, c10 = 0.f, c11 = 0.f, c12 = 0.f;
    int n0 = 0, n1 = 0, last0 = 0, last1 = 0;

    for (int base = 0; base < total; base += BATCH) {
        if (__syncthreads_count(done0 && done1) == kRenderThreads) break;
        for (int q = tid; q < BATCH; q += kRenderThreads) {
            const int idx = base + q;
            if (idx < total) {
                const uint32_t g = a.vals[range.x + idx];
                const float2 m = a.xy[g];
                const float4 co = a.conic_o[g];
                s_m[q] = make_float4(m.x, m.y, skip_threshold(co.w), co.w);
                s_c[q] = make_float4(-0.5f * co.x, -co.y, -0.5f * co.z, 0.f);
                s_rgb[q] = a.rgbd[g];
            }
        }
        __syncthreads();
        const int cnt = min(BATCH, total - base);
        for (int j = 0; j < cnt && !(done0 && done1); ++j) {
            const float4 m = s_m[j];
            const float4 c = s_c[j];
            float A, B;
            power_terms(c.x, c.y, m.x - pxf, A, B);
            if (!done0) {
                ++n0;
                const float power = power_from(A, B, c.z, m.y - py0f);
                if (power <= 0.f && power >= m.z) {
                    const float alpha = fminf(kAlphaMax, __fmul_rn(m.w, __expf(power)));
                    if (alpha >= kAlphaMin) {
                        const float testT = __fmul_rn(T0, 1.f - alpha);
                        if (testT < kTStop) {
                            done0 = true;
                        } else {
                            const float4 rgb = s_rgb[j];
                            const float w = alpha * T0;
                            c00 = fmaf(rgb.x, w, c00);
                            c01 = fmaf(rgb.y, w, c01);
                            c02 = fmaf(rgb.z, w, c02);
                            T0 = testT;
                            last0 = n0;
                        }
                    }
                }
            }
            if (!done1) {
                ++n1;
                const float power = power_from(A, B, c.z, m.y - py1f);
                if (power <= 0.f && power >= m.z) {
                    const float alpha = fminf(kAlphaMax, __fmul_rn(m.w, __expf(power)));
                    if (alpha >= kAlphaMin) {
                        const float testT = __fmul_rn(T1, 1.f - alpha);
                        if (testT < kTStop) {
                            done1 = true;
                        } else {
                            const float4 rgb = s_rgb[j];
                            const float w = alpha * T1;
                            c10 = fmaf(rgb.x, w, c10);
                            c11 = fmaf(rgb.y, w, c11);
                            c12 = fmaf(rgb.z, w, c12);
                            T1 = testT;
                            last1 = n1;
                        }
                    }
                }
            }
        }
    }
    const size_t plane = (size_t)C.W * C.H;
    float *img = a.img + 3 * C.pix_base;
    if (in0) {
        const size_t pix = (size_t)py0 * C.W + px;
        img[pix] = fmaf(T0, a.bg[0], c00);
        img[plane + pix] = fmaf(T0, a.bg[1], c01);
        img[2 * plane + pix] = fmaf(T0, a.bg[2], c02);
        a.tfinal[C.pix_base + pix] = T0;
        a.ncontrib[C.pix_base + pix] = last0;
        a.neval[C.pix_base + pix] = n0;
    }
    if (in1) {
        const size_t pix = (size_t)py1 * C.W + px;
        img[pix] = fmaf(T1, a.bg[0], c10);
        img[plane + pix] = fmaf(T1, a.bg[1], c11);
        img[2 * plane + pix] = fmaf(T1, a.bg[2], c12);
        a.tfinal[C.pix_base + pix] = T1;
        a.ncontrib[C.pix_base + pix] = last1;
        a.neval[C.pix_base + pix] = n1;
    }
}

// One block per tile of a single camera.
template <int BATCH>
__global__ void __launch_bounds__(kRenderThreads) render_kernel(RenderArgs a) {
    __shared__ float4 s_m[BATCH], s_c[BATCH], s_rgb[BATCH];
    render_tile<BATCH>(a, blockIdx.x, 0, s_m, s_c, s_rgb);
}

// Persistent blocks take tiles_per_fetch consecutive tiles at a time from a
// global counter over the tiles of all cameras in the set.
template <int BATCH>
__global__ void __launch_bounds__(kRenderThreads) render_persistent_kernel(RenderArgs a) {
    __shared__ float4 s_m[BATCH], s_c[BATCH], s_rgb[BATCH];
    __shared__ uint32_t s_next;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(a.queue, (uint32_t)a.tiles_per_fetch);
        __syncthreads();
        const uint32_t t0 = s_next;
        __syncthreads();
        if (t0 >= a.ts.total_tiles) break;
        const uint32_t t1 = min(t0 + (uint32_t)a.tiles_per_fetch, a.ts.total_tiles);
        for (uint32_t t = t0; t < t1; ++t) render_tile<BATCH>(a, t, camera_of(a.ts, t), s_m, s_c, s_rgb);
    }
}

template <int BATCH>
static cudaError_t launch_render_b(const RenderArgs &a, cudaStream_t s) {
    if (a.queue) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_persistent_kernel<BATCH>, kRenderThreads, 0);
        if (a.blocks_per_sm > 0 && a.blocks_per_sm < per_sm) per_sm = a.blocks_per_sm;
        note_launch("render_persistent_kernel", s), render_persistent_kernel<BATCH><<<sms * (per_sm > 0 ? per_sm : 1), kRenderThreads, 0, s>>>(a);
    } else {
        note_launch("render_kernel", s), render_kernel<BATCH><<<a.ts.total_tiles, kRenderThreads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_render(const RenderArgs &a, int batch, cudaStream_t s) {
    if (a.ts.total_tiles == 0) return cudaSuccess;
    switch (batch) {
    case 64: return launch_render_b<64>(a, s);
    case 128: return launch_render_b<128>(a, s);
    default: return launch_render_b<256>(a, s);
    }
}

}  // namespace qb
