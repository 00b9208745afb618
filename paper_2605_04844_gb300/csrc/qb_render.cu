// qb_render.cu -- K6: tile-parallel front-to-back compositing (Sec. 2
// "Render", Eq. 2).
//
// One 256-thread block per 16x16 tile, one pixel per thread.  The tile's
// depth-sorted Gaussian list is walked in batches: each thread stages one
// Gaussian (mu^2D, conic+opacity, colour) into shared memory, then every
// pixel consumes the batch.  Per entry (3DGS conventions):
//   q = a dx^2 + 2 b dx dy + c dy^2, skip if -q/2 > 0 (and, before the exp,
//   skip exponents so low that alpha is certainly below 1/255);
//   alpha = min(0.99, o exp(-q/2)), skip if alpha < 1/255;
//   T' = T (1 - alpha); stop before adding once T' < 1e-4;
//   C += alpha T c; T = T'.
// The block leaves as soon as every pixel has stopped.
#include "qb_kernels.cuh"

namespace qb {

constexpr int kRenderThreads = kTile * kTile;

__global__ void __launch_bounds__(kRenderThreads) render_kernel(RenderArgs a) {
    __shared__ float4 s_xy[kRenderThreads];  // mu_x, mu_y, skip threshold on the exponent
    __shared__ float4 s_co[kRenderThreads];
    __shared__ float4 s_rgb[kRenderThreads];

    const int tile = blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int tid = threadIdx.x;
    const int px = tx * kTile + (tid & (kTile - 1));
    const int py = ty * kTile + (tid >> kTileShift);
    const bool inside = px < a.W && py < a.H;
    const float pxf = (float)px, pyf = (float)py;
    bool done = !inside;

    const uint2 range = a.ranges[tile];
    const int total = (int)(range.y - range.x);
    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    int contributor = 0, last = 0;

    for (int base = 0; base < total; base += kRenderThreads) {
        if (__syncthreads_count(done) == kRenderThreads) break;
        const int idx = base + tid;
        if (idx < total) {
            const uint32_t g = a.vals[range.x + idx];
            const float2 m = a.xy[g];
            const float4 co = a.conic_o[g];
            s_xy[tid] = make_float4(m.x, m.y, skip_threshold(co.w), 0.f);
            s_co[tid] = co;
            s_rgb[tid] = a.rgbd[g];
        }
        __syncthreads();
        const int cnt = min(kRenderThreads, total - base);
        for (int j = 0; !done && j < cnt; ++j) {
            ++contributor;
            const float4 m = s_xy[j];
            const float4 co = s_co[j];
            const float dx = m.x - pxf, dy = m.y - pyf;
            const float power = eval_power(co, dx, dy);
            if (power > 0.f || power < m.z) continue;  // m.z: alpha certainly below 1/255
            const float alpha = fminf(kAlphaMax, __fmul_rn(co.w, __expf(power)));
            if (alpha < kAlphaMin) continue;
            const float testT = __fmul_rn(T, 1.f - alpha);
            if (testT < kTStop) {
                done = true;
                continue;
            }
            const float4 c = s_rgb[j];
            const float w = alpha * T;
            C0 = fmaf(c.x, w, C0);
            C1 = fmaf(c.y, w, C1);
            C2 = fmaf(c.z, w, C2);
            T = testT;
            last = contributor;
        }
    }
    if (inside) {
        const size_t pix = (size_t)py * a.W + px;
        const size_t plane = (size_t)a.W * a.H;
        a.img[pix] = fmaf(T, a.bg[0], C0);
        a.img[plane + pix] = fmaf(T, a.bg[1], C1);
        a.img[2 * plane + pix] = fmaf(T, a.bg[2], C2);
        a.tfinal[pix] = T;
        a.ncontrib[pix] = last;
        a.neval[pix] = contributor;
    }
}

cudaError_t launch_render(const RenderArgs &a, int batch, cudaStream_t s) {
    (void)batch;
    const int ntiles = a.tiles_x * a.tiles_y;
    if (ntiles == 0) return cudaSuccess;
    render_kernel<<<ntiles, kRenderThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace qb
