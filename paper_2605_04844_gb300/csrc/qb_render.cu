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
// The thread's two pixels are evaluated together with the packed FP32x2
// instructions (fma/mul/add .f32x2); each packed lane rounds exactly like
// the scalar operation it replaces.  A tile ends as soon as all of its
// pixels have stopped.
#include "qb_kernels.cuh"

namespace qb {

constexpr int kRenderThreads = 128;  // two pixels per thread

// Per staged entry, five float4 in shared memory laid out for the packed
// FP32x2 arithmetic of sm_100+: every operand the two pixels of a thread
// share is stored twice, so a pair register loads it without a move.
//   sx = (mu_x, mu_x, mu_y, mu_y), sq = (ca, ca, cb, cb),
//   sk = (cc, cc, skip threshold, opacity), sc1 = (r, r, g, g), sc2 = (b, b, -, -).
struct RenderStage {
    float4 *sx, *sq, *sk, *sc1, *sc2;
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Both pixels of the thread are composited in lock step: every entry's
// exponent is evaluated for the pair with packed operations; entries whose
// exponent is out of range for every pixel of the warp skip the rest.  An
// entry a pixel rejects (or a pixel that has stopped) takes weight 0, which
// leaves its colour and transmittance bit-for-bit unchanged, so the branch-free
// update composes exactly the entries the per-pixel rules of the header accept.
template <int BATCH>
__device__ __forceinline__ void render_tile(const RenderArgs &a, uint32_t gtile, int ci, const RenderStage &S) {
    const CamTile &C = a.ts.cam[ci];
    const uint32_t lt = gtile - C.tile_base;
    const int tx = (int)(lt % (uint32_t)C.tiles_x), ty = (int)(lt / (uint32_t)C.tiles_x);
    const int tid = threadIdx.x;
    const int px = tx * kTile + (tid & (kTile - 1));
    const int py0 = ty * kTile + (tid >> kTileShift), py1 = py0 + 8;
    const bool in0 = px < C.W && py0 < C.H, in1 = px < C.W && py1 < C.H;
    const float2 npx = f2(-(float)px, -(float)px), npy = f2(-(float)py0, -(float)py1);
    bool done0 = !in0, done1 = !in1;

    const uint2 range = a.ranges[gtile];
    const int total = (int)(range.y - range.x);
    float2 T = f2(1.f, 1.f), cr = f2(0.f, 0.f), cg = f2(0.f, 0.f), cb = f2(0.f, 0.f);
    int n0 = 0, n1 = 0, last0 = 0, last1 = 0;

    for (int base = 0; base < total; base += BATCH) {
        if (__syncthreads_count(done0 && done1) == kRenderThreads) break;
        for (int q = tid; q < BATCH; q += kRenderThreads) {
            const int idx = base + q;
            if (idx < total) {
                const uint32_t g = a.vals[range.x + idx];
                const float2 m = a.xy[g];
                const float4 co = a.conic_o[g];
                const float4 rgb = a.rgbd[g];
                const float ca = -0.5f * co.x, cbv = -co.y, cc = -0.5f * co.z;
                S.sx[q] = make_float4(m.x, m.x, m.y, m.y);
                S.sq[q] = make_float4(ca, ca, cbv, cbv);
                S.sk[q] = make_float4(cc, cc, skip_threshold(co.w), co.w);
                S.sc1[q] = make_float4(rgb.x, rgb.x, rgb.y, rgb.y);
                S.sc2[q] = make_float4(rgb.z, rgb.z, 0.f, 0.f);
            }
        }
        __syncthreads();
        const int cnt = min(BATCH, total - base);
        for (int j = 0; j < cnt; ++j) {
            // every 32 entries: leave once all pixels of the warp have stopped
            if ((j & 31) == 0 && __all_sync(0xffffffffu, done0 && done1)) break;
            const float4 X = S.sx[j], Q = S.sq[j], K = S.sk[j];
            // power = A + dy (B + cc dy), A = ca dx^2, B = cb dx (the operation
            // sequence of power_terms / power_from, per pixel)
            const float2 dx = __fadd2_rn(f2(X.x, X.y), npx);
            const float2 A = __fmul2_rn(__fmul2_rn(f2(Q.x, Q.y), dx), dx);
            const float2 B = __fmul2_rn(f2(Q.z, Q.w), dx);
            const float2 dy = __fadd2_rn(f2(X.z, X.w), npy);
            const float2 pw = __ffma2_rn(dy, __ffma2_rn(f2(K.x, K.y), dy, B), A);
            const bool e0 = !done0 && pw.x <= 0.f && pw.x >= K.z;
            const bool e1 = !done1 && pw.y <= 0.f && pw.y >= K.z;
            if (!__any_sync(0xffffffffu, e0 || e1)) continue;
            const float a0 = fminf(kAlphaMax, __fmul_rn(K.w, __expf(pw.x)));
            const float a1 = fminf(kAlphaMax, __fmul_rn(K.w, __expf(pw.y)));
            const bool ok0 = e0 && a0 >= kAlphaMin, ok1 = e1 && a1 >= kAlphaMin;
            // T (1 - alpha); fma(alpha, -1, 1) is 1 - alpha rounded once
            const float2 tT = __fmul2_rn(T, __ffma2_rn(f2(a0, a1), f2(-1.f, -1.f), f2(1.f, 1.f)));
            const bool st0 = ok0 && tT.x < kTStop, st1 = ok1 && tT.y < kTStop;
            const bool ac0 = ok0 && !st0, ac1 = ok1 && !st1;
            // entries evaluated so far by a pixel still running: base + j + 1
            const int nj = base + j + 1;
            if (st0) n0 = nj;
            if (st1) n1 = nj;
            done0 = done0 || st0;
            done1 = done1 || st1;
            // alpha of the accepted entries, 0 elsewhere: T (1 - 0) = T and
            // c + r * 0 = c exactly, so the updates need no select
            const float2 aa = f2(ac0 ? a0 : 0.f, ac1 ? a1 : 0.f);
            const float2 w = __fmul2_rn(aa, T);
            const float4 C1 = S.sc1[j], C2 = S.sc2[j];
            cr = __ffma2_rn(f2(C1.x, C1.y), w, cr);
            cg = __ffma2_rn(f2(C1.z, C1.w), w, cg);
            cb = __ffma2_rn(f2(C2.x, C2.y), w, cb);
            T = __fmul2_rn(T, __ffma2_rn(aa, f2(-1.f, -1.f), f2(1.f, 1.f)));
            last0 = ac0 ? nj : last0;
            last1 = ac1 ? nj : last1;
        }
    }
    // a pixel that never stopped evaluated the whole list
    if (!done0) n0 = total;
    if (!done1) n1 = total;
    const size_t plane = (size_t)C.W * C.H;
    float *img = a.img + 3 * C.pix_base;
    if (in0) {
        const size_t pix = (size_t)py0 * C.W + px;
        img[pix] = fmaf(T.x, a.bg[0], cr.x);
        img[plane + pix] = fmaf(T.x, a.bg[1], cg.x);
        img[2 * plane + pix] = fmaf(T.x, a.bg[2], cb.x);
        a.tfinal[C.pix_base + pix] = T.x;
        a.ncontrib[C.pix_base + pix] = last0;
        a.neval[C.pix_base + pix] = n0;
    }
    if (in1) {
        const size_t pix = (size_t)py1 * C.W + px;
        img[pix] = fmaf(T.y, a.bg[0], cr.y);
        img[plane + pix] = fmaf(T.y, a.bg[1], cg.y);
        img[2 * plane + pix] = fmaf(T.y, a.bg[2], cb.y);
        a.tfinal[C.pix_base + pix] = T.y;
        a.ncontrib[C.pix_base + pix] = last1;
        a.neval[C.pix_base + pix] = n1;
    }
}

// One block per tile of a single camera.
template <int BATCH>
__global__ void __launch_bounds__(kRenderThreads) render_kernel(RenderArgs a) {
    __shared__ float4 s_stage[5][BATCH];
    const RenderStage S{s_stage[0], s_stage[1], s_stage[2], s_stage[3], s_stage[4]};
    render_tile<BATCH>(a, blockIdx.x, 0, S);
}

// Persistent blocks take tiles_per_fetch consecutive tiles at a time from a
// global counter over the tiles of all cameras in the set.
template <int BATCH>
__global__ void __launch_bounds__(kRenderThreads) render_persistent_kernel(RenderArgs a) {
    __shared__ float4 s_stage[5][BATCH];
    __shared__ uint32_t s_next;
    const RenderStage S{s_stage[0], s_stage[1], s_stage[2], s_stage[3], s_stage[4]};
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(a.queue, (uint32_t)a.tiles_per_fetch);
        __syncthreads();
        const uint32_t t0 = s_next;
        __syncthreads();
        if (t0 >= a.ts.total_tiles) break;
        const uint32_t t1 = min(t0 + (uint32_t)a.tiles_per_fetch, a.ts.total_tiles);
        for (uint32_t t = t0; t < t1; ++t) render_tile<BATCH>(a, t, camera_of(a.ts, t), S);
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
