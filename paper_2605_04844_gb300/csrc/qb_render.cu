// qb_render.cu -- K6: tile-parallel front-to-back compositing (Sec. 2
// "Render", Eq. 2), as one block per tile (single frame) or as a persistent
// kernel that takes tiles of several cameras from a global work queue.
//
// A tile is rendered by 64 threads, two warps each owning one half of the
// tile (rows 0-7 or 8-15); a thread owns four pixels of one column of its
// half, rows r, r + 2, r + 4 and r + 6, evaluated as two packed pairs (r, r + 2)
// and (r + 4, r + 6) that share the column's dx terms.  The tile's
// depth-sorted Gaussian list is walked in
// batches staged in shared memory (mu^2D, the skip threshold, opacity, the
// rescaled conic and the colour).  Per entry and pixel (3DGS conventions):
//   power = -(a dx^2 + 2 b dx dy + c dy^2)/2, skip if it is so low that alpha
//   is certainly below 1/255 (power > 0 arises only as a float32 rounding of
//   0 and is kept);
//   alpha = min(0.99, o e^power), skip if alpha < 1/255;
//   T' = T (1 - alpha); stop before adding once T' < 1e-4;
//   C += alpha T c; T = T'.
// Each pair is evaluated with the packed FP32x2 instructions (fma/mul/add
// .f32x2); each packed lane rounds exactly like the scalar operation it
// replaces.  A tile ends as soon as all of its pixels have stopped.
// While staging a batch, each entry's alpha ellipse is tested against the
// two half tiles (ellipse_meets_rect); a warp then walks only the entries
// that reach its half, a third of the warp-entries of a 1M-Gaussian 1080p
// frame fewer, with identical results (a skipped entry is one every pixel of
// the half would have rejected).
#include "qb_kernels.cuh"

namespace qb {

constexpr int kRenderThreads = 64;  // four pixels per thread
constexpr float kCapTest = 0.98f;    // opacities above this may meet the 0.99 cap
#define kNaN __int_as_float(0x7fc00000)
constexpr int kRenderPairs = 2;     // packed pixel pairs per thread

// Per staged entry, five float4 in shared memory laid out for the packed
// FP32x2 arithmetic of sm_100+: every operand the two pixels of a pair
// share is stored twice, so a pair register loads it without a move.
//   sx = (mu_x, mu_x, mu_y, mu_y), sq = (ca, ca, cb, cb),
//   sk = (cc, cc, skip threshold, +-opacity), sc1 = (r, r, g, g),
//   sc2 = (b, b, rr, ce).
// An elongated Gaussian (qb_internal.cuh) carries a negative opacity and the
// exact power form's rr = b / a and ce = -1 / (2 Sigma22): its exponent is
// ca u^2 + ce dy^2 with u = dx + rr dy, which does not cancel.
// mask[w * BATCH / 32 + k] holds, for warp w (rows 8w .. 8w + 7 of the tile),
// one bit per entry 32k .. 32k + 31 of the batch: set where the entry's
// alpha ellipse (exponent above its skip threshold) meets the warp's 16 x 8
// pixels.  A warp walks only the set bits; every pixel of a cleared entry
// would have rejected it.
struct RenderStage {
    float4 *sx, *sq, *sk, *sc1, *sc2;
    uint32_t *mask;
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// The compositing state of one packed pair of pixels.
struct RenderPair {
    float2 T, cr, cg, cb, npy;
    bool done0, done1;
    int n0, n1, last0, last1;  // n0, n1: the counted variant only
};

// Both pixels of a pair are composited in lock step: every entry's exponent
// is evaluated for the pair with packed operations; entries whose exponent
// is out of range for every pixel of the warp skip the rest.  An entry a
// pixel rejects (or a pixel that has stopped) takes weight 0, which leaves
// its colour and transmittance bit-for-bit unchanged, so the branch-free
// update composes exactly the entries the per-pixel rules of the header
// accept.
// COUNT (measurement only) also adds the tile's (pixel, entry) evaluations
// and the evaluations whose power test passed to a.counts[0], a.counts[1].
template <int BATCH, bool COUNT = false>
__device__ __forceinline__ void render_tile(const RenderArgs &a, uint32_t gtile, const CamTile &C, const RenderStage &S) {
    const uint32_t lt = gtile - C.tile_base;
    const uint32_t *vals = a.vals + C.vals_base;
    const int tx = (int)(lt % (uint32_t)C.tiles_x), ty = (int)(lt / (uint32_t)C.tiles_x);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int px = tx * kTile + (lane & (kTile - 1));
    const int pyb = ty * kTile + wid * 8 + (lane >> kTileShift);
    const float2 npx = f2(-(float)px, -(float)px);
    RenderPair P[kRenderPairs];
#pragma unroll
    for (int r = 0; r < kRenderPairs; ++r) {
        const int y0 = pyb + 4 * r, y1 = y0 + 2;
        const bool in0 = px < C.W && y0 < C.H, in1 = px < C.W && y1 < C.H;
        P[r].done0 = !in0;
        P[r].done1 = !in1;
        // a pixel outside the image (later: one that has stopped) carries a
        // NaN row, so its exponent is NaN and fails every test
        P[r].npy = f2(in0 ? -(float)y0 : kNaN, in1 ? -(float)y1 : kNaN);
        P[r].T = f2(1.f, 1.f);
        P[r].cr = P[r].cg = P[r].cb = f2(0.f, 0.f);
        P[r].n0 = P[r].n1 = P[r].last0 = P[r].last1 = 0;
    }
    auto all_done = [&]() {
        bool d = true;
#pragma unroll
        for (int r = 0; r < kRenderPairs; ++r) d = d && P[r].done0 && P[r].done1;
        return d;
    };

    const uint2 range = a.ranges[gtile];
    const int total = (int)(range.y - range.x);
    uint32_t npass = 0;  // COUNT only

    for (int base = 0; base < total; base += BATCH) {
        if (__syncthreads_count(all_done()) == kRenderThreads) break;
#pragma unroll 1
        for (int q = tid; q < BATCH; q += kRenderThreads) {
            const int idx = base + q;
            bool hit0 = false, hit1 = false;
            if (idx < total) {
                const uint32_t g = C.rec_base + vals[range.x + idx];
                const float2 m = a.xy[g];
                const float4 co = a.conic_o[g];
                const float4 rgb = a.rgbd[g];
                const float2 sh = a.shape[g];
                const float ca = -0.5f * co.x, cbv = -co.y, cc = -0.5f * co.z;
                const float skip = skip_threshold(co.w);
                S.sx[q] = make_float4(m.x, m.x, m.y, m.y);
                S.sq[q] = make_float4(ca, ca, cbv, cbv);
                S.sk[q] = make_float4(cc, cc, skip, sh.y != 0.f ? -co.w : co.w);
                S.sc1[q] = make_float4(rgb.x, rgb.x, rgb.y, rgb.y);
                S.sc2[q] = make_float4(rgb.z, rgb.z, sh.x, sh.y);
                const float x0 = (float)(tx * kTile), y0 = (float)(ty * kTile);
                hit0 = ellipse_meets_rect(m.x, m.y, co.x, co.y, co.z, skip, sh.y != 0.f, x0, y0, x0 + 15.f, y0 + 7.f);
                hit1 = ellipse_meets_rect(m.x, m.y, co.x, co.y, co.z, skip, sh.y != 0.f, x0, y0 + 8.f, x0 + 15.f,
                                          y0 + 15.f);
            }
            const uint32_t b0 = __ballot_sync(0xffffffffu, hit0), b1 = __ballot_sync(0xffffffffu, hit1);
            if (lane == 0) {
                S.mask[q >> 5] = b0;
                S.mask[BATCH / 32 + (q >> 5)] = b1;
            }
        }
        __syncthreads();
        const int cnt = min(BATCH, total - base);
        for (int w0 = 0; w0 < cnt; w0 += 32) {
            // every 32 entries: leave once all pixels of the warp have stopped
            if (__all_sync(0xffffffffu, all_done())) break;
            uint32_t bits = S.mask[wid * (BATCH / 32) + (w0 >> 5)];
            while (bits) {
                const int j = w0 + __ffs(bits) - 1;
                bits &= bits - 1;
                const float4 X = S.sx[j], Q = S.sq[j], K = S.sk[j];
                const float2 dx = __fadd2_rn(f2(X.x, X.y), npx);
                float2 pw[kRenderPairs];
                if (K.w >= 0.f) {
                    // power = A + dy (B + cc dy), A = ca dx^2, B = cb dx; dx, A and
                    // B are the column's, shared by the thread's four pixels
                    const float2 A = __fmul2_rn(__fmul2_rn(f2(Q.x, Q.y), dx), dx);
                    const float2 B = __fmul2_rn(f2(Q.z, Q.w), dx);
#pragma unroll
                    for (int r = 0; r < kRenderPairs; ++r) {
                        const float2 dy = __fadd2_rn(f2(X.z, X.w), P[r].npy);
                        pw[r] = __ffma2_rn(dy, __ffma2_rn(f2(K.x, K.y), dy, B), A);
                    }
                } else {
                    // elongated (the same for the whole warp): power = ca u^2 +
                    // ce dy^2, u = dx + rr dy
                    const float4 E = S.sc2[j];
#pragma unroll
                    for (int r = 0; r < kRenderPairs; ++r) {
                        const float2 dy = __fadd2_rn(f2(X.z, X.w), P[r].npy);
                        const float2 u = __ffma2_rn(f2(E.z, E.z), dy, dx);
                        pw[r] = __ffma2_rn(__fmul2_rn(f2(Q.x, Q.y), u), u, __fmul2_rn(__fmul2_rn(f2(E.w, E.w), dy), dy));
                    }
                }
                const float op = fabsf(K.w);
                bool e0[kRenderPairs], e1[kRenderPairs];
                bool any = false;
#pragma unroll
                for (int r = 0; r < kRenderPairs; ++r) {
                    // power >= skip; the rule power <= 0 needs no test: a
                    // positive exponent is a float32 rounding of 0 (the conic is
                    // positive definite), where alpha = o e^power rounds like o
                    e0[r] = pw[r].x >= K.z;
                    e1[r] = pw[r].y >= K.z;
                    if (COUNT) npass += (uint32_t)e0[r] + (uint32_t)e1[r];
                    any = any || e0[r] || e1[r];
                }
                if (!__any_sync(0xffffffffu, any)) continue;
                const float4 C1 = S.sc1[j], C2 = S.sc2[j];
                // entries evaluated so far by a pixel still running: base + j + 1
                const int nj = base + j + 1;
                // o G can reach the 0.99 cap only for o near it (G <= 1 up to
                // the exponential's rounding); the same for the whole warp
                const bool capped = op > kCapTest;
#pragma unroll
                for (int r = 0; r < kRenderPairs; ++r) {
                    RenderPair &q = P[r];
                    float2 al = __fmul2_rn(f2(op, op), f2(__expf(pw[r].x), __expf(pw[r].y)));
                    if (capped) al = f2(fminf(kAlphaMax, al.x), fminf(kAlphaMax, al.y));
                    const float a0 = al.x, a1 = al.y;
                    const bool ok0 = e0[r] && a0 >= kAlphaMin, ok1 = e1[r] && a1 >= kAlphaMin;
                    // T (1 - alpha); fma(alpha, -1, 1) is 1 - alpha rounded once
                    const float2 tT = __fmul2_rn(q.T, __ffma2_rn(al, f2(-1.f, -1.f), f2(1.f, 1.f)));
                    const bool st0 = ok0 && tT.x < kTStop, st1 = ok1 && tT.y < kTStop;
                    const bool ac0 = ok0 && !st0, ac1 = ok1 && !st1;
                    if (st0 || st1) {  // once in a pixel's life: record the stop, poison its row
                        if (st0) q.done0 = true, q.npy.x = kNaN;
                        if (st1) q.done1 = true, q.npy.y = kNaN;
                        if (COUNT && st0) q.n0 = nj;
                        if (COUNT && st1) q.n1 = nj;
                    }
                    // alpha of the accepted entries, 0 elsewhere: T (1 - 0) = T and
                    // c + r * 0 = c exactly, so the updates need no select
                    const float2 aa = f2(ac0 ? a0 : 0.f, ac1 ? a1 : 0.f);
                    const float2 w = __fmul2_rn(aa, q.T);
                    q.cr = __ffma2_rn(f2(C1.x, C1.y), w, q.cr);
                    q.cg = __ffma2_rn(f2(C1.z, C1.w), w, q.cg);
                    q.cb = __ffma2_rn(f2(C2.x, C2.y), w, q.cb);
                    q.T = __fmul2_rn(q.T, __ffma2_rn(aa, f2(-1.f, -1.f), f2(1.f, 1.f)));
                    q.last0 = ac0 ? nj : q.last0;
                    q.last1 = ac1 ? nj : q.last1;
                }
            }
        }
    }
    const size_t plane = (size_t)C.W * C.H;
    float *img = a.img + 3 * C.pix_base;
    unsigned long long ev = 0;
#pragma unroll
    for (int r = 0; r < kRenderPairs; ++r) {
        RenderPair &q = P[r];
        // a pixel that never stopped evaluated the whole list
        if (COUNT && !q.done0) q.n0 = total;
        if (COUNT && !q.done1) q.n1 = total;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int py = pyb + 4 * r + 2 * h;
            if (px >= C.W || py >= C.H) continue;
            const size_t pix = (size_t)py * C.W + px;
            const float T = h ? q.T.y : q.T.x;
            img[pix] = fmaf(T, a.bg[0], h ? q.cr.y : q.cr.x);
            img[plane + pix] = fmaf(T, a.bg[1], h ? q.cg.y : q.cg.x);
            img[2 * plane + pix] = fmaf(T, a.bg[2], h ? q.cb.y : q.cb.x);
            a.tfinal[C.pix_base + pix] = T;
            a.ncontrib[C.pix_base + pix] = h ? q.last1 : q.last0;
            if (COUNT) {
                a.neval[C.pix_base + pix] = h ? q.n1 : q.n0;
                ev += (unsigned long long)(h ? q.n1 : q.n0);
            }
        }
    }
    if (a.order_out.cnt) {
        // the tile's largest last-contributor count (the backward walks that
        // many entries) files it for the backward
        __shared__ int s_last[2];
        int m = 0;
#pragma unroll
        for (int r = 0; r < kRenderPairs; ++r) m = max(m, max(P[r].last0, P[r].last1));
        m = __reduce_max_sync(0xffffffffu, m);
        if (lane == 0) s_last[wid] = m;
        __syncthreads();
        if (tid == 0) order_file(a.order_out, a.ts.total_tiles, gtile, (uint32_t)max(s_last[0], s_last[1]));
    }
    if (COUNT) {
        unsigned long long ps = npass;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ev += __shfl_xor_sync(0xffffffffu, ev, o);
            ps += __shfl_xor_sync(0xffffffffu, ps, o);
        }
        if (lane == 0) {
            atomicAdd(a.counts, ev);
            atomicAdd(a.counts + 1, ps);
        }
    }
}

// One block per tile of a single camera; with an order, the blocks (which
// start roughly in index order) take the heaviest tiles first, so that the
// last blocks to start are short ones.
template <int BATCH, bool COUNT>
__global__ void __launch_bounds__(kRenderThreads) render_kernel(RenderArgs a) {
    __shared__ float4 s_stage[5][BATCH];
    __shared__ uint32_t s_mask[2 * BATCH / 32];
    const RenderStage S{s_stage[0], s_stage[1], s_stage[2], s_stage[3], s_stage[4], s_mask};
    const uint32_t t = a.order.cnt ? order_pick(a.order, a.ts.total_tiles, blockIdx.x) : (uint32_t)blockIdx.x;
    render_tile<BATCH, COUNT>(a, t, a.ts.cam[0], S);
}

// A warp per tile walks the tile's list 32 entries at a time for four sample
// pixels (offsets 3 and 12 in x and y): each lane takes one entry's
// 1 - alpha at each pixel (the render's accept rules on the plain conic
// form), a product scan over the lanes gives the transmittance after every
// entry, and the first entry that takes a pixel below the stop ends that
// pixel.  The estimate is the largest stop position, or the list length when
// a pixel has not stopped within kWorkChunks chunks.  The next chunk's
// records and the one after's indices are loaded while a chunk is scanned.
constexpr int kWorkPix = 4;  // sample pixels per tile, at these offsets in the tile
__device__ constexpr int kWorkX[kWorkPix] = {3, 12, 3, 12};
__device__ constexpr int kWorkY[kWorkPix] = {3, 3, 12, 12};
constexpr uint32_t kWorkChunks = 32;  // beyond 1024 entries every tile files into the top bucket
__global__ void __launch_bounds__(256) tile_work_kernel(RenderArgs a) {
    const int lane = threadIdx.x & 31;
    const uint32_t t = blockIdx.x * 8u + (threadIdx.x >> 5);
    if (t >= a.ts.total_tiles) return;  // warp-uniform
    const CamTile &C = a.ts.cam[0];
    const int tx = (int)(t % (uint32_t)C.tiles_x), ty = (int)(t / (uint32_t)C.tiles_x);
    float sx[kWorkPix], sy[kWorkPix], T[kWorkPix];
    bool done[kWorkPix];
#pragma unroll
    for (int k = 0; k < kWorkPix; ++k) {
        const int x = tx * kTile + kWorkX[k], y = ty * kTile + kWorkY[k];
        sx[k] = (float)x;
        sy[k] = (float)y;
        T[k] = 1.f;
        done[k] = x >= C.W || y >= C.H;
    }
    const uint2 range = a.ranges[t];
    const uint32_t total = range.y - range.x;
    const uint32_t *vals = a.vals + range.x;
    // records of chunk 0, indices of chunk 1
    float2 m = make_float2(0.f, 0.f);
    float4 co = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane < total) {
        const uint32_t g = vals[lane];
        m = a.xy[g];
        co = a.conic_o[g];
    }
    uint32_t gn = 32 + lane < total ? vals[32 + lane] : 0u;
    uint32_t work = 0;
    bool open = true;
    for (uint32_t c = 0; c < kWorkChunks && 32 * c < total; ++c) {
        const uint32_t base = 32 * c;
        const bool have = base + lane < total;
        const float2 mc = m;
        const float4 cc = co;
        if (base + 32 + lane < total) {  // prefetch: records of chunk c + 1, indices of chunk c + 2
            m = a.xy[gn];
            co = a.conic_o[gn];
            gn = base + 64 + lane < total ? vals[base + 64 + lane] : 0u;
        }
        float om[kWorkPix];
#pragma unroll
        for (int k = 0; k < kWorkPix; ++k) om[k] = 1.f;
        if (have) {
            const float skip = skip_threshold(cc.w);
#pragma unroll
            for (int k = 0; k < kWorkPix; ++k) {
                const float dx = mc.x - sx[k], dy = mc.y - sy[k];
                const float pw = -0.5f * (cc.x * dx * dx + cc.z * dy * dy) - cc.y * dx * dy;
                if (pw >= skip) {
                    const float al = fminf(kAlphaMax, cc.w * __expf(pw));
                    if (al >= kAlphaMin) om[k] = 1.f - al;
                }
            }
        }
        bool all = true;
#pragma unroll
        for (int k = 0; k < kWorkPix; ++k) {
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float v = __shfl_up_sync(0xffffffffu, om[k], o);
                if (lane >= o) om[k] *= v;
            }
            const float Tl = T[k] * om[k];
            const uint32_t stop = __ballot_sync(0xffffffffu, Tl < kTStop);
            if (!done[k] && stop) {
                done[k] = true;
                work = max(work, base + (uint32_t)__ffs(stop));
            }
            T[k] = __shfl_sync(0xffffffffu, Tl, 31);
            all = all && done[k];
        }
        if (all) {
            open = false;
            break;
        }
    }
    if (open) {
        bool any_open = false;
#pragma unroll
        for (int k = 0; k < kWorkPix; ++k) any_open = any_open || !done[k];
        if (any_open) work = total;
    }
    if (lane == 0) order_file(a.order, a.ts.total_tiles, t, work);
}

cudaError_t launch_tile_work(const RenderArgs &a, cudaStream_t s) {
    if (a.ts.total_tiles == 0) return cudaSuccess;
    note_launch("tile_work_kernel", s), tile_work_kernel<<<(a.ts.total_tiles + 7) / 8, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// Persistent blocks take tiles_per_fetch consecutive tiles at a time from a
// global counter over the tiles of all cameras in the set.
template <int BATCH>
__global__ void __launch_bounds__(kRenderThreads) render_persistent_kernel(RenderArgs a) {
    __shared__ float4 s_stage[5][BATCH];
    __shared__ uint32_t s_mask[2 * BATCH / 32];
    __shared__ uint32_t s_next;
    const RenderStage S{s_stage[0], s_stage[1], s_stage[2], s_stage[3], s_stage[4], s_mask};
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(a.queue, (uint32_t)a.tiles_per_fetch);
        __syncthreads();
        const uint32_t t0 = s_next;
        __syncthreads();
        if (t0 >= a.ts.total_tiles) break;
        const uint32_t t1 = min(t0 + (uint32_t)a.tiles_per_fetch, a.ts.total_tiles);
        for (uint32_t t = t0; t < t1; ++t) {
            if (a.cam_table) {
                const CamTile C = a.cam_table[camera_in_table(a.cam_table, a.ts.n_cams, t)];
                render_tile<BATCH>(a, t, C, S);
            } else {
                render_tile<BATCH>(a, t, a.ts.cam[camera_of(a.ts, t)], S);
            }
        }
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
    } else if (a.counts) {
        note_launch("render_kernel_counted", s),
            render_kernel<BATCH, true><<<a.ts.total_tiles, kRenderThreads, 0, s>>>(a);
    } else {
        note_launch("render_kernel", s), render_kernel<BATCH, false><<<a.ts.total_tiles, kRenderThreads, 0, s>>>(a);
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
