// qb_backward.cu -- K7 render backward and K8 preprocess backward of the
// differentiable rasteriser (Sec. 4.1 states the rasteriser is differentiable;
// the gradients below differentiate Eq. 2 and the Sec. 2 projection).
//
// K7: a 64-thread block per tile (each warp a half tile, four pixels of a
// column per thread, rows r, r+2, r+4, r+6 of the half, evaluated as two
// pairs with the packed FP32x2 instructions) walks the tile list in reverse,
// from the largest last-contributor position of its pixels down to 0; the
// blocks take the tiles by decreasing walk length, the order the forward
// render filed.  Each pixel recomputes
// alpha exactly as the forward did and the transmittance by division,
// T_k = T_{k+1} / (1 - alpha_k); with B_k = sum_{i>k} T_i alpha_i c_i + T_final bg
// the colour behind entry k,
//   dC/dc_k     = T_k alpha_k
//   dC/dalpha_k = T_k c_k - B_k / (1 - alpha_k)
// and B enters dL/dalpha only through S2 = sum_c dL/dC_c B_c, which is carried
// per pixel instead of B.  alpha = min(0.99, o G), G = exp(power): zero
// derivative where the cap binds.
// The 9 per-Gaussian sums (mu_x, mu_y, Sigma11, Sigma12, Sigma22, o, r, g, b;
// the covariance entries are the well-conditioned parametrisation, with
// dL/dLambda = -Sigma dL/dSigma Sigma) are reduced over the warp by a
// transpose-reduction (12 shuffles) that leaves one sum on each of 9 lanes,
// which add them to float64 accumulators in parallel.  The same tile routine
// serves one block per tile and a persistent kernel over several cameras.
//
// K8: one thread per Gaussian chains the (mu^2D, Sigma2D, o, colour)
// gradients of every camera of the set to means, (log-)scales, quaternions,
// opacity (logits) and SH, summing over cameras in registers.
#include "qb_kernels.cuh"
#include "qb_project.cuh"

namespace qb {

constexpr int kBwdPix = 4;                            // pixels per thread (one column)
constexpr int kBwdThreads = kTile * kTile / kBwdPix;  // threads per tile
static_assert(kBwdThreads == 64 && kBwdPix == 4, "two warps per tile, each a half tile of 16 x 8 pixels");
constexpr int kBwdBatch = 128;  // entries staged per shared-memory batch

// float -> double by rebuilding the IEEE-754 bit pattern with integer
// operations (exponent rebias 127 -> 1023, mantissa 23 -> 52 bits), so the
// float64 atomics below need no float64 arithmetic in the SM; float32
// subnormals (|v| < 1.2e-38) become zero.
__device__ __forceinline__ double widen(float v) {
    const uint32_t u = __float_as_uint(v);
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    const uint64_t bits = ((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                          ((uint64_t)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

// Sum g[0..8] over the warp and add the 9 totals to dst[0..8].  Each butterfly
// step halves the vector every lane carries (9 -> 5 -> 3 -> 2 -> 1): lanes on
// the lower side of a step keep the first half, those on the upper side the
// second half.  Afterwards lane l (bit 0 clear) holds element
// 5 b4 + 3 b3 + 2 b2 + b1 of the original vector, when that index is real.
__device__ __forceinline__ void warp_reduce9_add(const float g[9], double *dst, int lane) {
    const unsigned F = 0xffffffffu;
    float w[5];
    const bool u4 = lane & 16;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float lo = g[i], hi = (i + 5 < 9) ? g[i + 5] : 0.f;
        w[i] = (u4 ? hi : lo) + __shfl_xor_sync(F, u4 ? lo : hi, 16);
    }
    float x[3];
    const bool u3 = lane & 8;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float lo = w[i], hi = (i + 3 < 5) ? w[i + 3] : 0.f;
        x[i] = (u3 ? hi : lo) + __shfl_xor_sync(F, u3 ? lo : hi, 8);
    }
    float y[2];
    const bool u2 = lane & 4;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float lo = x[i], hi = (i + 2 < 3) ? x[i + 2] : 0.f;
        y[i] = (u2 ? hi : lo) + __shfl_xor_sync(F, u2 ? lo : hi, 4);
    }
    const bool u1 = lane & 2;
    float z = (u1 ? y[1] : y[0]) + __shfl_xor_sync(F, u1 ? y[0] : y[1], 2);
    z += __shfl_xor_sync(F, z, 1);
    const int ix = 2 * ((lane >> 2) & 1) + ((lane >> 1) & 1);
    const int iw = 3 * ((lane >> 3) & 1) + ix;
    const int iv = 5 * ((lane >> 4) & 1) + iw;
    if (!(lane & 1) && ix < 3 && iw < 5 && iv < 9 && z != 0.f) atomicAdd(dst + iv, widen(z));
}

// Staged entries of a backward batch, laid out for the packed FP32x2
// arithmetic (operands the pixels of a thread share are stored twice):
//   s0 = (mu_x, mu_x, mu_y, mu_y), s1 = (ca, ca, cb, cb),
//   s2 = (cc, cc, skip threshold, elongated), s3 = (r, r, g, g), s4 = (b, b, o, o),
//   s5 = (rr, rr, ce, ce),
// with (ca, cb, cc) = (-a/2, -b, -c/2) the rescaled conic of the forward and,
// for an elongated Gaussian (s2.w = 1), the exact power form's terms
// (qb_render.cu): power = ca u^2 + ce dy^2, u = dx + rr dy.
struct BwdStage {
    uint32_t *id;
    float4 *s0, *s1, *s2, *s3, *s4, *s5;
    int *maxlast;
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// The per-pixel state of a pair of pixels (one packed lane each): the
// transmittance in front of the current entry, T; -S2 with
// S2 = sum_c dL/dC_c B_c (the colour behind the entry, B_c, only enters the
// gradient through this sum, which is updated as S2 += w S1 when an entry of
// weight w = alpha T is passed); and dL/dC per channel.
struct BwdPair {
    float2 T, nS2, g0, g1, g2, npy;
    int last0, last1;
};

// A tile by kBwdThreads threads: two warps, each owning one half of the tile
// (rows 0-7 or 8-15, a compact footprint, so a small ellipse reaches one
// warp more often than both); a thread owns kBwdPix pixels of one column of
// its half (rows r, r + 2, r + 4, r + 6) as two packed pairs (r, r + 2) and
// (r + 4, r + 6).  Per entry, for every pixel:
//   T <- T / (1 - alpha)                       (T in front of the entry)
//   dL/dc_k     += alpha T dL/dC
//   dL/dalpha    = T S1 - S2 / (1 - alpha),    S1 = sum_c dL/dC_c c_k,c
//   S2          += alpha T S1
// and, where the opacity cap does not bind (o G < 0.99), with
// v = -dpower/dmu = (2 ca dx + cb dy, cb dx + 2 cc dy):
//   dL/do += G dL/dalpha, dpower = o G dL/dalpha,
//   dL/dmu += dpower v, dL/dSigma += dpower (vx^2/2, vx vy, vy^2/2).
// An entry a pixel does not composite takes alpha = 0 (T, S2 unchanged, no
// contribution), so the pairs run in lock step without branches.
__device__ __forceinline__ void render_bwd_tile(const BwdArgs &a, uint32_t gtile, const CamTile &C, const BwdStage &S) {
    const uint32_t lt = gtile - C.tile_base;
    const uint32_t *vals = a.vals + C.vals_base;
    const int tx = (int)(lt % (uint32_t)C.tiles_x), ty = (int)(lt / (uint32_t)C.tiles_x);
    const int tid = threadIdx.x, lane = tid & 31;
    const int px = tx * kTile + (lane & (kTile - 1));
    const int py_first = ty * kTile + (tid >> 5) * 8 + (lane >> kTileShift);
    const float2 npx = f2(-(float)px, -(float)px);
    const size_t plane = (size_t)C.W * C.H;
    const float *dl = a.dL_dimg + 3 * C.pix_base;

    BwdPair P[2];
    int mylast = 0;
#pragma unroll
    for (int h = 0; h < kBwdPix; ++h) {
        const int py = py_first + 2 * h;
        float T = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
        int last = 0;
        if (px < C.W && py < C.H) {
            const size_t pix = (size_t)py * C.W + px;
            T = a.tfinal[C.pix_base + pix];
            last = a.ncontrib[C.pix_base + pix];
            g0 = dl[pix];
            g1 = dl[plane + pix];
            g2 = dl[2 * plane + pix];
        }
        // the colour behind the last entry is the background seen through T
        const float nS2 = -(g0 * (T * a.bg[0]) + g1 * (T * a.bg[1]) + g2 * (T * a.bg[2]));
        BwdPair &q = P[h >> 1];
        if (h & 1) {
            q.T.y = T, q.nS2.y = nS2, q.g0.y = g0, q.g1.y = g1, q.g2.y = g2, q.npy.y = -(float)py, q.last1 = last;
        } else {
            q.T.x = T, q.nS2.x = nS2, q.g0.x = g0, q.g1.x = g1, q.g2.x = g2, q.npy.x = -(float)py, q.last0 = last;
        }
        mylast = max(mylast, last);
    }
    if (tid == 0) *S.maxlast = 0;
    __syncthreads();
    if (mylast > 0) atomicMax(S.maxlast, mylast);
    __syncthreads();
    const int maxlast = *S.maxlast;
    const uint32_t rstart = a.ranges[gtile].x;
    const float2 one = f2(1.f, 1.f), two = f2(2.f, 2.f);

    for (int end = maxlast; end > 0; end -= kBwdBatch) {
        const int cnt = min(kBwdBatch, end);
        const int start = end - cnt;
        __syncthreads();
        for (int k = tid; k < cnt; k += kBwdThreads) {
            const uint32_t g = C.rec_base + vals[rstart + start + k];
            S.id[k] = g;
            const float2 m = a.xy[g];
            const float4 co = a.conic_o[g];
            const float4 rgb = a.rgbd[g];
            const float2 sh = a.shape[g];
            const float ca = -0.5f * co.x, cb = -co.y, cc = -0.5f * co.z;
            S.s0[k] = make_float4(m.x, m.x, m.y, m.y);
            S.s1[k] = make_float4(ca, ca, cb, cb);
            S.s2[k] = make_float4(cc, cc, skip_threshold(co.w), sh.y != 0.f ? 1.f : 0.f);
            S.s3[k] = make_float4(rgb.x, rgb.x, rgb.y, rgb.y);
            S.s4[k] = make_float4(rgb.z, rgb.z, co.w, co.w);
            if (sh.y != 0.f) S.s5[k] = make_float4(sh.x, sh.x, sh.y, sh.y);  // read for elongated entries only
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const int p = start + j;
            const float4 X = S.s0[j], Q = S.s1[j], K = S.s2[j];
            const float2 dx = __fadd2_rn(f2(X.x, X.y), npx);
            const float2 cadx = __fmul2_rn(f2(Q.x, Q.y), dx);
            const float2 A = __fmul2_rn(cadx, dx);
            const float2 B = __fmul2_rn(f2(Q.z, Q.w), dx);
            const float2 cc2 = f2(K.x, K.y);
            const bool elong = K.w != 0.f;  // the same for the whole warp
            float2 dy[2], pw[2], cau[2];
            float4 E;
            if (!elong) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    dy[r] = __fadd2_rn(f2(X.z, X.w), P[r].npy);
                    pw[r] = __ffma2_rn(dy[r], __ffma2_rn(cc2, dy[r], B), A);
                }
            } else {
                // the forward's exact power form (the same operations)
                E = S.s5[j];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    dy[r] = __fadd2_rn(f2(X.z, X.w), P[r].npy);
                    const float2 u = __ffma2_rn(f2(E.x, E.y), dy[r], dx);
                    cau[r] = __fmul2_rn(f2(Q.x, Q.y), u);
                    pw[r] = __ffma2_rn(cau[r], u, __fmul2_rn(__fmul2_rn(f2(E.z, E.w), dy[r]), dy[r]));
                }
            }
            bool e[4];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                // the forward's test: power >= skip (a positive power is a
                // rounding of 0, kept)
                e[2 * r] = p < P[r].last0 && pw[r].x >= K.z;
                e[2 * r + 1] = p < P[r].last1 && pw[r].y >= K.z;
            }
            if (!__any_sync(0xffffffffu, e[0] || e[1] || e[2] || e[3])) continue;
            const float4 C1 = S.s3[j], C2 = S.s4[j];
            const float2 o2 = f2(C2.z, C2.w);
            float2 X0, X1, X2, X3, X4, X5, X6, X7, X8;
            bool contrib = false;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                BwdPair &q = P[r];
                const float2 G = f2(__expf(pw[r].x), __expf(pw[r].y));
                const float2 oG = __fmul2_rn(o2, G);
                const float al0 = fminf(kAlphaMax, oG.x), al1 = fminf(kAlphaMax, oG.y);
                const bool c0 = e[2 * r] && al0 >= kAlphaMin, c1 = e[2 * r + 1] && al1 >= kAlphaMin;
                contrib = contrib || c0 || c1;
                const float2 na = f2(c0 ? -al0 : 0.f, c1 ? -al1 : 0.f);
                const float2 om = __fadd2_rn(one, na);  // 1 - alpha (1 where not composited)
                const float2 inv = f2(c0 ? __fdividef(1.f, om.x) : 1.f, c1 ? __fdividef(1.f, om.y) : 1.f);
                q.T = __fmul2_rn(q.T, inv);
                const float2 nw = __fmul2_rn(na, q.T);  // -alpha T
                const float2 S1 = __ffma2_rn(q.g0, f2(C1.x, C1.y),
                                             __ffma2_rn(q.g1, f2(C1.z, C1.w), __fmul2_rn(q.g2, f2(C2.x, C2.y))));
                const float2 dal = __ffma2_rn(inv, q.nS2, __fmul2_rn(q.T, S1));
                q.nS2 = __ffma2_rn(nw, S1, q.nS2);
                // derivative through o G where the cap does not bind
                const float2 Gm = f2(c0 && oG.x < kAlphaMax ? G.x : 0.f, c1 && oG.y < kAlphaMax ? G.y : 0.f);
                const float2 dp = __fmul2_rn(dal, __fmul2_rn(o2, Gm));
                // dpower/dmu: (2 ca dx + cb dy, cb dx + 2 cc dy), or in the
                // exact form (2 ca u, 2 ca u rr + 2 ce dy), which does not cancel
                float2 vx, vy;
                if (!elong) {
                    vx = __ffma2_rn(f2(Q.z, Q.w), dy[r], __fmul2_rn(two, cadx));
                    vy = __ffma2_rn(two, __fmul2_rn(cc2, dy[r]), B);
                } else {
                    vx = __fmul2_rn(two, cau[r]);
                    vy = __ffma2_rn(__fmul2_rn(two, cau[r]), f2(E.x, E.y), __fmul2_rn(two, __fmul2_rn(f2(E.z, E.w), dy[r])));
                }
                const float2 dpvx = __fmul2_rn(dp, vx), dpvy = __fmul2_rn(dp, vy);
                if (r == 0) {
                    X0 = dpvx;
                    X1 = dpvy;
                    X2 = __fmul2_rn(dpvx, vx);
                    X3 = __fmul2_rn(dpvx, vy);
                    X4 = __fmul2_rn(dpvy, vy);
                    X5 = __fmul2_rn(Gm, dal);
                    X6 = __fmul2_rn(nw, q.g0);
                    X7 = __fmul2_rn(nw, q.g1);
                    X8 = __fmul2_rn(nw, q.g2);
                } else {
                    X0 = __fadd2_rn(X0, dpvx);
                    X1 = __fadd2_rn(X1, dpvy);
                    X2 = __ffma2_rn(dpvx, vx, X2);
                    X3 = __ffma2_rn(dpvx, vy, X3);
                    X4 = __ffma2_rn(dpvy, vy, X4);
                    X5 = __ffma2_rn(Gm, dal, X5);
                    X6 = __ffma2_rn(nw, q.g0, X6);
                    X7 = __ffma2_rn(nw, q.g1, X7);
                    X8 = __ffma2_rn(nw, q.g2, X8);
                }
            }
            if (__ballot_sync(0xffffffffu, contrib)) {
                const float gv[9] = {X0.x + X0.y, X1.x + X1.y, 0.5f * (X2.x + X2.y), X3.x + X3.y,
                                     0.5f * (X4.x + X4.y), X5.x + X5.y, -(X6.x + X6.y), -(X7.x + X7.y),
                                     -(X8.x + X8.y)};
                warp_reduce9_add(gv, a.g_screen + (size_t)S.id[j] * 9, lane);
            }
        }
    }
}

// One block per tile; with an order, the heaviest tiles first (as the forward).
__global__ void __launch_bounds__(kBwdThreads) render_bwd_kernel(BwdArgs a) {
    __shared__ uint32_t s_id[kBwdBatch];
    __shared__ float4 s_st[6][kBwdBatch];
    __shared__ int s_maxlast;
    const BwdStage S{s_id, s_st[0], s_st[1], s_st[2], s_st[3], s_st[4], s_st[5], &s_maxlast};
    const uint32_t t = a.order.cnt ? order_pick(a.order, a.ts.total_tiles, blockIdx.x) : (uint32_t)blockIdx.x;
    render_bwd_tile(a, t, a.ts.cam[0], S);
}

__global__ void __launch_bounds__(kBwdThreads) render_bwd_persistent_kernel(BwdArgs a) {
    __shared__ uint32_t s_id[kBwdBatch];
    __shared__ float4 s_st[6][kBwdBatch];
    __shared__ int s_maxlast;
    __shared__ uint32_t s_next;
    const BwdStage S{s_id, s_st[0], s_st[1], s_st[2], s_st[3], s_st[4], s_st[5], &s_maxlast};
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
                render_bwd_tile(a, t, C, S);
            } else {
                render_bwd_tile(a, t, a.ts.cam[camera_of(a.ts, t)], S);
            }
        }
    }
}

cudaError_t launch_render_bwd(const BwdArgs &a, cudaStream_t s) {
    if (a.ts.total_tiles == 0) return cudaSuccess;
    if (a.queue) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_bwd_persistent_kernel, kBwdThreads, 0);
        if (a.blocks_per_sm > 0 && a.blocks_per_sm < per_sm) per_sm = a.blocks_per_sm;
        note_launch("render_bwd_persistent_kernel", s), render_bwd_persistent_kernel<<<sms * (per_sm > 0 ? per_sm : 1), kBwdThreads, 0, s>>>(a);
    } else {
        note_launch("render_bwd_kernel", s), render_bwd_kernel<<<a.ts.total_tiles, kBwdThreads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// SH rows of 3 K floats, as float4 when K is even and the row pointer 16-byte
// aligned (all rows then are).
template <int K>
__device__ __forceinline__ void load_row(const float *p, bool vec, float (&out)[K * 3]) {
    if constexpr ((K * 3) % 4 == 0) {
        if (vec) {
#pragma unroll
            for (int q = 0; q < (K * 3) / 4; ++q) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(p) + q);
                out[4 * q] = v.x;
                out[4 * q + 1] = v.y;
                out[4 * q + 2] = v.z;
                out[4 * q + 3] = v.w;
            }
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < K * 3; ++k) out[k] = __ldg(p + k);
}

// grad += Y[k] * gcol[c] at row position 3 k + c.
template <int K>
__device__ __forceinline__ void add_row(float *p, bool vec, const float (&Y)[16], const float (&gcol)[3]) {
    if constexpr ((K * 3) % 4 == 0) {
        if (vec) {
#pragma unroll
            for (int q = 0; q < (K * 3) / 4; ++q) {
                float4 v = reinterpret_cast<float4 *>(p)[q];
                v.x += Y[(4 * q) / 3] * gcol[(4 * q) % 3];
                v.y += Y[(4 * q + 1) / 3] * gcol[(4 * q + 1) % 3];
                v.z += Y[(4 * q + 2) / 3] * gcol[(4 * q + 2) % 3];
                v.w += Y[(4 * q + 3) / 3] * gcol[(4 * q + 3) % 3];
                reinterpret_cast<float4 *>(p)[q] = v;
            }
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < K * 3; ++k) p[k] += Y[k / 3] * gcol[k % 3];
}

// SINGLE: one camera (a frame); the SH gradient Y gcol^T is then written
// directly instead of being summed over cameras in registers.
template <int DEG, bool SINGLE>
__global__ void __launch_bounds__(256) preprocess_bwd_kernel(PreBwdArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int KS = SINGLE ? 1 : K;  // sizes of the multi-camera accumulator
    const float m0 = a.means[3 * i], m1 = a.means[3 * i + 1], m2 = a.means[3 * i + 2];
    const float sc0 = a.scales[3 * i], sc1 = a.scales[3 * i + 1], sc2 = a.scales[3 * i + 2];
    const float qw = a.quats[4 * i], qx = a.quats[4 * i + 1], qy = a.quats[4 * i + 2], qz = a.quats[4 * i + 3];
    const float *sh = a.sh + (size_t)i * K * 3;
    const bool vec = a.sh_vec4;
    float gmean[3] = {0.f, 0.f, 0.f}, gsc[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, gop = 0.f;
    float gsh[KS * 3];
#pragma unroll
    for (int k = 0; k < KS * 3; ++k) gsh[k] = 0.f;
    float Y1[16], gcol1[3] = {0.f, 0.f, 0.f};  // SINGLE: the one camera's basis and colour gradient
    bool any = false;
    for (int cam = 0; cam < (SINGLE ? 1 : a.cams.n_cams); ++cam) {
        const size_t rec = (size_t)cam * a.n + i;
        const int meta = a.meta[rec];
        if (!(meta & kMetaVisible)) continue;
        const CamDev &cd = a.cams.cam[cam];
        Proj p;
        if (!project_gaussian(cd, m0, m1, m2, sc0, sc1, sc2, qw, qx, qy, qz, a.raw, p)) continue;
        any = true;
        const double *gsd = a.g_screen + rec * 9;
        const float gmx = (float)gsd[0], gmy = (float)gsd[1];
        gop += (float)gsd[5];
        const float grgb[3] = {(float)gsd[6], (float)gsd[7], (float)gsd[8]};
        // gradient w.r.t. Sigma2D = [s11 s12; s12 s22] (s12 one parameter) as the
        // full-matrix gradient H with dL = tr(H^T dSigma)
        const float H00 = (float)gsd[2], H01 = 0.5f * (float)gsd[3], H11 = (float)gsd[4];
        // Sigma2D = A A^T + 0.3 I  ->  dL/dA = 2 H A
        float gA[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            gA[k] = 2.f * (H00 * p.A[k] + H01 * p.A[3 + k]);
            gA[3 + k] = 2.f * (H01 * p.A[k] + H11 * p.A[3 + k]);
        }
        // A = M (R S), M = J W
        const float *V = cd.V;
        float M0[3], M1[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            M0[j] = fmaf(p.J00, V[j], p.J02 * V[8 + j]);
            M1[j] = fmaf(p.J11, V[4 + j], p.J12 * V[8 + j]);
        }
        float gM0[3], gM1[3], gR[9];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            gM0[j] = 0.f;
            gM1[j] = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float rs = p.R[3 * j + k] * p.s[k];
                gM0[j] += gA[k] * rs;
                gM1[j] += gA[3 + k] * rs;
                const float grs = M0[j] * gA[k] + M1[j] * gA[3 + k];
                gR[3 * j + k] = grs * p.s[k];
                gsc[k] += (a.raw ? p.s[k] : 1.f) * grs * p.R[3 * j + k];
            }
        }
        float gJ00 = 0.f, gJ02 = 0.f, gJ11 = 0.f, gJ12 = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            gJ00 += gM0[j] * V[j];
            gJ02 += gM0[j] * V[8 + j];
            gJ11 += gM1[j] * V[4 + j];
            gJ12 += gM1[j] * V[8 + j];
        }
        // J(t) and mu^2D(t) -> t
        const float tz = p.tz, tzi = 1.f / tz, tzi2 = tzi * tzi;
        float gtx = gmx * cd.fx * tzi, gty = gmy * cd.fy * tzi;
        float gtz = -(gmx * cd.fx * p.tx + gmy * cd.fy * p.ty) * tzi2;
        gtz += -(gJ00 * cd.fx + gJ11 * cd.fy) * tzi2;
        if (p.clx) {
            gtz += -gJ02 * p.J02 * tzi;  // J02 = -fx L / tz
        } else {
            gtx += -gJ02 * cd.fx * tzi2;
            gtz += gJ02 * 2.f * cd.fx * p.tx * tzi2 * tzi;
        }
        if (p.cly) {
            gtz += -gJ12 * p.J12 * tzi;
        } else {
            gty += -gJ12 * cd.fy * tzi2;
            gtz += gJ12 * 2.f * cd.fy * p.ty * tzi2 * tzi;
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) gmean[j] += V[j] * gtx + V[4 + j] * gty + V[8 + j] * gtz;

        // rotation of the normalised quaternion -> quaternion
        const float w = p.qn[0], x = p.qn[1], y = p.qn[2], z = p.qn[3];
        const float gw = gR[1] * (-2.f * z) + gR[2] * (2.f * y) + gR[3] * (2.f * z) + gR[5] * (-2.f * x) +
                         gR[6] * (-2.f * y) + gR[7] * (2.f * x);
        const float gx = gR[1] * (2.f * y) + gR[2] * (2.f * z) + gR[3] * (2.f * y) + gR[4] * (-4.f * x) +
                         gR[5] * (-2.f * w) + gR[6] * (2.f * z) + gR[7] * (2.f * w) + gR[8] * (-4.f * x);
        const float gy = gR[0] * (-4.f * y) + gR[1] * (2.f * x) + gR[2] * (2.f * w) + gR[3] * (2.f * x) +
                         gR[5] * (2.f * z) + gR[6] * (-2.f * w) + gR[7] * (2.f * z) + gR[8] * (-4.f * y);
        const float gz = gR[0] * (-4.f * z) + gR[1] * (-2.f * w) + gR[2] * (2.f * x) + gR[3] * (2.f * w) +
                         gR[4] * (-4.f * z) + gR[5] * (2.f * y) + gR[6] * (2.f * x) + gR[7] * (2.f * y);
        const float dot = gw * w + gx * x + gy * y + gz * z;
        const float iq = 1.f / p.qnorm;
        gq[0] += (gw - w * dot) * iq;
        gq[1] += (gx - x * dot) * iq;
        gq[2] += (gy - y * dot) * iq;
        gq[3] += (gz - z * dot) * iq;

        // colour from SH
        const float vx = m0 - cd.campos[0], vy = m1 - cd.campos[1], vz = m2 - cd.campos[2];
        const float vn = sqrtf(vx * vx + vy * vy + vz * vz), ivn = 1.f / vn;
        const float dx = vx * ivn, dy = vy * ivn, dz = vz * ivn;
        float Y[16];
        sh_eval<DEG>(dx, dy, dz, Y);
        float gcol[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) gcol[ch] = (meta >> (kMetaClampShift + ch)) & 1 ? 0.f : grgb[ch];
        if constexpr (SINGLE) {
#pragma unroll
            for (int k = 0; k < 16; ++k) Y1[k] = k < K ? Y[k] : 0.f;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) gcol1[ch] = gcol[ch];
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                gsh[3 * k] += Y[k] * gcol[0];
                gsh[3 * k + 1] += Y[k] * gcol[1];
                gsh[3 * k + 2] += Y[k] * gcol[2];
            }
        }
        if (DEG > 0) {
            float c[K * 3], wsh[16];
            load_row<K>(sh, vec, c);
#pragma unroll
            for (int k = 0; k < K; ++k) wsh[k] = c[3 * k] * gcol[0] + c[3 * k + 1] * gcol[1] + c[3 * k + 2] * gcol[2];
            float ddx, ddy, ddz;
            sh_grad<DEG>(dx, dy, dz, wsh, ddx, ddy, ddz);
            const float r = ddx * dx + ddy * dy + ddz * dz;
            gmean[0] += (ddx - r * dx) * ivn;
            gmean[1] += (ddy - r * dy) * ivn;
            gmean[2] += (ddz - r * dz) * ivn;
        }
    }
    if (!any) return;
    // opacity: o = sigmoid(logit) when raw
    const float ov = a.opac[i];
    const float o = a.raw ? 1.f / (1.f + expf(-ov)) : ov;
    a.go[i] += a.raw ? gop * o * (1.f - o) : gop;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        a.gm[3 * i + j] += gmean[j];
        a.gs[3 * i + j] += gsc[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) a.gq[4 * i + j] += gq[j];
    float *gshp = a.gsh + (size_t)i * K * 3;
    if constexpr (SINGLE) {
        add_row<K>(gshp, a.gsh_vec4, Y1, gcol1);
    } else {
#pragma unroll
        for (int k = 0; k < K * 3; ++k) gshp[k] += gsh[k];
    }
}

cudaError_t launch_preprocess_bwd(const PreBwdArgs &a, int deg, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    dim3 grid((a.n + 255) / 256), block(256);
    const bool one = a.cams.n_cams == 1;
    switch (deg) {
    case 0: one ? (note_launch("preprocess_bwd_kernel", s), preprocess_bwd_kernel<0, true><<<grid, block, 0, s>>>(a))
                : (note_launch("preprocess_bwd_kernel", s), preprocess_bwd_kernel<0, false><<<grid, block, 0, s>>>(a)); break;
    case 1: one ? (note_launch("preprocess_bwd_kernel", s), preprocess_bwd_kernel<1, true><<<grid, block, 0, s>>>(a))
                : (note_launch("preprocess_bwd_kernel", s), preprocess_bwd_kernel<1, false><<<grid, block, 0, s>>>(a)); break;
    case 2: one ? (note_launch("preprocess_bwd_kernel", s), preprocess_bwd_kernel<2, true><<<grid, block, 0, s>>>(a))
                : (note_launch("preprocess_bwd_kernel", s), preprocess_bwd_kernel<2, false><<<grid, block, 0, s>>>(a)); break;
    default: one ? (note_launch("preprocess_bwd_kernel", s), preprocess_bwd_kernel<3, true><<<grid, block, 0, s>>>(a))
                 : (note_launch("preprocess_bwd_kernel", s), preprocess_bwd_kernel<3, false><<<grid, block, 0, s>>>(a)); break;
    }
    return cudaGetLastError();
}

}  // namespace qb
