// qb_preprocess.cu -- K1: Gaussian-parallel preprocess (Sec. 2 "Preprocess",
// Sec. 3.1 QuadBox construction, Sec. 3.2 QPass count).
//
// One thread per Gaussian.  Reads the raw parameters (44 B + 12 (deg+1)^2 B),
// writes mu^2D, conic+opacity, colour+depth, the box record, the 3-sigma
// radius, a meta word and the tile count (68 B).  Culled Gaussians write only
// their count and meta word and skip the SH read.
#include "qb_kernels.cuh"
#include "qb_project.cuh"

namespace qb {

template <int DEG>
__global__ void __launch_bounds__(256, 3) preprocess_kernel(PreArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int ci = blockIdx.y;  // camera of this grid row
    const CamDev &cam = a.cams.cam[ci];
    const size_t o = (size_t)ci * a.n + i;  // output record
    const float m0 = a.means[3 * i], m1 = a.means[3 * i + 1], m2 = a.means[3 * i + 2];
    Proj p;
    float4 q4;
    if (a.quat_vec4) {
        q4 = __ldg(reinterpret_cast<const float4 *>(a.quats) + i);
    } else {
        q4 = make_float4(a.quats[4 * i], a.quats[4 * i + 1], a.quats[4 * i + 2], a.quats[4 * i + 3]);
    }
    bool ok = project_gaussian(cam, m0, m1, m2, a.scales[3 * i], a.scales[3 * i + 1], a.scales[3 * i + 2], q4.x,
                               q4.y, q4.z, q4.w, a.raw, p);
    if (ok) {
        float ov = a.opac[i];
        p.o = a.raw ? 1.0f / (1.0f + expf(-ov)) : ov;
        ok = p.o >= kAlphaMin;  // no pixel of this Gaussian reaches alpha_min
    }
    if (!ok) {
        a.counts[o] = 0u;
        a.meta[o] = 0;
        a.shape[o] = make_float2(0.f, 0.f);
        if (a.depth_keys) {  // no tiles: sorts after every Gaussian that has some
            a.depth_keys[o] = 0x7fffffffu;
            a.depth_vals[o] = (uint32_t)o;
        }
        return;
    }
    BoxTerms bt = box_terms(p);

    // view-dependent colour
    constexpr int K = (DEG + 1) * (DEG + 1);
    float dx = m0 - cam.campos[0], dy = m1 - cam.campos[1], dz = m2 - cam.campos[2];
    float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
    float Y[16];
    sh_eval<DEG>(dx * inv, dy * inv, dz * inv, Y);
    const float *sh = a.sh + (size_t)i * (K * 3);
    float rgb[3] = {0.5f, 0.5f, 0.5f};
    if ((K * 3) % 4 == 0 && a.sh_vec4) {
        // 16-byte loads of the coefficient row (3K floats, K even)
        float c[K * 3];
        const float4 *sh4 = reinterpret_cast<const float4 *>(sh);
#pragma unroll
        for (int q = 0; q < (K * 3) / 4; ++q) {
            const float4 v = __ldg(sh4 + q);
            c[4 * q] = v.x;
            c[4 * q + 1] = v.y;
            c[4 * q + 2] = v.z;
            c[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            rgb[0] = fmaf(Y[k], c[3 * k], rgb[0]);
            rgb[1] = fmaf(Y[k], c[3 * k + 1], rgb[1]);
            rgb[2] = fmaf(Y[k], c[3 * k + 2], rgb[2]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            rgb[0] = fmaf(Y[k], __ldg(sh + 3 * k), rgb[0]);
            rgb[1] = fmaf(Y[k], __ldg(sh + 3 * k + 1), rgb[1]);
            rgb[2] = fmaf(Y[k], __ldg(sh + 3 * k + 2), rgb[2]);
        }
    }
    int meta = kMetaVisible | (bt.orient ? kMetaOrient : 0);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        if (rgb[ch] < 0.f) {
            meta |= 1 << (kMetaClampShift + ch);
            rgb[ch] = 0.f;
        }
    }

    Rect rects[4];
    box_rects(p.mx, p.my, bt.box, bt.r3, bt.orient, a.mode, a.clamp3s, cam.W, cam.H, rects);
    uint32_t cnt = 0;
    QPass qp;
    if (qpass_setup(rects, qp)) {
        QSeg seg[7];
        const int ns = qpass_segments(qp, seg);
        // QPass count: the lines of each run of equal intervals times its length
#pragma unroll
        for (int q = 0; q < 7; ++q) cnt += (uint32_t)(seg[q].nl * seg[q].len);
        if (a.segs && cnt > 0u) {
            // the segments, for the emit (which then skips the box and QPass setup)
            uint32_t w[16];
            int ylo = 1 << 14, yhi = -1;  // tile rows the segments cover
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                if (seg_empty(seg[q])) continue;
                const int a0 = qp.columns ? seg[q].lo : seg[q].s0;
                const int a1 = a0 + (qp.columns ? seg[q].len : seg[q].nl) - 1;
                ylo = min(ylo, a0);
                yhi = max(yhi, a1);
            }
            w[0] = (uint32_t)ns | ((uint32_t)qp.columns << 3) | ((uint32_t)ylo << 4) | ((uint32_t)yhi << 18);
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                w[1 + 2 * q] = q < ns ? (uint32_t)seg[q].s0 | ((uint32_t)seg[q].lo << 16) : 0u;
                w[2 + 2 * q] = q < ns ? (uint32_t)seg[q].nl | ((uint32_t)seg[q].len << 16) : 0u;
            }
            w[15] = 0u;
            uint4 *dst = a.segs + 4 * o;
            const int nc = seg_chunks(ns);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c < nc) dst[c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
        }
        const int tiles_x = (cam.W + kTile - 1) >> kTileShift;
        if (a.tile_diff && cnt == 1u) {
            // one tile (the common case): count it directly
            int t = 0;
#pragma unroll
            for (int q = 0; q < 7; ++q)
                if (!seg_empty(seg[q]))
                    t = qp.columns ? seg[q].lo * tiles_x + seg[q].s0 : seg[q].s0 * tiles_x + seg[q].lo;
            atomicAdd(a.tile_single + a.single_off[ci] + t, 1);
        } else if (a.tile_diff) {
            // per-tile pair counts as a 2D difference array: +1/-1 at the corners
            // of every rectangle of the Gaussian's tile set
            const int stride = tiles_x + 1;
            int *D = a.tile_diff + a.diff_off[ci];
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                if (seg_empty(seg[q])) continue;
                const int l0 = seg[q].s0, l1 = seg[q].s0 + seg[q].nl - 1;
                const int u0 = seg[q].lo, u1 = seg[q].lo + seg[q].len - 1;
                const int x0 = qp.columns ? l0 : u0, x1 = qp.columns ? l1 : u1;
                const int y0 = qp.columns ? u0 : l0, y1 = qp.columns ? u1 : l1;
                atomicAdd(D + y0 * stride + x0, 1);
                atomicAdd(D + y0 * stride + x1 + 1, -1);
                atomicAdd(D + (y1 + 1) * stride + x0, -1);
                atomicAdd(D + (y1 + 1) * stride + x1 + 1, 1);
            }
        }
    }
    if (a.mode == QB_BIN_QUADBOX_NAIVE) cnt = naive_count(rects);  // the same set, counted the naive way

    a.xy[o] = make_float2(p.mx, p.my);
    // the exact power form's terms (qb_internal.cuh), for elongated Gaussians only
    float2 shape = make_float2(0.f, 0.f);
    if (p.det < kElongatedF2 * (p.s11 * p.s22)) {
        const float inv22 = 1.0f / p.s22;
        shape = make_float2(-p.s12 * inv22, -0.5f * inv22);
    }
    a.shape[o] = shape;
    a.conic_o[o] = make_float4(p.a, p.b, p.c, p.o);
    a.rgbd[o] = make_float4(rgb[0], rgb[1], rgb[2], p.tz);
    a.box[o] = bt.box;
    a.r3[o] = bt.r3;
    a.meta[o] = meta;
    a.counts[o] = cnt;
    if (a.depth_keys) {
        // the depth-order sort's input: positive float depths order like their
        // bits; Gaussians without tiles sort last
        a.depth_keys[o] = cnt ? (__float_as_uint(p.tz) & 0x7fffffffu) : 0x7fffffffu;
        a.depth_vals[o] = (uint32_t)o;
    }
}

cudaError_t launch_preprocess(const PreArgs &a, int deg, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    dim3 grid((a.n + 255) / 256, a.cams.n_cams), block(256);
    switch (deg) {
    case 0: note_launch("preprocess_kernel", s), preprocess_kernel<0><<<grid, block, 0, s>>>(a); break;
    case 1: note_launch("preprocess_kernel", s), preprocess_kernel<1><<<grid, block, 0, s>>>(a); break;
    case 2: note_launch("preprocess_kernel", s), preprocess_kernel<2><<<grid, block, 0, s>>>(a); break;
    default: note_launch("preprocess_kernel", s), preprocess_kernel<3><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace qb
