// qb_project.cuh -- per-Gaussian EWA projection (Sec. 2) and the opacity-aware
// QuadBox terms (Sec. 3.1), shared by the preprocess kernel and the
// backward's recomputation.
#pragma once

#include "qb_internal.cuh"
#include "qb_sh.cuh"

namespace qb {

struct Proj {
    float tx, ty, tz;      // view-space mean
    float R[9];            // rotation of the normalised quaternion
    float qn[4];           // normalised quaternion (w, x, y, z)
    float qnorm;
    float s[3];            // scales (after exp when raw)
    float A[6];            // A = J W R S  (2 x 3), Sigma2D = A A^T + 0.3 I
    float J00, J02, J11, J12;
    bool clx, cly;         // Jacobian clamp active
    float s11, s12, s22, det;
    float a, b, c, o;      // conic and opacity
    float mx, my;          // mu^2D
};

// Kahan's fused 2x2 determinant p*s - q*r, accurate to about 1.5 ulp.
__device__ __forceinline__ float det2(float p, float q, float r, float s) {
    float w = q * r;
    float e = fmaf(-q, r, w);
    float f = fmaf(p, s, -w);
    return f + e;
}

// Returns false when the Gaussian is culled (behind the near plane, or not
// finite).  Opacity is handled by the caller.
__device__ __forceinline__ bool project_gaussian(const CamDev &cam, float m0, float m1, float m2, float sc0,
                                                 float sc1, float sc2, float qw, float qx, float qy, float qz,
                                                 bool raw, Proj &p) {
    const float *V = cam.V;
    p.tx = fmaf(V[0], m0, fmaf(V[1], m1, fmaf(V[2], m2, V[3])));
    p.ty = fmaf(V[4], m0, fmaf(V[5], m1, fmaf(V[6], m2, V[7])));
    p.tz = fmaf(V[8], m0, fmaf(V[9], m1, fmaf(V[10], m2, V[11])));
    if (!(p.tz > cam.znear)) return false;

    p.s[0] = raw ? expf(sc0) : sc0;
    p.s[1] = raw ? expf(sc1) : sc1;
    p.s[2] = raw ? expf(sc2) : sc2;
    p.qnorm = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    float inv = 1.0f / p.qnorm;
    float w = qw * inv, x = qx * inv, y = qy * inv, z = qz * inv;
    p.qn[0] = w; p.qn[1] = x; p.qn[2] = y; p.qn[3] = z;
    float *R = p.R;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);

    // Jacobian of the perspective map at the mean, with the tangent clamp
    // entering J only (3DGS convention).
    float tzi = 1.0f / p.tz;
    float txtz = p.tx * tzi, tytz = p.ty * tzi;
    float cxtz = fminf(cam.limx, fmaxf(-cam.limx, txtz));
    float cytz = fminf(cam.limy, fmaxf(-cam.limy, tytz));
    p.clx = cxtz != txtz;
    p.cly = cytz != tytz;
    p.J00 = cam.fx * tzi;
    p.J11 = cam.fy * tzi;
    p.J02 = -cam.fx * cxtz * tzi;  // -fx * (clamped tx) / tz^2
    p.J12 = -cam.fy * cytz * tzi;
    // M = J W (2 x 3)
    float M0[3], M1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        M0[j] = fmaf(p.J00, V[j], p.J02 * V[8 + j]);
        M1[j] = fmaf(p.J11, V[4 + j], p.J12 * V[8 + j]);
    }
    // A = M R S; Sigma2D = A A^T + 0.3 I (sums of squares on the diagonal)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float r0 = R[k], r1 = R[3 + k], r2 = R[6 + k];
        p.A[k] = (M0[0] * r0 + M0[1] * r1 + M0[2] * r2) * p.s[k];
        p.A[3 + k] = (M1[0] * r0 + M1[1] * r1 + M1[2] * r2) * p.s[k];
    }
    const float *A = p.A;
    float aa = A[0] * A[0] + A[1] * A[1] + A[2] * A[2];
    float bb = A[3] * A[3] + A[4] * A[4] + A[5] * A[5];
    p.s11 = aa + kDilation;
    p.s22 = bb + kDilation;
    p.s12 = A[0] * A[3] + A[1] * A[4] + A[2] * A[5];
    // det(A A^T + cI) = det(A A^T) + c tr(A A^T) + c^2, with det(A A^T) by
    // Cauchy-Binet as a sum of squared 2x2 minors (no cancellation).
    float m01 = det2(A[0], A[1], A[3], A[4]);
    float m02 = det2(A[0], A[2], A[3], A[5]);
    float m12 = det2(A[1], A[2], A[4], A[5]);
    p.det = (m01 * m01 + m02 * m02 + m12 * m12) + kDilation * (aa + bb) + kDilation * kDilation;
    float idet = 1.0f / p.det;
    p.a = p.s22 * idet;
    p.b = -p.s12 * idet;
    p.c = p.s11 * idet;
    p.mx = fmaf(cam.fx, txtz, cam.cx);
    p.my = fmaf(cam.fy, tytz, cam.cy);
    return isfinite(p.det) && isfinite(p.mx) && isfinite(p.my) && isfinite(p.a) && isfinite(p.c) &&
           isfinite(p.b) && p.det > 0.f;
}

// Box terms from the conic (Sec. 3.1): gamma (Eq. 3 kept side), the AdR
// extents (Eq. extents-inv with Lambda^-1 = Sigma2D), the stretching factor
// (Eq. f-closed, form 1/sqrt(c (Lambda^-1)_22)) and the 3-sigma radius of
// the vanilla box (Sec. 2).  The box threshold adds a margin to gamma that
// covers the renderer's float32 evaluation of the ellipse test.
struct BoxTerms {
    float4 box;  // x_max, y_max, f x_max, f y_max
    float r3;
    bool orient;
};

__device__ __forceinline__ BoxTerms box_terms(const Proj &p) {
    BoxTerms t;
    float gamma = 2.0f * logf(255.0f * p.o);
    float inv_f2 = p.c * p.s22;                 // 1 / f^2
    float f = 1.0f / sqrtf(inv_f2);
    float gamma_b = gamma * (1.0f + 3.814697265625e-06f * inv_f2) + 1e-3f;  // 2^-18
    float xmax = sqrtf(gamma_b * p.s11);
    float ymax = sqrtf(gamma_b * p.s22);
    t.box = make_float4(xmax, ymax, __fmul_rn(f, xmax), __fmul_rn(f, ymax));
    float half = 0.5f * (p.s11 - p.s22);
    float lmax = 0.5f * (p.s11 + p.s22) + sqrtf(fmaxf(0.1f, half * half + p.s12 * p.s12));
    t.r3 = ceilf(3.0f * sqrtf(lmax));
    t.orient = p.s12 >= 0.f;
    return t;
}

}  // namespace qb
