// qb_backward.cu -- K7 render backward and K8 preprocess backward of the
// differentiable rasteriser (Sec. 4.1 states the rasteriser is differentiable;
// the gradients below differentiate Eq. 2 and the Sec. 2 projection).
//
// K7: one 256-thread block per tile walks the tile list in reverse, from the
// largest last-contributor position of its pixels down to 0.  Each pixel
// recomputes alpha exactly as the forward did and the transmittance by
// division, T_k = T_{k+1} / (1 - alpha_k), keeping the colour behind the
// current entry, B_k = sum_{i>k} T_i alpha_i c_i + T_final bg:
//   dC/dc_k     = T_k alpha_k
//   dC/dalpha_k = T_k c_k - B_k / (1 - alpha_k)
// alpha = min(0.99, o G), G = exp(power): zero derivative where the cap binds.
// Per Gaussian the 32 lanes of a warp are summed with shuffles and one lane
// adds the 9 screen-space gradients atomically in float64: (mu_x, mu_y,
// Sigma11, Sigma12, Sigma22, o, r, g, b), the covariance entries being the
// well-conditioned parametrisation (dL/dLambda = -Sigma dL/dSigma Sigma).
//
// K8: one thread per Gaussian chains the (mu^2D, Sigma2D, o, colour) gradients
// to means, (log-)scales, quaternions, opacity (logits) and SH.
#include "qb_kernels.cuh"
#include "qb_project.cuh"

namespace qb {

constexpr int kBwdThreads = kTile * kTile;

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

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kBwdThreads) render_bwd_kernel(BwdArgs a) {
    __shared__ uint32_t s_id[kBwdThreads];
    __shared__ float4 s_xy[kBwdThreads];  // mu_x, mu_y, skip threshold
    __shared__ float4 s_co[kBwdThreads];
    __shared__ float4 s_rgb[kBwdThreads];
    __shared__ int s_maxlast;

    const int tile = blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int tid = threadIdx.x, lane = tid & 31;
    const int px = tx * kTile + (tid & (kTile - 1));
    const int py = ty * kTile + (tid >> kTileShift);
    const bool inside = px < a.W && py < a.H;
    const float pxf = (float)px, pyf = (float)py;
    const size_t pix = (size_t)py * a.W + px, plane = (size_t)a.W * a.H;

    float T = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    int last = 0;
    if (inside) {
        T = a.tfinal[pix];
        last = a.ncontrib[pix];
        g0 = a.dL_dimg[pix];
        g1 = a.dL_dimg[plane + pix];
        g2 = a.dL_dimg[2 * plane + pix];
    }
    float B0 = T * a.bg[0], B1 = T * a.bg[1], B2 = T * a.bg[2];
    if (tid == 0) s_maxlast = 0;
    __syncthreads();
    if (last > 0) atomicMax(&s_maxlast, last);
    __syncthreads();
    const int maxlast = s_maxlast;
    const uint32_t rstart = a.ranges[tile].x;

    for (int end = maxlast; end > 0; end -= kBwdThreads) {
        const int cnt = min(kBwdThreads, end);
        const int start = end - cnt;
        __syncthreads();
        if (tid < cnt) {
            const uint32_t g = a.vals[rstart + start + tid];
            s_id[tid] = g;
            const float2 m = a.xy[g];
            const float4 co = a.conic_o[g];
            s_xy[tid] = make_float4(m.x, m.y, skip_threshold(co.w), 0.f);
            s_co[tid] = co;
            s_rgb[tid] = a.rgbd[g];
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const int p = start + j;
            float gv[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool contrib = false;
            if (p < last) {
                const float4 m = s_xy[j];
                const float4 co = s_co[j];
                const float dx = m.x - pxf, dy = m.y - pyf;
                const float power = eval_power(co, dx, dy);
                if (power <= 0.f && power >= m.z) {
                    const float G = __expf(power);
                    const float oG = __fmul_rn(co.w, G);
                    const float alpha = fminf(kAlphaMax, oG);
                    if (alpha >= kAlphaMin) {
                        contrib = true;
                        const float om = 1.f - alpha;
                        T = T / om;  // transmittance in front of this entry
                        const float4 c = s_rgb[j];
                        const float w = alpha * T;
                        gv[6] = w * g0;
                        gv[7] = w * g1;
                        gv[8] = w * g2;
                        const float inv = 1.f / om;
                        const float dalpha = g0 * (T * c.x - B0 * inv) + g1 * (T * c.y - B1 * inv) +
                                             g2 * (T * c.z - B2 * inv);
                        B0 = fmaf(w, c.x, B0);
                        B1 = fmaf(w, c.y, B1);
                        B2 = fmaf(w, c.z, B2);
                        if (oG < kAlphaMax) {
                            // power = -d^T Lambda d / 2 with Lambda = Sigma^-1 and u = Lambda d:
                            // dpower/dmu = -u, dpower/dSigma = u u^T / 2
                            const float dpower = dalpha * oG;
                            const float ux = co.x * dx + co.y * dy, uy = co.y * dx + co.z * dy;
                            gv[5] = G * dalpha;
                            gv[0] = -dpower * ux;
                            gv[1] = -dpower * uy;
                            gv[2] = 0.5f * dpower * ux * ux;
                            gv[3] = dpower * ux * uy;
                            gv[4] = 0.5f * dpower * uy * uy;
                        }
                    }
                }
            }
            if (__ballot_sync(0xffffffffu, contrib)) {
#pragma unroll
                for (int v = 0; v < 9; ++v) gv[v] = warp_sum(gv[v]);
                if (lane == 0) {
                    // float64 accumulation across warps and tiles: a large Gaussian
                    // sums thousands of terms of both signs
                    double *dst = a.g_screen + (size_t)s_id[j] * 9;
#pragma unroll
                    for (int v = 0; v < 9; ++v)
                        if (gv[v] != 0.f) atomicAdd(dst + v, widen(gv[v]));
                }
            }
        }
    }
}

cudaError_t launch_render_bwd(const BwdArgs &a, cudaStream_t s) {
    const int ntiles = a.tiles_x * a.tiles_y;
    if (ntiles == 0) return cudaSuccess;
    render_bwd_kernel<<<ntiles, kBwdThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <int DEG>
__global__ void __launch_bounds__(256) preprocess_bwd_kernel(PreBwdArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int meta = a.meta[i];
    if (!(meta & kMetaVisible)) return;
    const CamDev &cam = a.cam;
    const float m0 = a.means[3 * i], m1 = a.means[3 * i + 1], m2 = a.means[3 * i + 2];
    Proj p;
    if (!project_gaussian(cam, m0, m1, m2, a.scales[3 * i], a.scales[3 * i + 1], a.scales[3 * i + 2],
                          a.quats[4 * i], a.quats[4 * i + 1], a.quats[4 * i + 2], a.quats[4 * i + 3], a.raw, p))
        return;
    const double *gsc = a.g_screen + (size_t)i * 9;
    const float gmx = (float)gsc[0], gmy = (float)gsc[1], gop = (float)gsc[5];
    const float grgb[3] = {(float)gsc[6], (float)gsc[7], (float)gsc[8]};
    // gradient w.r.t. Sigma2D = [s11 s12; s12 s22] (s12 one parameter) as the
    // full-matrix gradient H with dL = tr(H^T dSigma)
    const float H00 = (float)gsc[2], H01 = 0.5f * (float)gsc[3], H11 = (float)gsc[4];
    // Sigma2D = A A^T + 0.3 I  ->  dL/dA = 2 H A
    float gA[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        gA[k] = 2.f * (H00 * p.A[k] + H01 * p.A[3 + k]);
        gA[3 + k] = 2.f * (H01 * p.A[k] + H11 * p.A[3 + k]);
    }
    // A = M (R S), M = J W
    const float *V = cam.V;
    float M0[3], M1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        M0[j] = fmaf(p.J00, V[j], p.J02 * V[8 + j]);
        M1[j] = fmaf(p.J11, V[4 + j], p.J12 * V[8 + j]);
    }
    float gM0[3], gM1[3], gR[9], gs[3] = {0.f, 0.f, 0.f};
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
            gs[k] += grs * p.R[3 * j + k];
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
    float gtx = gmx * cam.fx * tzi, gty = gmy * cam.fy * tzi;
    float gtz = -(gmx * cam.fx * p.tx + gmy * cam.fy * p.ty) * tzi2;
    gtz += -(gJ00 * cam.fx + gJ11 * cam.fy) * tzi2;
    if (p.clx) {
        gtz += -gJ02 * p.J02 * tzi;  // J02 = -fx L / tz
    } else {
        gtx += -gJ02 * cam.fx * tzi2;
        gtz += gJ02 * 2.f * cam.fx * p.tx * tzi2 * tzi;
    }
    if (p.cly) {
        gtz += -gJ12 * p.J12 * tzi;
    } else {
        gty += -gJ12 * cam.fy * tzi2;
        gtz += gJ12 * 2.f * cam.fy * p.ty * tzi2 * tzi;
    }
    float gmean[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) gmean[j] = V[j] * gtx + V[4 + j] * gty + V[8 + j] * gtz;

    // rotation of the normalised quaternion -> quaternion
    const float w = p.qn[0], x = p.qn[1], y = p.qn[2], z = p.qn[3];
    float gw = gR[1] * (-2.f * z) + gR[2] * (2.f * y) + gR[3] * (2.f * z) + gR[5] * (-2.f * x) +
               gR[6] * (-2.f * y) + gR[7] * (2.f * x);
    float gx = gR[1] * (2.f * y) + gR[2] * (2.f * z) + gR[3] * (2.f * y) + gR[4] * (-4.f * x) +
               gR[5] * (-2.f * w) + gR[6] * (2.f * z) + gR[7] * (2.f * w) + gR[8] * (-4.f * x);
    float gy = gR[0] * (-4.f * y) + gR[1] * (2.f * x) + gR[2] * (2.f * w) + gR[3] * (2.f * x) +
               gR[5] * (2.f * z) + gR[6] * (-2.f * w) + gR[7] * (2.f * z) + gR[8] * (-4.f * y);
    float gz = gR[0] * (-4.f * z) + gR[1] * (-2.f * w) + gR[2] * (2.f * x) + gR[3] * (2.f * w) +
               gR[4] * (-4.f * z) + gR[5] * (2.f * y) + gR[6] * (2.f * x) + gR[7] * (2.f * y);
    const float dot = gw * w + gx * x + gy * y + gz * z;
    const float iq = 1.f / p.qnorm;
    a.gq[4 * i] += (gw - w * dot) * iq;
    a.gq[4 * i + 1] += (gx - x * dot) * iq;
    a.gq[4 * i + 2] += (gy - y * dot) * iq;
    a.gq[4 * i + 3] += (gz - z * dot) * iq;
#pragma unroll
    for (int k = 0; k < 3; ++k) a.gs[3 * i + k] += a.raw ? gs[k] * p.s[k] : gs[k];

    // opacity
    const float ov = a.opac[i];
    const float o = a.raw ? 1.f / (1.f + expf(-ov)) : ov;
    a.go[i] += a.raw ? gop * o * (1.f - o) : gop;

    // colour from SH
    constexpr int K = (DEG + 1) * (DEG + 1);
    const float vx = m0 - cam.campos[0], vy = m1 - cam.campos[1], vz = m2 - cam.campos[2];
    const float vn = sqrtf(vx * vx + vy * vy + vz * vz), ivn = 1.f / vn;
    const float dx = vx * ivn, dy = vy * ivn, dz = vz * ivn;
    float Y[16];
    sh_eval<DEG>(dx, dy, dz, Y);
    float gcol[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) gcol[ch] = (meta >> (kMetaClampShift + ch)) & 1 ? 0.f : grgb[ch];
    const float *sh = a.sh + (size_t)i * K * 3;
    float *gsh = a.gsh + (size_t)i * K * 3;
    float wsh[16];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        gsh[3 * k] += Y[k] * gcol[0];
        gsh[3 * k + 1] += Y[k] * gcol[1];
        gsh[3 * k + 2] += Y[k] * gcol[2];
        wsh[k] = sh[3 * k] * gcol[0] + sh[3 * k + 1] * gcol[1] + sh[3 * k + 2] * gcol[2];
    }
    if (DEG > 0) {
        float ddx, ddy, ddz;
        sh_grad<DEG>(dx, dy, dz, wsh, ddx, ddy, ddz);
        const float r = ddx * dx + ddy * dy + ddz * dz;
        gmean[0] += (ddx - r * dx) * ivn;
        gmean[1] += (ddy - r * dy) * ivn;
        gmean[2] += (ddz - r * dz) * ivn;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) a.gm[3 * i + j] += gmean[j];
}

cudaError_t launch_preprocess_bwd(const PreBwdArgs &a, int deg, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    dim3 grid((a.n + 255) / 256), block(256);
    switch (deg) {
    case 0: preprocess_bwd_kernel<0><<<grid, block, 0, s>>>(a); break;
    case 1: preprocess_bwd_kernel<1><<<grid, block, 0, s>>>(a); break;
    case 2: preprocess_bwd_kernel<2><<<grid, block, 0, s>>>(a); break;
    default: preprocess_bwd_kernel<3><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace qb
