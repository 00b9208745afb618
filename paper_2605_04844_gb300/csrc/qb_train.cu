// qb_train.cu -- one optimisation step around the differentiable rasteriser:
// the L1 image loss and its gradient, and a fused Adam update of the raw
// scene parameters (Kingma & Ba's bias-corrected rule).  Both are plain
// elementwise HBM-bound kernels; the loss is summed per block in FP64.
#include "qb_kernels.cuh"

namespace qb {

// dL[i] = sign(img[i] - target[i]) * scale (0 where equal); *loss += scale *
// sum |img - target| when loss is non-null.
__global__ void __launch_bounds__(256) l1_grad_kernel(const float *__restrict__ img, const float *__restrict__ target,
                                                      float *__restrict__ dL, uint64_t n, float scale, double *loss) {
    double acc = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float d = img[i] - target[i];
        dL[i] = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
        acc += fabs((double)d);
    }
    if (!loss) return;
    __shared__ double s[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        atomicAdd(loss, t * (double)scale);
    }
}

// Adam, step t (1-based): m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
// p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
__global__ void __launch_bounds__(256) adam_kernel(float *__restrict__ p, const float *__restrict__ g,
                                                   float *__restrict__ m, float *__restrict__ v, uint64_t n, float lr,
                                                   float b1, float b2, float eps, float c1, float c2) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

static unsigned grid_for(uint64_t n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (n + 255) / 256, cap = (uint64_t)(sms > 0 ? sms : 1) * 8;
    return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

cudaError_t launch_l1_grad(const float *img, const float *target, float *dL, uint64_t n, float scale, double *loss,
                           cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launch("l1_grad_kernel", s), l1_grad_kernel<<<grid_for(n), 256, 0, s>>>(img, target, dL, n, scale, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, uint64_t n, float lr, float b1, float b2,
                        float eps, int t, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    note_launch("adam_kernel", s), adam_kernel<<<grid_for(n), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace qb
