// qb_binning.cu -- K2 exclusive scan of the per-Gaussian tile counts and K3
// DuplicateWithKeys with QPass traversal (Sec. 2, Sec. 3.2), plus K5, the
// per-tile ranges of the sorted pairs.
#include "qb_kernels.cuh"

namespace qb {

constexpr int kScanBlock = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanBlock * kScanItems;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Inclusive block scan (blockDim.x a multiple of 32, <= 1024); *total gets
// the block sum.
template <typename T>
__device__ __forceinline__ T block_incl_scan(T v, T *total) {
    __shared__ T warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        T s = lane < nw ? warp_sums[lane] : T(0);
        s = warp_incl_scan(s);
        warp_sums[lane] = s;
    }
    __syncthreads();
    T before = wid > 0 ? warp_sums[wid - 1] : T(0);
    *total = warp_sums[nw - 1];
    __syncthreads();
    return incl + before;
}

__global__ void __launch_bounds__(kScanBlock) scan_reduce_kernel(const uint32_t *counts, int n, uint64_t *partials) {
    const size_t base = (size_t)blockIdx.x * kScanChunk;
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        size_t idx = base + (size_t)k * kScanBlock + threadIdx.x;
        if (idx < (size_t)n) s += counts[idx];
    }
    uint64_t total;
    block_incl_scan<uint64_t>(s, &total);
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_partials_kernel(uint64_t *partials, int nb, uint64_t *n_pairs) {
    uint64_t running = 0;
    for (int base = 0; base < nb; base += 1024) {
        int idx = base + threadIdx.x;
        uint64_t v = idx < nb ? partials[idx] : 0;
        uint64_t total;
        uint64_t incl = block_incl_scan<uint64_t>(v, &total);
        if (idx < nb) partials[idx] = running + incl - v;
        running += total;
    }
    if (threadIdx.x == 0) *n_pairs = running;
}

// Each thread scans kScanItems consecutive counts.
__global__ void __launch_bounds__(kScanBlock) scan_down_kernel(const uint32_t *counts, int n, const uint64_t *partials,
                                                               uint32_t *offsets) {
    const size_t base = (size_t)blockIdx.x * kScanChunk + (size_t)threadIdx.x * kScanItems;
    uint32_t c[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        size_t idx = base + k;
        c[k] = idx < (size_t)n ? counts[idx] : 0u;
        s += c[k];
    }
    uint64_t total;
    uint64_t incl = block_incl_scan<uint64_t>(s, &total);
    uint64_t run = partials[blockIdx.x] + incl - s;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        size_t idx = base + k;
        if (idx < (size_t)n) offsets[idx] = (uint32_t)run;  // P <= 2^30 is checked before use
        run += c[k];
    }
}

size_t scan_partials_count(int n) { return (size_t)((n + kScanChunk - 1) / kScanChunk) + 1; }

cudaError_t launch_scan(const uint32_t *counts, int n, uint32_t *offsets, uint64_t *partials, uint64_t *n_pairs,
                        cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(n_pairs, 0, sizeof(uint64_t), s);
    int nb = (n + kScanChunk - 1) / kScanChunk;
    scan_reduce_kernel<<<nb, kScanBlock, 0, s>>>(counts, n, partials);
    scan_partials_kernel<<<1, 1024, 0, s>>>(partials, nb, n_pairs);
    scan_down_kernel<<<nb, kScanBlock, 0, s>>>(counts, n, partials, offsets);
    return cudaGetLastError();
}

// K3: one thread per Gaussian writes its pairs at its scan offset, so the pair
// list is in Gaussian order and a stable sort breaks depth ties by index.
__global__ void __launch_bounds__(256) emit_kernel(EmitArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const uint64_t P = *a.n_pairs;
    if (P > a.capacity) {
        if (i == 0) atomicOr(a.err, kErrCapacity);
        return;
    }
    const uint32_t c = a.counts[i];
    if (c == 0u) return;
    const uint32_t off = a.offsets[i];
    const float2 xy = a.xy[i];
    const int meta = a.meta[i];
    const uint64_t dbits = (uint64_t)(__float_as_uint(a.rgbd[i].w) & 0x7fffffffu);
    Rect r[4];
    box_rects(xy.x, xy.y, a.box[i], a.r3[i], (meta & kMetaOrient) != 0, a.mode, a.clamp3s, a.W, a.H, r);
    uint64_t *keys = a.keys + off;
    uint32_t *vals = a.vals + off;
    uint32_t k = 0;
    const uint32_t tx_n = (uint32_t)a.tiles_x;
    if (a.mode == QB_BIN_AABB3S || a.mode == QB_BIN_ADR) {
        for (int ty = r[0].y0; ty <= r[0].y1; ++ty)
            for (int tx = r[0].x0; tx <= r[0].x1 && k < c; ++tx, ++k) {
                keys[k] = ((uint64_t)((uint32_t)ty * tx_n + (uint32_t)tx) << kDepthBits) | dbits;
                vals[k] = (uint32_t)i;
            }
    } else if (a.mode == QB_BIN_QUADBOX_NAIVE) {
        for (int q = 0; q < 4; ++q) {
            if (rect_empty(r[q])) continue;
            for (int ty = r[q].y0; ty <= r[q].y1; ++ty)
                for (int tx = r[q].x0; tx <= r[q].x1; ++tx) {
                    bool seen = false;
                    for (int p = 0; p < q; ++p) seen |= in_rect(r[p], tx, ty);
                    if (seen || k >= c) continue;
                    keys[k] = ((uint64_t)((uint32_t)ty * tx_n + (uint32_t)tx) << kDepthBits) | dbits;
                    vals[k] = (uint32_t)i;
                    ++k;
                }
        }
    } else {
        QPass qp;
        if (!qpass_setup(r, qp)) return;
        for (int s = qp.s0; s <= qp.s1; ++s) {
            int lo, hi;
            qpass_line(qp, s, lo, hi);
            for (int u = lo; u <= hi && k < c; ++u, ++k) {
                uint32_t tx = qp.columns ? s : u, ty = qp.columns ? u : s;
                keys[k] = ((uint64_t)(ty * tx_n + tx) << kDepthBits) | dbits;
                vals[k] = (uint32_t)i;
            }
        }
    }
}

cudaError_t launch_emit(const EmitArgs &a, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    emit_kernel<<<(a.n + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// K5: tile boundaries of the sorted keys; ranges must be zero on entry.
__global__ void ranges_kernel(const uint64_t *keys, uint64_t n_max, const uint64_t *n_dev, uint2 *ranges,
                              uint32_t ntiles) {
    uint64_t n = n_dev ? min(*n_dev, n_max) : n_max;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t tile = (uint32_t)(keys[idx] >> kDepthBits);
        if (tile >= ntiles) continue;  // never for keys written by the emit kernel
        if (idx == 0 || (uint32_t)(keys[idx - 1] >> kDepthBits) != tile) ranges[tile].x = (uint32_t)idx;
        if (idx == n - 1 || (uint32_t)(keys[idx + 1] >> kDepthBits) != tile) ranges[tile].y = (uint32_t)(idx + 1);
    }
}

cudaError_t launch_ranges(const uint64_t *keys, uint64_t n_max, const uint64_t *n_dev, uint2 *ranges, int ntiles,
                          cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)ntiles, s);
    if (e != cudaSuccess || n_max == 0) return e;
    uint64_t blocks = (n_max + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    ranges_kernel<<<(unsigned)blocks, 256, 0, s>>>(keys, n_max, n_dev, ranges, (uint32_t)ntiles);
    return cudaGetLastError();
}

}  // namespace qb
