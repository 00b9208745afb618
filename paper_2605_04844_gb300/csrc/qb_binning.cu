// qb_binning.cu -- K2 exclusive scan of the per-Gaussian tile counts, K3
// DuplicateWithKeys with QPass traversal (Sec. 2, Sec. 3.2), and K5, the
// per-tile ranges of the sorted pairs.
//
// Pairs are emitted in an "emission order" of the Gaussians: index order for
// the full-key path, depth order for the depth-first path.  The scan runs in
// that order, so each Gaussian's pairs are one contiguous run and a warp's 32
// Gaussians own one contiguous output range.
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

__device__ __forceinline__ uint32_t count_at(const uint32_t *counts, const uint32_t *perm, size_t j) {
    return perm ? counts[perm[j]] : counts[j];
}

__global__ void __launch_bounds__(kScanBlock) scan_reduce_kernel(const uint32_t *counts, const uint32_t *perm, int n,
                                                                 uint64_t *partials) {
    const size_t base = (size_t)blockIdx.x * kScanChunk;
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        size_t idx = base + (size_t)k * kScanBlock + threadIdx.x;
        if (idx < (size_t)n) s += count_at(counts, perm, idx);
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

// Each thread scans kScanItems consecutive counts (in emission order).
__global__ void __launch_bounds__(kScanBlock) scan_down_kernel(const uint32_t *counts, const uint32_t *perm, int n,
                                                               const uint64_t *partials, uint32_t *offsets) {
    const size_t base = (size_t)blockIdx.x * kScanChunk + (size_t)threadIdx.x * kScanItems;
    uint32_t c[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        size_t idx = base + k;
        c[k] = idx < (size_t)n ? count_at(counts, perm, idx) : 0u;
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

cudaError_t launch_scan(const uint32_t *counts, const uint32_t *perm, int n, uint32_t *offsets, uint64_t *partials,
                        uint64_t *n_pairs, cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(n_pairs, 0, sizeof(uint64_t), s);
    int nb = (n + kScanChunk - 1) / kScanChunk;
    scan_reduce_kernel<<<nb, kScanBlock, 0, s>>>(counts, perm, n, partials);
    scan_partials_kernel<<<1, 1024, 0, s>>>(partials, nb, n_pairs);
    scan_down_kernel<<<nb, kScanBlock, 0, s>>>(counts, perm, n, partials, offsets);
    return cudaGetLastError();
}

// Depth keys for the depth-first path: the float bits of the view depth of
// every Gaussian that has tiles (positive floats order like their bits);
// Gaussians without tiles sort last.
__global__ void depth_keys_kernel(int n, const float4 *rgbd, const uint32_t *counts, uint32_t *keys, uint32_t *vals) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = counts[i] ? (__float_as_uint(rgbd[i].w) & 0x7fffffffu) : 0x7fffffffu;
    vals[i] = (uint32_t)i;
}

cudaError_t launch_depth_keys(int n, const float4 *rgbd, const uint32_t *counts, uint32_t *keys, uint32_t *vals,
                              cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    depth_keys_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, rgbd, counts, keys, vals);
    return cudaGetLastError();
}

template <typename KeyT>
__device__ __forceinline__ KeyT make_key(uint32_t tile, uint32_t dbits);
template <>
__device__ __forceinline__ uint64_t make_key<uint64_t>(uint32_t tile, uint32_t dbits) {
    return ((uint64_t)tile << kDepthBits) | dbits;
}
template <>
__device__ __forceinline__ uint32_t make_key<uint32_t>(uint32_t tile, uint32_t) {
    return tile;
}

__device__ __forceinline__ uint32_t lanemask_le() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}

constexpr int kEmitWarps = 8;
constexpr int kSegPerWarp = 32 * 7;

// K3 (QPass modes and the single-box modes): each warp takes 32 consecutive
// Gaussians of the emission order, decomposes each one's QPass traversal into
// its segments (runs of scan lines with one merged interval), and then writes
// the warp's whole output range 32 consecutive pairs at a time: lane q of a
// chunk finds the segment holding its position from a ballot of the segment
// starts that fall in the chunk, and derives its tile from the position
// within that segment.  Stores are contiguous across the warp.
template <typename KeyT>
__global__ void __launch_bounds__(kEmitWarps * 32) emit_warp_kernel(EmitArgs a, KeyT *__restrict__ keys) {
    __shared__ uint32_t s_start[kEmitWarps][kSegPerWarp];
    __shared__ uint32_t s_geo[kEmitWarps][kSegPerWarp];
    __shared__ uint32_t s_len[kEmitWarps][kSegPerWarp];
    __shared__ uint32_t s_gid[kEmitWarps][32];
    __shared__ uint32_t s_dbits[kEmitWarps][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t j = ((size_t)blockIdx.x * kEmitWarps + wid) * 32 + lane;
    if (*a.n_pairs > a.capacity) {
        if (j == 0) atomicOr(a.err, kErrCapacity);
        return;
    }
    uint32_t gid = 0, cnt = 0, off = 0;
    if (j < (size_t)a.n) {
        gid = a.perm ? a.perm[j] : (uint32_t)j;
        cnt = a.counts[gid];
        off = a.offsets[j];
    }
    const uint32_t base = __shfl_sync(0xffffffffu, off, 0);
    const uint32_t total = __reduce_add_sync(0xffffffffu, cnt);
    if (total == 0u) return;

    QSeg seg[7];
    int ns = 0;
    bool columns = false;
    uint32_t dbits = 0;
    if (cnt > 0u) {
        const float2 xy = a.xy[gid];
        const int meta = a.meta[gid];
        dbits = __float_as_uint(a.rgbd[gid].w) & 0x7fffffffu;
        Rect r[4];
        box_rects(xy.x, xy.y, a.box[gid], a.r3[gid], (meta & kMetaOrient) != 0, a.mode, a.clamp3s, a.W, a.H, r);
        QPass qp;
        if (qpass_setup(r, qp)) {
            ns = qpass_segments(qp, seg);
            columns = qp.columns;
        }
    }
    s_gid[wid][lane] = gid;
    s_dbits[wid][lane] = dbits;
    const int sincl = warp_incl_scan(ns);
    const int sbase = sincl - ns;
    const int nseg = __shfl_sync(0xffffffffu, sincl, 31);
    uint32_t rel = off - base;
    for (int q = 0; q < ns; ++q) {
        s_start[wid][sbase + q] = rel;
        s_geo[wid][sbase + q] = (uint32_t)seg[q].s0 | ((uint32_t)seg[q].lo << 16);
        s_len[wid][sbase + q] = (uint32_t)seg[q].len | ((uint32_t)lane << 16) | ((uint32_t)columns << 24);
        rel += (uint32_t)(seg[q].nl * seg[q].len);
    }
    __syncwarp();

    const uint32_t le = lanemask_le();
    const uint32_t tx_n = (uint32_t)a.tiles_x;
    int cur = -1;  // last segment starting before the current chunk
    for (uint32_t c0 = 0; c0 < total; c0 += 32) {
        const int cand = cur + 1 + lane;
        uint32_t bit = 0u;
        if (cand < nseg) {
            const uint32_t st = s_start[wid][cand];
            if (st < c0 + 32u) bit = 1u << (st - c0);
        }
        const uint32_t M = __reduce_or_sync(0xffffffffu, bit);
        const uint32_t p = c0 + lane;
        if (p < total) {
            const int idx = cur + __popc(M & le);
            const uint32_t st = s_start[wid][idx], geo = s_geo[wid][idx], ln = s_len[wid][idx];
            const uint32_t k = p - st, len = ln & 0xffffu;
            const uint32_t line = (geo & 0xffffu) + k / len;
            const uint32_t u = (geo >> 16) + k % len;
            const bool cols = (ln >> 24) & 1u;
            const uint32_t owner = (ln >> 16) & 0xffu;
            const uint32_t tile = (cols ? u : line) * tx_n + (cols ? line : u);
            keys[base + p] = make_key<KeyT>(tile, s_dbits[wid][owner]);
            a.vals[base + p] = s_gid[wid][owner];
        }
        cur += __popc(M);
    }
}

// K3 for QuadBox-dagger (QB_BIN_QUADBOX_NAIVE, the paper's ablation without
// QPass): one thread per Gaussian runs nested loops over each sub-box and
// skips tiles an earlier sub-box already holds.
template <typename KeyT>
__global__ void __launch_bounds__(256) emit_naive_kernel(EmitArgs a, KeyT *__restrict__ keys) {
    const size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (size_t)a.n) return;
    if (*a.n_pairs > a.capacity) {
        if (j == 0) atomicOr(a.err, kErrCapacity);
        return;
    }
    const uint32_t gid = a.perm ? a.perm[j] : (uint32_t)j;
    const uint32_t c = a.counts[gid];
    if (c == 0u) return;
    const uint32_t off = a.offsets[j];
    const float2 xy = a.xy[gid];
    const int meta = a.meta[gid];
    const uint32_t dbits = __float_as_uint(a.rgbd[gid].w) & 0x7fffffffu;
    Rect r[4];
    box_rects(xy.x, xy.y, a.box[gid], a.r3[gid], (meta & kMetaOrient) != 0, a.mode, a.clamp3s, a.W, a.H, r);
    uint32_t k = 0;
    const uint32_t tx_n = (uint32_t)a.tiles_x;
    for (int q = 0; q < 4; ++q) {
        if (rect_empty(r[q])) continue;
        for (int ty = r[q].y0; ty <= r[q].y1; ++ty)
            for (int tx = r[q].x0; tx <= r[q].x1; ++tx) {
                bool seen = false;
                for (int p = 0; p < q; ++p) seen |= in_rect(r[p], tx, ty);
                if (seen || k >= c) continue;
                keys[off + k] = make_key<KeyT>((uint32_t)ty * tx_n + (uint32_t)tx, dbits);
                a.vals[off + k] = gid;
                ++k;
            }
    }
}

template <typename KeyT>
cudaError_t launch_emit(const EmitArgs &a, KeyT *keys, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (a.mode == QB_BIN_QUADBOX_NAIVE) {
        emit_naive_kernel<KeyT><<<(a.n + 255) / 256, 256, 0, s>>>(a, keys);
    } else {
        const int per_block = kEmitWarps * 32;
        emit_warp_kernel<KeyT><<<(a.n + per_block - 1) / per_block, per_block, 0, s>>>(a, keys);
    }
    return cudaGetLastError();
}

template cudaError_t launch_emit<uint64_t>(const EmitArgs &, uint64_t *, cudaStream_t);
template cudaError_t launch_emit<uint32_t>(const EmitArgs &, uint32_t *, cudaStream_t);

// K5: tile boundaries of the sorted keys; ranges must be zero on entry.
template <typename KeyT>
__device__ __forceinline__ uint32_t tile_of(KeyT k) {
    return sizeof(KeyT) == 8 ? (uint32_t)((uint64_t)k >> kDepthBits) : (uint32_t)k;
}

template <typename KeyT>
__global__ void ranges_kernel(const KeyT *keys, uint64_t n_max, const uint64_t *n_dev, uint2 *ranges,
                              uint32_t ntiles) {
    uint64_t n = n_dev ? min(*n_dev, n_max) : n_max;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t tile = tile_of(keys[idx]);
        if (tile >= ntiles) continue;  // never for keys written by the emit kernels
        if (idx == 0 || tile_of(keys[idx - 1]) != tile) ranges[tile].x = (uint32_t)idx;
        if (idx == n - 1 || tile_of(keys[idx + 1]) != tile) ranges[tile].y = (uint32_t)(idx + 1);
    }
}

template <typename KeyT>
cudaError_t launch_ranges(const KeyT *keys, uint64_t n_max, const uint64_t *n_dev, uint2 *ranges, int ntiles,
                          cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)ntiles, s);
    if (e != cudaSuccess || n_max == 0) return e;
    uint64_t blocks = (n_max + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    ranges_kernel<KeyT><<<(unsigned)blocks, 256, 0, s>>>(keys, n_max, n_dev, ranges, (uint32_t)ntiles);
    return cudaGetLastError();
}

template cudaError_t launch_ranges<uint64_t>(const uint64_t *, uint64_t, const uint64_t *, uint2 *, int, cudaStream_t);
template cudaError_t launch_ranges<uint32_t>(const uint32_t *, uint64_t, const uint64_t *, uint2 *, int, cudaStream_t);

}  // namespace qb
