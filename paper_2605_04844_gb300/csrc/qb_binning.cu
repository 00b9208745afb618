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
constexpr uint32_t kEmitChunk = 2048;  // output positions per warp

// K3 (QPass modes and the single-box modes), balanced over the output: warp w
// owns the pair positions [w C, (w+1) C).  It finds the first Gaussian whose
// run reaches into that range (32-ary search over the emission-order
// offsets), then takes the following Gaussians 32 at a time: each lane
// decomposes its Gaussian's QPass traversal into segments (runs of scan lines
// with one merged interval), and the warp writes the range 32 consecutive
// positions at a time; lane q finds the segment holding its position from a
// ballot of the segment starts that fall in its group.  Stores are contiguous
// across the warp, and every warp writes at most C pairs however large the
// Gaussians are.
template <typename KeyT>
__global__ void __launch_bounds__(kEmitWarps * 32) emit_warp_kernel(EmitArgs a, KeyT *__restrict__ keys) {
    __shared__ int32_t s_start[kEmitWarps][kSegPerWarp];
    __shared__ uint32_t s_geo[kEmitWarps][kSegPerWarp];
    __shared__ uint32_t s_len[kEmitWarps][kSegPerWarp];
    __shared__ float s_inv[kEmitWarps][kSegPerWarp];
    __shared__ uint32_t s_gid[kEmitWarps][32];
    __shared__ uint32_t s_dbits[kEmitWarps][32];
    __shared__ uint32_t s_tbase[kEmitWarps][32];  // first global tile of the owner's camera
    __shared__ uint32_t s_tx[kEmitWarps][32];     // tiles per row of the owner's camera
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t P = *a.n_pairs;
    const uint64_t warp_id = (uint64_t)blockIdx.x * kEmitWarps + wid;
    if (P > a.capacity) {
        if (warp_id == 0 && lane == 0) atomicOr(a.err, kErrCapacity);
        return;
    }
    const uint64_t C = warp_id * kEmitChunk;
    if (C >= P || a.n == 0) return;
    const int32_t L = (int32_t)min((uint64_t)kEmitChunk, P - C);

    // last emission position j with offsets[j] <= C (offsets are non-decreasing)
    int64_t lo = 0, hi = a.n - 1;  // invariant: offsets[lo] <= C, answer in [lo, hi]
    while (hi > lo) {
        const int64_t span = hi - lo;
        const int64_t probe = lo + (span * (lane + 1) + 31) / 32;  // 32 probes in (lo, hi]
        const bool le = probe <= hi && (uint64_t)a.offsets[probe] <= C;
        const uint32_t m = __ballot_sync(0xffffffffu, le);
        const int k = m ? 31 - __clz(m) : -1;  // highest probing lane with offsets <= C
        const int64_t new_lo = k >= 0 ? lo + (span * (k + 1) + 31) / 32 : lo;
        const int64_t nk = k + 1;
        const int64_t new_hi = nk < 32 ? lo + (span * (nk + 1) + 31) / 32 - 1 : hi;
        lo = new_lo;
        const int64_t cand_hi = new_hi > new_lo ? new_hi : new_lo;
        hi = cand_hi < hi ? cand_hi : hi;
    }
    int64_t j0 = lo;

    const uint32_t le_mask = lanemask_le();
    int32_t done_to = 0;  // chunk positions [0, done_to) written
    while (done_to < L && j0 < a.n) {
        const int64_t j = j0 + lane;
        uint32_t gid = 0, cnt = 0;
        int64_t rel = (int64_t)1 << 40;
        if (j < a.n) {
            gid = a.perm ? a.perm[j] : (uint32_t)j;
            cnt = a.counts[gid];
            rel = (int64_t)a.offsets[j] - (int64_t)C;
        }
        const bool relevant = cnt > 0u && rel < L && rel + (int64_t)cnt > 0;
        QSeg seg[7];
        int ns = 0;
        bool columns = false;
        uint32_t dbits = 0, tbase = 0, tx_n = 1;
        if (relevant) {
            const CamTile &cam = a.ts.cam[gid / (uint32_t)a.n_per_cam];
            tbase = cam.tile_base;
            tx_n = (uint32_t)cam.tiles_x;
            const float2 xy = a.xy[gid];
            const int meta = a.meta[gid];
            dbits = __float_as_uint(a.rgbd[gid].w) & 0x7fffffffu;
            Rect r[4];
            box_rects(xy.x, xy.y, a.box[gid], a.r3[gid], (meta & kMetaOrient) != 0, a.mode, a.clamp3s, cam.W,
                      cam.H, r);
            QPass qp;
            if (qpass_setup(r, qp)) {
                ns = qpass_segments(qp, seg);
                columns = qp.columns;
            }
        }
        __syncwarp();
        s_gid[wid][lane] = gid;
        s_dbits[wid][lane] = dbits;
        s_tbase[wid][lane] = tbase;
        s_tx[wid][lane] = tx_n;
        const int sincl = warp_incl_scan(ns);
        const int sbase = sincl - ns;
        const int nseg = __shfl_sync(0xffffffffu, sincl, 31);
        int32_t r0 = (int32_t)(rel > -((int64_t)1 << 30) ? rel : -((int64_t)1 << 30));
        for (int q = 0; q < ns; ++q) {
            s_start[wid][sbase + q] = r0;
            s_geo[wid][sbase + q] = (uint32_t)seg[q].s0 | ((uint32_t)seg[q].lo << 16);
            s_len[wid][sbase + q] = (uint32_t)seg[q].len | ((uint32_t)lane << 16) | ((uint32_t)columns << 24);
            s_inv[wid][sbase + q] = 1.0f / (float)seg[q].len;
            r0 += seg[q].nl * seg[q].len;
        }
        // end of this batch's pairs within the chunk
        const int64_t last_end = __shfl_sync(0xffffffffu, rel + (int64_t)cnt, 31);
        const int32_t batch_end = (int32_t)(last_end < (int64_t)L ? last_end : (int64_t)L);
        __syncwarp();
        // cur: last segment starting at or before done_to
        int cur = -1;
        for (int b = 0; b < nseg; b += 32) {
            const bool le = b + lane < nseg && s_start[wid][b + lane] <= done_to;
            cur += __popc(__ballot_sync(0xffffffffu, le));
        }
        for (int32_t c0 = done_to; c0 < batch_end; c0 += 32) {
            const int cand = cur + 1 + lane;
            uint32_t bit = 0u;
            if (cand < nseg) {
                const int32_t st = s_start[wid][cand];
                if (st < c0 + 32) bit = 1u << (st - c0);
            }
            const uint32_t M = __reduce_or_sync(0xffffffffu, bit);
            const int32_t p = c0 + lane;
            if (p < batch_end) {
                const int idx = cur + __popc(M & le_mask);
                const int32_t st = s_start[wid][idx];
                const uint32_t geo = s_geo[wid][idx], ln = s_len[wid][idx];
                const uint32_t k = (uint32_t)(p - st), len = ln & 0xffffu;
                // k / len through the reciprocal (k < 2^24, so the estimate is
                // off by at most one) and one exact correction
                int32_t q = (int32_t)((float)k * s_inv[wid][idx]);
                int32_t r = (int32_t)k - q * (int32_t)len;
                if (r < 0) { --q; r += (int32_t)len; }
                if (r >= (int32_t)len) { ++q; r -= (int32_t)len; }
                const uint32_t line = (geo & 0xffffu) + (uint32_t)q;
                const uint32_t u = (geo >> 16) + (uint32_t)r;
                const bool cols = (ln >> 24) & 1u;
                const uint32_t owner = (ln >> 16) & 0xffu;
                const uint32_t tile = s_tbase[wid][owner] + (cols ? u : line) * s_tx[wid][owner] + (cols ? line : u);
                keys[C + p] = make_key<KeyT>(tile, s_dbits[wid][owner]);
                a.vals[C + p] = s_gid[wid][owner];
            }
            cur += __popc(M);
        }
        done_to = max(done_to, batch_end);
        j0 += 32;
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
    const CamTile &cam = a.ts.cam[gid / (uint32_t)a.n_per_cam];
    Rect r[4];
    box_rects(xy.x, xy.y, a.box[gid], a.r3[gid], (meta & kMetaOrient) != 0, a.mode, a.clamp3s, cam.W, cam.H, r);
    uint32_t k = 0;
    const uint32_t tx_n = (uint32_t)cam.tiles_x;
    for (int q = 0; q < 4; ++q) {
        if (rect_empty(r[q])) continue;
        for (int ty = r[q].y0; ty <= r[q].y1; ++ty)
            for (int tx = r[q].x0; tx <= r[q].x1; ++tx) {
                bool seen = false;
                for (int p = 0; p < q; ++p) seen |= in_rect(r[p], tx, ty);
                if (seen || k >= c) continue;
                keys[off + k] = make_key<KeyT>(cam.tile_base + (uint32_t)ty * tx_n + (uint32_t)tx, dbits);
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
        const uint64_t pairs = a.n_pairs_host != UINT64_MAX ? a.n_pairs_host : a.capacity;
        const uint64_t warps = (pairs + kEmitChunk - 1) / kEmitChunk;
        const uint64_t blocks = (warps + kEmitWarps - 1) / kEmitWarps;
        if (blocks > 0) emit_warp_kernel<KeyT><<<(unsigned)blocks, kEmitWarps * 32, 0, s>>>(a, keys);
        else if (a.n > 0) emit_warp_kernel<KeyT><<<1, kEmitWarps * 32, 0, s>>>(a, keys);  // flags overflow
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
    uint64_t n = n_dev ? (*n_dev > n_max ? 0 : *n_dev) : n_max;  // overflow (flagged by the emit): no pairs
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

// Per-tile pair counts from the difference arrays written by the preprocess:
// for every camera of the set a 2D prefix sum plus the single-tile counts
// gives each tile's count; an exclusive scan over the global tile ids gives
// the ranges of the tile-sorted pairs; the counts summed per digit give the
// exclusive bucket offsets of every pass of the tile sort.  One block.
__global__ void __launch_bounds__(1024) tile_prep_kernel(int *D, const int *single, TileSet ts, TileOffsets off,
                                                         uint2 *ranges, uint32_t *hist, int hist_stride, int rb,
                                                         int passes, uint64_t capacity) {
    extern __shared__ uint32_t sh_hist[];  // passes * 2^rb
    const int R = 1 << rb;
    for (int j = threadIdx.x; j < passes * R; j += blockDim.x) sh_hist[j] = 0u;
    for (int c = 0; c < ts.n_cams; ++c) {
        const int tx = ts.cam[c].tiles_x, ty = ts.cam[c].tiles_y, stride = tx + 1;
        int *Dc = D + off.diff[c];
        const int *Sc = single + off.single[c];
        for (int y = threadIdx.x; y < ty; y += blockDim.x) {
            int run = 0;
            for (int x = 0; x < tx; ++x) {
                run += Dc[y * stride + x];
                Dc[y * stride + x] = run;
            }
        }
        __syncthreads();
        for (int x = threadIdx.x; x < tx; x += blockDim.x) {
            int run = 0;
            for (int y = 0; y < ty; ++y) {
                run += Dc[y * stride + x];
                Dc[y * stride + x] = run + Sc[y * tx + x];
            }
        }
        __syncthreads();
    }
    // exclusive scan of the counts over global tile ids, each thread a chunk
    const int ntiles = (int)ts.total_tiles;
    const int per = (ntiles + blockDim.x - 1) / blockDim.x;
    const int t0 = threadIdx.x * per, t1 = min(ntiles, t0 + per);
    auto count_of = [&](int t) -> uint32_t {
        const int c = camera_of(ts, (uint32_t)t);
        const int lt = t - (int)ts.cam[c].tile_base, tx = ts.cam[c].tiles_x;
        return (uint32_t)D[off.diff[c] + (lt / tx) * (tx + 1) + lt % tx];
    };
    uint64_t local64 = 0;
    for (int t = t0; t < t1; ++t) local64 += count_of(t);
    uint64_t total64;
    block_incl_scan<uint64_t>(local64, &total64);
    // more pairs than the buffers hold (the emit flags it): every tile empty
    const bool over = total64 > capacity;
    uint32_t local = over ? 0u : (uint32_t)local64;
    uint32_t total;
    uint32_t run = block_incl_scan<uint32_t>(local, &total) - local;
    for (int t = t0; t < t1; ++t) {
        const uint32_t c = over ? 0u : count_of(t);
        ranges[t] = c ? make_uint2(run, run + c) : make_uint2(0u, 0u);  // [0,0) for an empty tile
        run += c;
        for (int p = 0; p < passes; ++p) atomicAdd(&sh_hist[p * R + ((t >> (p * rb)) & (R - 1))], c);
    }
    __syncthreads();
    // exclusive offsets per pass
    for (int p = 0; p < passes; ++p) {
        const int per_d = (R + blockDim.x - 1) / blockDim.x;
        const int d0 = threadIdx.x * per_d, d1 = min(R, d0 + per_d);
        uint32_t s = 0;
        for (int d = d0; d < d1; ++d) s += sh_hist[p * R + d];
        uint32_t tot;
        uint32_t r = block_incl_scan<uint32_t>(s, &tot) - s;
        for (int d = d0; d < d1; ++d) {
            hist[p * hist_stride + d] = r;
            r += sh_hist[p * R + d];
        }
    }
}

cudaError_t launch_tile_prep(int *tile_diff, const int *tile_single, const TileSet &ts, const uint32_t *diff_off,
                             const uint32_t *single_off, uint2 *ranges, uint32_t *hist, int hist_stride,
                             int digit_bits, int passes, uint64_t capacity, cudaStream_t s) {
    TileOffsets off;
    for (int c = 0; c < kMaxGroupCams; ++c) {
        off.diff[c] = c < ts.n_cams ? diff_off[c] : 0u;
        off.single[c] = c < ts.n_cams ? single_off[c] : 0u;
    }
    const size_t smem = (size_t)passes * ((size_t)1 << digit_bits) * 4;
    tile_prep_kernel<<<1, 1024, smem, s>>>(tile_diff, tile_single, ts, off, ranges, hist, hist_stride, digit_bits,
                                           passes, capacity);
    return cudaGetLastError();
}

template cudaError_t launch_ranges<uint64_t>(const uint64_t *, uint64_t, const uint64_t *, uint2 *, int, cudaStream_t);
template cudaError_t launch_ranges<uint32_t>(const uint32_t *, uint64_t, const uint64_t *, uint2 *, int, cudaStream_t);

}  // namespace qb
