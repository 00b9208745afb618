// qb_binning.cu -- K2 exclusive scan of the per-Gaussian tile counts, K3
// DuplicateWithKeys with QPass traversal (Sec. 2, Sec. 3.2), and K5, the
// per-tile ranges of the sorted pairs.
//
// Pairs are emitted in an "emission order" of the Gaussians: index order for
// the full-key path, depth order for the depth-first path.  The scan runs in
// that order, so each Gaussian's pairs are one contiguous run and a warp's 32
// Gaussians own one contiguous output range.
#include "qb_sweep.cuh"

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

// K2 in one pass: block b (taken in launch order from a counter, so every
// earlier block is already running) scans its kScanChunk counts, publishes
// its sum, looks back over the earlier blocks' published words for its
// running total (decoupled look-back) and writes its offsets.  Status word of
// a block: flag (bit 63: sum of the block, bit 62: total through the block)
// and a 62-bit count.  The last block writes P.
constexpr uint64_t kScanAgg = 1ull << 63, kScanIncl = 1ull << 62, kScanCount = kScanIncl - 1;

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Besides the offsets it can write the counts in emission order (counts_e)
// and, for every run of kEmitStride output positions starting at c
// kEmitStride, the emission position whose pairs hold that start
// (chunk_first[c], c < chunk_cap), so the emit's warps find their first
// Gaussian with one load instead of a search.
__global__ void __launch_bounds__(kScanBlock) scan_onepass_kernel(const uint32_t *__restrict__ counts,
                                                                  const uint32_t *__restrict__ perm, int n,
                                                                  uint32_t *__restrict__ offsets, uint64_t *status,
                                                                  uint32_t *counter, uint64_t *n_pairs, uint32_t *err,
                                                                  uint32_t *__restrict__ counts_e,
                                                                  uint32_t *__restrict__ chunk_first, uint32_t chunk_cap) {
    __shared__ uint32_t s_block;
    __shared__ uint64_t s_prefix;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) s_block = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t b = s_block;
    const int nb = (n + kScanChunk - 1) / kScanChunk;
    // each thread scans kScanItems consecutive counts (in emission order)
    const size_t base = (size_t)b * kScanChunk + (size_t)tid * kScanItems;
    uint32_t c[kScanItems];
    uint64_t sum = 0;
    if (base + kScanItems <= (size_t)n && perm) {
        uint32_t g[kScanItems];
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            const uint4 v = reinterpret_cast<const uint4 *>(perm + base)[q];
            g[4 * q] = v.x, g[4 * q + 1] = v.y, g[4 * q + 2] = v.z, g[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) c[k] = counts[g[k]];
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) c[k] = base + k < (size_t)n ? count_at(counts, perm, base + k) : 0u;
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) sum += c[k];
    uint64_t total;
    const uint64_t incl = block_incl_scan<uint64_t>(sum, &total);
    // publish, then look back (warp 0, 32 earlier blocks per step)
    if (tid == 0) st_relaxed_u64(status + b, (b == 0 ? kScanIncl : kScanAgg) | total);
    if (tid < 32) {
        // The words of blocks t, t - 1, ..., t - 31 are read together; the
        // sums of the lanes before the first word not yet published are
        // added, up to and including the first inclusive word, which ends the
        // walk.  (Before block 0 reads as an inclusive zero.)
        uint64_t acc = 0;
        int64_t t = (int64_t)b - 1;
        int spins = 0;
        while (t >= 0) {
            const int64_t mine = t - lane;
            const uint64_t w = mine >= 0 ? ld_relaxed_u64(status + mine) : kScanIncl;
            const uint32_t ready = __ballot_sync(0xffffffffu, (w & (kScanAgg | kScanIncl)) != 0);
            const uint32_t inclm = __ballot_sync(0xffffffffu, (w & kScanIncl) != 0);
            const int first_unready = ready == 0xffffffffu ? 32 : __ffs(~ready) - 1;
            const int first_incl = inclm ? __ffs(inclm) - 1 : 32;
            const bool ends = first_incl < first_unready;
            const int used = ends ? first_incl + 1 : first_unready;
            uint64_t v = lane < used ? (w & kScanCount) : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            acc += v;
            if (ends) break;
            if (used > 0) {
                t -= used;
                continue;
            }
            // the nearest earlier block has not published yet
            if (++spins > kSpinLimit) {
                if (lane == 0) atomicOr(err, kErrTimeout);
                break;
            }
            __nanosleep(64);
        }
        if (lane == 0) {
            if (b > 0) st_relaxed_u64(status + b, kScanIncl | ((acc + total) & kScanCount));
            s_prefix = acc;
            if ((int)b == nb - 1) *n_pairs = acc + total;
        }
    }
    __syncthreads();
    uint64_t run = s_prefix + incl - sum;
    if (chunk_first) {
        uint64_t r = run;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (c[k] > 0u) {
                // the run starts [r, r + c) of this Gaussian that begin a chunk
                const uint64_t c0 = (r + kEmitStride - 1) / kEmitStride, c1 = (r + c[k] - 1) / kEmitStride;
                for (uint64_t ch = c0; ch <= c1 && ch < chunk_cap; ++ch) chunk_first[ch] = (uint32_t)(base + k);
            }
            r += c[k];
        }
    }
    if (counts_e) {
        if (base + kScanItems <= (size_t)n) {
#pragma unroll
            for (int q = 0; q < kScanItems / 4; ++q)
                reinterpret_cast<uint4 *>(counts_e + base)[q] = make_uint4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < kScanItems; ++k)
                if (base + k < (size_t)n) counts_e[base + k] = c[k];
        }
    }
    if (base + kScanItems <= (size_t)n) {
        uint32_t o[kScanItems];
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            o[k] = (uint32_t)run;  // P <= 2^30 is checked before use
            run += c[k];
        }
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q)
            reinterpret_cast<uint4 *>(offsets + base)[q] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (base + k < (size_t)n) offsets[base + k] = (uint32_t)run;
            run += c[k];
        }
    }
}

// status words for the blocks, then the block counter
size_t scan_partials_count(int n) { return (size_t)((n + kScanChunk - 1) / kScanChunk) + 1; }

cudaError_t launch_scan(const uint32_t *counts, const uint32_t *perm, int n, uint32_t *offsets, uint64_t *partials,
                        uint64_t *n_pairs, uint32_t *err, cudaStream_t s, uint32_t *counts_e, uint32_t *chunk_first,
                        uint32_t chunk_cap) {
    if (n == 0) return cudaMemsetAsync(n_pairs, 0, sizeof(uint64_t), s);
    const int nb = (n + kScanChunk - 1) / kScanChunk;
    cudaError_t e = cudaMemsetAsync(partials, 0, ((size_t)nb + 1) * sizeof(uint64_t), s);
    if (e != cudaSuccess) return e;
    note_launch("scan_onepass_kernel", s), scan_onepass_kernel<<<nb, kScanBlock, 0, s>>>(
        counts, perm, n, offsets, partials, reinterpret_cast<uint32_t *>(partials + nb), n_pairs, err, counts_e,
        chunk_first, chunk_cap);
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

constexpr int kEmitWarps = 4;  // warps per block (8 measured 0.7 % slower on the forward)
constexpr int kSegPerWarp = 32 * 7;
constexpr uint32_t kEmitChunk = 1024;  // output positions per warp (512, 2048, 4096 measured slower)
static_assert(kEmitChunk % kEmitStride == 0, "a warp's range starts on the scan's chunk table");

// One warp's table of QPass segments for a batch of 32 Gaussians.
struct SegTable {
    int32_t start[kSegPerWarp];  // chunk position of the segment's first pair
    uint32_t geo[kSegPerWarp];   // first line | first cell << 16
    uint32_t len[kSegPerWarp];   // cells per line | owner lane << 16 | column flag << 24
    float inv[kSegPerWarp];      // 1 / cells per line
    uint32_t gid[32], dbits[32];
    uint32_t tbase[32];  // first global tile of the owner's camera
    uint32_t tx[32];     // tiles per row of the owner's camera
};

// K3 (QPass modes and the single-box modes) for the pair positions
// [C, C + L) of the emission order, run by one warp.  It finds the first
// Gaussian whose run reaches into that range (32-ary search over the
// emission-order offsets), then takes the following Gaussians 32 at a time:
// each lane decomposes its Gaussian's QPass traversal into segments (runs of
// scan lines with one merged interval), and the warp produces the range 32
// consecutive positions at a time; lane q finds the segment holding its
// position from a ballot of the segment starts that fall in its group.
// sink(valid, p, tile, gid, depth bits) is called by all 32 lanes together
// once per group of 32 positions; valid lanes carry position C + p.
template <typename KeyOut, class Sink>
__device__ __forceinline__ void emit_range(const EmitArgs &a, uint64_t C, int32_t L, SegTable &S, Sink &&sink) {
    const int lane = threadIdx.x & 31;
    // last emission position j with offsets[j] <= C (offsets are non-decreasing):
    // from the scan's table when it wrote one (C is a multiple of the stride)
    int64_t lo = 0, hi = a.n - 1;  // invariant: offsets[lo] <= C, answer in [lo, hi]
    if (a.chunk_first) lo = hi = a.chunk_first[C / kEmitStride];
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
    int32_t done_to = 0;  // chunk positions [0, done_to) produced
    while (done_to < L && j0 < a.n) {
        const int64_t j = j0 + lane;
        uint32_t gid = 0, cnt = 0;
        int64_t rel = (int64_t)1 << 40;
        if (j < a.n) {
            gid = a.perm ? a.perm[j] : (uint32_t)j;
            cnt = a.counts_e ? a.counts_e[j] : a.counts[gid];
            rel = (int64_t)a.offsets[j] - (int64_t)C;
        }
        const bool relevant = cnt > 0u && rel < L && rel + (int64_t)cnt > 0;
        QSeg seg[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) seg[q] = QSeg{0, 0, 0, 0};
        bool columns = false;
        uint32_t dbits = 0, tbase = 0, tx_n = 1;
        if (relevant) {
            // the preprocess's segment record (slots beyond its count are zero)
            const CamTile &cam = a.ts.cam[gid / (uint32_t)a.n_per_cam];
            tbase = cam.tile_base;
            tx_n = (uint32_t)cam.tiles_x;
            if (sizeof(KeyOut) == 8) dbits = __float_as_uint(a.rgbd[gid].w) & 0x7fffffffu;
            const uint4 *src = a.segs + 4 * (size_t)gid;
            uint32_t w[16];
            const uint4 c0 = src[0];
            w[0] = c0.x; w[1] = c0.y; w[2] = c0.z; w[3] = c0.w;
            const int n_in = (int)(c0.x & 7u);
            columns = (c0.x >> 3) & 1u;
            const int nc = seg_chunks(n_in);
#pragma unroll
            for (int c = 1; c < 4; ++c) {
                const uint4 v = c < nc ? src[c] : make_uint4(0u, 0u, 0u, 0u);
                w[4 * c] = v.x; w[4 * c + 1] = v.y; w[4 * c + 2] = v.z; w[4 * c + 3] = v.w;
            }
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                if (q >= n_in) continue;
                seg[q].s0 = (int)(w[1 + 2 * q] & 0xffffu);
                seg[q].lo = (int)(w[1 + 2 * q] >> 16);
                seg[q].nl = (int)(w[2 + 2 * q] & 0xffffu);
                seg[q].len = (int)(w[2 + 2 * q] >> 16);
            }
        }
        int ns = 0;
#pragma unroll
        for (int q = 0; q < 7; ++q) ns += seg_empty(seg[q]) ? 0 : 1;
        __syncwarp();
        S.gid[lane] = gid;
        S.dbits[lane] = dbits;
        S.tbase[lane] = tbase;
        S.tx[lane] = tx_n;
        const int sincl = warp_incl_scan(ns);
        const int nseg = __shfl_sync(0xffffffffu, sincl, 31);
        int32_t r0 = (int32_t)(rel > -((int64_t)1 << 30) ? rel : -((int64_t)1 << 30));
        int k = sincl - ns;  // this lane's first table entry
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            if (seg_empty(seg[q])) continue;
            S.start[k] = r0;
            S.geo[k] = (uint32_t)seg[q].s0 | ((uint32_t)seg[q].lo << 16);
            S.len[k] = (uint32_t)seg[q].len | ((uint32_t)lane << 16) | ((uint32_t)columns << 24);
            S.inv[k] = 1.0f / (float)seg[q].len;
            r0 += seg[q].nl * seg[q].len;
            ++k;
        }
        // end of this batch's pairs within the chunk
        const int64_t last_end = __shfl_sync(0xffffffffu, rel + (int64_t)cnt, 31);
        const int32_t batch_end = (int32_t)(last_end < (int64_t)L ? last_end : (int64_t)L);
        __syncwarp();
        // cur: last segment starting at or before done_to
        int cur = -1;
        for (int b = 0; b < nseg; b += 32) {
            const bool le = b + lane < nseg && S.start[b + lane] <= done_to;
            cur += __popc(__ballot_sync(0xffffffffu, le));
        }
        for (int32_t c0 = done_to; c0 < batch_end; c0 += 32) {
            const int cand = cur + 1 + lane;
            uint32_t bit = 0u;
            if (cand < nseg) {
                const int32_t st = S.start[cand];
                if (st < c0 + 32) bit = 1u << (st - c0);
            }
            const uint32_t M = __reduce_or_sync(0xffffffffu, bit);
            const int32_t p = c0 + lane;
            const bool valid = p < batch_end;
            uint32_t tile = 0u, gid_out = 0u, dbits_out = 0u;
            if (valid) {
                const int idx = cur + __popc(M & le_mask);
                const int32_t st = S.start[idx];
                const uint32_t geo = S.geo[idx], ln = S.len[idx];
                const uint32_t k = (uint32_t)(p - st), len = ln & 0xffffu;
                // k / len through the reciprocal (k < 2^24, so the estimate is
                // off by at most one) and one exact correction
                int32_t q = (int32_t)((float)k * S.inv[idx]);
                int32_t r = (int32_t)k - q * (int32_t)len;
                if (r < 0) { --q; r += (int32_t)len; }
                if (r >= (int32_t)len) { ++q; r -= (int32_t)len; }
                const uint32_t line = (geo & 0xffffu) + (uint32_t)q;
                const uint32_t u = (geo >> 16) + (uint32_t)r;
                const bool cols = (ln >> 24) & 1u;
                const uint32_t owner = (ln >> 16) & 0xffu;
                tile = S.tbase[owner] + (cols ? u : line) * S.tx[owner] + (cols ? line : u);
                gid_out = S.gid[owner];
                dbits_out = S.dbits[owner];
            }
            sink(valid, p, tile, gid_out, dbits_out);  // all lanes, converged
            cur += __popc(M);
        }
        done_to = max(done_to, batch_end);
        j0 += 32;
    }
}

// K3 balanced over the output: warp w owns the pair positions
// [w C, (w+1) C), so stores are contiguous across the warp and every warp
// writes at most C pairs however large the Gaussians are.
template <typename KeyT>
__global__ void __launch_bounds__(kEmitWarps * 32) emit_warp_kernel(EmitArgs a, KeyT *__restrict__ keys) {
    __shared__ SegTable s_seg[kEmitWarps];
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
    uint32_t *vals = a.vals;
    emit_range<KeyT>(a, C, L, s_seg[wid], [&](bool valid, int32_t p, uint32_t tile, uint32_t gid, uint32_t dbits) {
        if (valid) {
            keys[C + p] = make_key<KeyT>(tile, dbits);
            vals[C + p] = gid;
        }
    });
}

// K3 fused with the first (lowest-digit) pass of the depth-first tile sort:
// a block of kSortWarps warps produces the pairs of one sort tile into shared
// memory (warp w the positions [256 w, 256 w + 256)), then runs the pass
// body on them, so the pairs reach HBM once, already bucketed by their low
// tile digit.  The bucket offsets of the pass come from the per-tile counts.
constexpr size_t kEmitSweepStage = (size_t)2 * kSortTile * 4;

template <int RB>
constexpr size_t emit_sweep_smem() {
    return kEmitSweepStage + kSortWarps * sizeof(SegTable) > sweep_smem<RB, uint32_t>()
               ? kEmitSweepStage + kSortWarps * sizeof(SegTable)
               : sweep_smem<RB, uint32_t>();
}

template <int RB, bool WRITE_KEYS>
__global__ void __launch_bounds__(kSortBlock) emit_sweep_kernel(EmitArgs a, uint32_t *__restrict__ kout,
                                                                uint32_t *__restrict__ vout,
                                                                const uint32_t *__restrict__ bin_off,
                                                                uint32_t *lookback, uint32_t *counter, uint32_t mask) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *s_k = reinterpret_cast<uint32_t *>(smem);
    uint32_t *s_v = s_k + kSortTile;
    SegTable *s_seg = reinterpret_cast<SegTable *>(smem + kEmitSweepStage);
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t P = *a.n_pairs;
    if (P > a.capacity) {  // block-uniform
        if (tile == 0 && tid == 0) atomicOr(a.err, kErrCapacity);
        return;
    }
    const uint64_t tbase = (uint64_t)tile * kSortTile;
    if (tbase >= P) return;  // block-uniform
    constexpr int kWarpSpan = 32 * kSortItems;
    const uint64_t C = tbase + (uint64_t)wid * kWarpSpan;
    const int32_t L = C < P ? (int32_t)min((uint64_t)kWarpSpan, P - C) : 0;
    uint32_t *wk = s_k + wid * kWarpSpan, *wv = s_v + wid * kWarpSpan;
    if (L > 0)
        emit_range<uint32_t>(a, C, L, s_seg[wid], [&](bool valid, int32_t p, uint32_t tile_id, uint32_t gid, uint32_t) {
            if (valid) {
                wk[p] = tile_id;
                wv[p] = gid;
            }
        });
    __syncthreads();
    uint32_t key[kSortItems], val[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const int q = 32 * k + lane;
        const bool valid = q < L;
        key[k] = valid ? wk[q] : ~0u;
        val[k] = valid ? wv[q] : 0u;
    }
    __syncthreads();  // the pass body reuses the staging memory
    sweep_tile<RB, uint32_t, WRITE_KEYS ? kOutPairs : kOutValues>(key, [&](int k) { return val[k]; }, (uint32_t)P,
                                                                  (uint32_t)tbase, tile, bin_off, lookback, 0, mask,
                                                                  a.err, kout, vout, smem);
}

template <int RB, bool WRITE_KEYS>
static cudaError_t launch_emit_sweep_b(const EmitArgs &a, uint32_t *kout, uint32_t *vout, const uint32_t *bin_off,
                                       uint32_t *lookback, uint32_t *counter, uint32_t mask, cudaStream_t s) {
    constexpr size_t smem = emit_sweep_smem<RB>();
    cudaError_t e = ensure_dyn_smem((const void *)emit_sweep_kernel<RB, WRITE_KEYS>, smem);
    if (e != cudaSuccess) return e;
    const uint64_t pairs = a.n_pairs_host != UINT64_MAX ? a.n_pairs_host : a.capacity;
    uint64_t blocks = (pairs + kSortTile - 1) / kSortTile;
    if (blocks == 0) blocks = 1;  // one block still flags an overflow
    note_launch("emit_sweep_kernel", s), emit_sweep_kernel<RB, WRITE_KEYS><<<(unsigned)blocks, kSortBlock, smem, s>>>(a, kout, vout, bin_off, lookback,
                                                                               counter, mask);
    return cudaGetLastError();
}

cudaError_t launch_emit_sweep(const EmitArgs &a, int digit_bits, bool write_keys, uint32_t *kout, uint32_t *vout,
                              const uint32_t *bin_off, uint32_t *lookback, uint32_t *counter, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
#define QB_SWEEP_CASE(RB)                                                                                        \
    case RB:                                                                                                     \
        return write_keys ? launch_emit_sweep_b<RB, true>(a, kout, vout, bin_off, lookback, counter, mask, s)    \
                          : launch_emit_sweep_b<RB, false>(a, kout, vout, bin_off, lookback, counter, mask, s);
    const uint32_t mask = (1u << digit_bits) - 1u;
    switch (digit_bits < 4 ? 4 : digit_bits) {  // the width of the first pass (pass_geo)
        QB_SWEEP_CASE(4)
        QB_SWEEP_CASE(5)
        QB_SWEEP_CASE(6)
        QB_SWEEP_CASE(7)
        QB_SWEEP_CASE(8)
        QB_SWEEP_CASE(9)
        QB_SWEEP_CASE(10)
        QB_SWEEP_CASE(11)
    default: return cudaErrorInvalidValue;
    }
#undef QB_SWEEP_CASE
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
        note_launch("emit_naive_kernel", s), emit_naive_kernel<KeyT><<<(a.n + 255) / 256, 256, 0, s>>>(a, keys);
    } else {
        const uint64_t pairs = a.n_pairs_host != UINT64_MAX ? a.n_pairs_host : a.capacity;
        const uint64_t warps = (pairs + kEmitChunk - 1) / kEmitChunk;
        const uint64_t blocks = (warps + kEmitWarps - 1) / kEmitWarps;
        if (blocks > 0) note_launch("emit_warp_kernel", s), emit_warp_kernel<KeyT><<<(unsigned)blocks, kEmitWarps * 32, 0, s>>>(a, keys);
        else if (a.n > 0) note_launch("emit_warp_kernel", s), emit_warp_kernel<KeyT><<<1, kEmitWarps * 32, 0, s>>>(a, keys);  // flags overflow
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

// The same for u32 tile ids, four keys per thread from one 16-byte load; the
// neighbours across threads come by shuffle, across warps by one extra load.
__global__ void ranges4_kernel(const uint32_t *__restrict__ keys, uint64_t n_max, const uint64_t *n_dev,
                               uint2 *ranges, uint32_t ntiles) {
    const unsigned F = 0xffffffffu;
    const uint32_t none = 0xffffffffu;  // no tile id
    const uint64_t n = n_dev ? (*n_dev > n_max ? 0 : *n_dev) : n_max;
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); 4 * base < n; base += stride) {
        const uint64_t i0 = 4 * (base + lane);  // the loop is warp-uniform
        uint32_t k[4];
        if (i0 + 4 <= n) {
            const uint4 v = reinterpret_cast<const uint4 *>(keys)[i0 / 4];  // 256-byte aligned buffer
            k[0] = v.x, k[1] = v.y, k[2] = v.z, k[3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) k[j] = i0 + j < n ? keys[i0 + j] : none;
        }
        uint32_t prev = __shfl_up_sync(F, k[3], 1), next = __shfl_down_sync(F, k[0], 1);
        if (lane == 0) prev = i0 > 0 ? keys[i0 - 1] : none;  // i0 <= 4 base < n
        if (lane == 31) next = i0 + 4 < n ? keys[i0 + 4] : none;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t t = k[j];
            if (t >= ntiles) continue;  // past the end (none), or never for keys written by the emit kernels
            const uint32_t p = j == 0 ? prev : k[j - 1], q = j == 3 ? next : k[j + 1];
            if (p != t) ranges[t].x = (uint32_t)(i0 + j);
            if (q != t) ranges[t].y = (uint32_t)(i0 + j + 1);
        }
    }
}

template <typename KeyT>
cudaError_t launch_ranges(const KeyT *keys, uint64_t n_max, const uint64_t *n_dev, uint2 *ranges, int ntiles,
                          cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)ntiles, s);
    if (e != cudaSuccess || n_max == 0) return e;
    if constexpr (sizeof(KeyT) == 4) {
        uint64_t blocks = (n_max / 4 + 255) / 256;
        if (blocks > 152 * 8) blocks = 152 * 8;
        if (blocks == 0) blocks = 1;
        note_launch("ranges4_kernel", s), ranges4_kernel<<<(unsigned)blocks, 256, 0, s>>>(keys, n_max, n_dev, ranges,
                                                                                          (uint32_t)ntiles);
    } else {
        uint64_t blocks = (n_max + 255) / 256;
        if (blocks > 152 * 16) blocks = 152 * 16;
        note_launch("ranges_kernel", s), ranges_kernel<KeyT><<<(unsigned)blocks, 256, 0, s>>>(keys, n_max, n_dev, ranges, (uint32_t)ntiles);
    }
    return cudaGetLastError();
}

// The tile id of every sorted pair position, from the ranges (one block per
// tile).
// Positions at or beyond n_out are not written.
__global__ void expand_ranges_kernel(const uint2 *ranges, uint32_t ntiles, uint32_t *out, uint64_t n_out) {
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint2 r = ranges[t];
        const uint64_t end = r.y < n_out ? r.y : n_out;
        for (uint64_t i = (uint64_t)r.x + threadIdx.x; i < end; i += blockDim.x) out[i] = t;
    }
}

cudaError_t launch_expand_ranges(const uint2 *ranges, int ntiles, uint32_t *out, uint64_t n_out, cudaStream_t s) {
    if (ntiles <= 0 || n_out == 0) return cudaSuccess;
    note_launch("expand_ranges_kernel", s), expand_ranges_kernel<<<ntiles < 65535 ? ntiles : 65535, 256, 0, s>>>(ranges, (uint32_t)ntiles, out, n_out);
    return cudaGetLastError();
}

// Per-tile pair counts from the emitted tile ids: a shared-memory histogram
// per block, merged into counts (zeroed by the caller) with global atomics.
// From the per-tile counts, run by one block: the ranges, and for every pass
// of the tile sort the exclusive bucket offsets of its digit.  s[0, ntiles)
// holds the counts (all zero when the pairs exceed the capacity) and becomes
// the exclusive offsets, s[ntiles] the total (prep_ranges); s_dsum has room
// for 2^kMaxDigitBits digit sums.
__device__ __forceinline__ void prep_ranges(uint32_t *s, int ntiles, uint2 *ranges) {
    // each thread turns a contiguous chunk into offsets, then the ranges
    // leave in tile order (coalesced)
    const int per = (ntiles + (int)blockDim.x - 1) / (int)blockDim.x;
    const int t0 = (int)threadIdx.x * per, t1 = min(ntiles, t0 + per);
    uint32_t local = 0;
#pragma unroll 8
    for (int t = t0; t < t1; ++t) local += s[t];
    uint32_t total;
    uint32_t run = block_incl_scan<uint32_t>(local, &total) - local;
    for (int t = t0; t < t1; ++t) {
        const uint32_t c = s[t];
        s[t] = run;
        run += c;
    }
    if (threadIdx.x == 0) s[ntiles] = total;
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const uint32_t o0 = s[t], o1 = s[t + 1];
        ranges[t] = o1 > o0 ? make_uint2(o0, o1) : make_uint2(0u, 0u);  // [0,0) for an empty tile
    }
}

// After prep_ranges.  A digit d of pass p (width b, shift h) covers the runs
// of 2^h consecutive tiles that start at u 2^(b+h) + d 2^h; each run's sum is
// a difference of two offsets.  The runs are spread over the block's threads
// (consecutive runs, consecutive digits: no conflicting shared atomics).
__device__ __forceinline__ void prep_digits(const uint32_t *s, uint32_t *s_dsum, int ntiles, uint32_t *hist,
                                            int hist_stride, const PassGeo &g) {
    for (int p = 0; p < g.passes; ++p) {
        const int Rp = 1 << g.bits[p], sh = g.shift[p];
        const int period = Rp << sh;
        const int runs = Rp * ((ntiles + period - 1) / period);
        for (int d = threadIdx.x; d < Rp; d += blockDim.x) s_dsum[d] = 0u;
        __syncthreads();
        for (int i = threadIdx.x; i < runs; i += blockDim.x) {
            const int d = i & (Rp - 1), u = i >> g.bits[p];
            const int a = u * period + (d << sh);
            if (a >= ntiles) continue;
            const int e = min(ntiles, a + (1 << sh));
            const uint32_t v = s[e] - s[a];
            if (v) atomicAdd(&s_dsum[d], v);
        }
        __syncthreads();
        // exclusive offsets over the digits, a contiguous chunk per thread
        const int per_d = (Rp + (int)blockDim.x - 1) / (int)blockDim.x;
        const int d0 = (int)threadIdx.x * per_d, d1 = min(Rp, d0 + per_d);
        uint32_t sum = 0;
        for (int d = d0; d < d1; ++d) sum += s_dsum[d];
        uint32_t tot;
        uint32_t r = block_incl_scan<uint32_t>(sum, &tot) - sum;
        for (int d = d0; d < d1; ++d) {
            hist[p * hist_stride + d] = r;
            r += s_dsum[d];
        }
        __syncthreads();
    }
}

// Shared-memory histogram of the emitted tile ids, added into counts.  With
// prep, the last block to finish (a counter at counts[ntiles], zero at
// launch) turns the totals into the ranges and the tile sort's bucket offsets
// (prep_ranges, prep_digits), so no separate launch waits for the histogram.
__global__ void __launch_bounds__(512) tile_count_kernel(const uint32_t *__restrict__ keys, uint64_t n_max,
                                                         const uint64_t *n_dev, uint32_t ntiles, uint32_t *counts,
                                                         bool prep, uint2 *ranges, uint32_t *hist, int hist_stride,
                                                         PassGeo g) {
    extern __shared__ uint32_t s_hist[];
    __shared__ bool s_last;
    for (uint32_t t = threadIdx.x; t < ntiles; t += blockDim.x) s_hist[t] = 0u;
    __syncthreads();
    const uint64_t n = device_count(n_dev, n_max);
    const uint64_t n4 = n / 4, stride = (uint64_t)gridDim.x * blockDim.x;
    const uint4 *k4 = reinterpret_cast<const uint4 *>(keys);  // 256-byte aligned buffer
    // four independent 16-byte loads in flight per thread
    constexpr int U = 4;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += U * stride) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t j = i + u * stride;
            v[u] = j < n4 ? __ldcs(k4 + j) : make_uint4(~0u, ~0u, ~0u, ~0u);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (v[u].x < ntiles) atomicAdd(&s_hist[v[u].x], 1u);
            if (v[u].y < ntiles) atomicAdd(&s_hist[v[u].y], 1u);
            if (v[u].z < ntiles) atomicAdd(&s_hist[v[u].z], 1u);
            if (v[u].w < ntiles) atomicAdd(&s_hist[v[u].w], 1u);
        }
    }
    for (uint64_t i = 4 * n4 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t k = keys[i];
        if (k < ntiles) atomicAdd(&s_hist[k], 1u);
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const uint32_t v = s_hist[t];
        if (v) atomicAdd(&counts[t], v);
    }
    if (!prep) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&counts[ntiles], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // (more pairs than the buffers hold: device_count gave 0 and every count is 0)
    // eight independent loads in flight per thread
    for (uint32_t b0 = 0; b0 < ntiles; b0 += 8 * blockDim.x) {
        uint32_t v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t t = b0 + k * blockDim.x + threadIdx.x;
            v[k] = t < ntiles ? __ldcg(counts + t) : 0u;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t t = b0 + k * blockDim.x + threadIdx.x;
            if (t < ntiles) s_hist[t] = v[k];
        }
    }
    __syncthreads();
    prep_ranges(s_hist, (int)ntiles, ranges);
    prep_digits(s_hist, s_hist + ntiles + 1, (int)ntiles, hist, hist_stride, g);
}

cudaError_t launch_tile_count(const uint32_t *keys, uint64_t n_max, const uint64_t *n_dev, int ntiles,
                              uint32_t *counts, uint2 *ranges, uint32_t *hist, int hist_stride, int digit_bits,
                              int tile_bits, cudaStream_t s) {
    // the counts and the finished-block counter after them
    cudaError_t e = cudaMemsetAsync(counts, 0, 4 * ((size_t)ntiles + 1), s);
    if (e != cudaSuccess || ntiles == 0) return e;
    // the histogram; for the last block's prep also the total and the digit sums
    const size_t smem = 4 * ((size_t)ntiles + 1 + ((size_t)1 << kMaxDigitBits));
    if ((e = ensure_dyn_smem((const void *)tile_count_kernel, smem)) != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t blocks = (n_max / 4 + 511) / 512;
    if (blocks > (uint64_t)sms * 2) blocks = (uint64_t)sms * 2;
    if (blocks == 0) blocks = 1;
    const PassGeo g = pass_geo(tile_bits, digit_bits);
    note_launch("tile_count_kernel", s), tile_count_kernel<<<(unsigned)blocks, 512, smem, s>>>(
        keys, n_max, n_dev, (uint32_t)ntiles, counts, ranges != nullptr, ranges, hist, hist_stride, g);
    return cudaGetLastError();
}

// Per-tile pair counts from the difference arrays written by the preprocess:
// for every camera of the set a 2D prefix sum plus the single-tile counts
// gives each tile's count; an exclusive scan over the global tile ids gives
// the ranges of the tile-sorted pairs; the counts summed per digit give the
// exclusive bucket offsets of every pass of the tile sort.  One block.
__global__ void __launch_bounds__(1024) tile_prep_kernel(int *D, const int *single, TileSet ts, TileOffsets off,
                                                         uint2 *ranges, uint32_t *hist,
                                                         int hist_stride, int rb, PassGeo g, uint64_t capacity) {
    extern __shared__ uint32_t sh_hist[];  // passes x 2^rb
    const int R = 1 << rb, passes = g.passes;
    for (int j = threadIdx.x; j < passes * R; j += blockDim.x) sh_hist[j] = 0u;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int c = 0; c < ts.n_cams; ++c) {
        const int tx = ts.cam[c].tiles_x, ty = ts.cam[c].tiles_y, stride = tx + 1;
        int *Dc = D + off.diff[c];
        const int *Sc = single + off.single[c];
        // prefix along x: one warp per row, 32 cells at a time
        for (int y = wid; y < ty; y += nwarps) {
            int carry = 0;
            for (int x0 = 0; x0 < tx; x0 += 32) {
                const int x = x0 + lane;
                const int v = x < tx ? Dc[y * stride + x] : 0;
                const int incl = warp_incl_scan(v) + carry;
                if (x < tx) Dc[y * stride + x] = incl;
                carry = __shfl_sync(0xffffffffu, incl, 31);
            }
        }
        __syncthreads();
        // prefix along y: one thread per column, eight rows loaded at a time
        for (int x = threadIdx.x; x < tx; x += blockDim.x) {
            int run = 0;
            for (int y0 = 0; y0 < ty; y0 += 8) {
                int v[8], sg[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const bool in = y0 + k < ty;
                    v[k] = in ? Dc[(y0 + k) * stride + x] : 0;
                    sg[k] = in ? Sc[(y0 + k) * tx + x] : 0;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    run += v[k];
                    if (y0 + k < ty) Dc[(y0 + k) * stride + x] = run + sg[k];
                }
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
        for (int p = 0; p < passes; ++p)
            if (c) atomicAdd(&sh_hist[p * R + ((t >> g.shift[p]) & ((1 << g.bits[p]) - 1))], c);
    }
    __syncthreads();
    // exclusive offsets per pass
    for (int p = 0; p < passes; ++p) {
        const int Rp = 1 << g.bits[p];
        const int per_d = (Rp + blockDim.x - 1) / blockDim.x;
        const int d0 = threadIdx.x * per_d, d1 = min(Rp, d0 + per_d);
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

cudaError_t launch_tile_prep(int *tile_diff, const int *tile_single, const TileSet &ts,
                             const uint32_t *diff_off, const uint32_t *single_off, uint2 *ranges, uint32_t *hist,
                             int hist_stride, int digit_bits, int tile_bits, uint64_t capacity, cudaStream_t s) {
    const PassGeo g = pass_geo(tile_bits, digit_bits);
    const int passes = g.passes;
    TileOffsets off;
    for (int c = 0; c < kMaxGroupCams; ++c) {
        off.diff[c] = c < ts.n_cams ? diff_off[c] : 0u;
        off.single[c] = c < ts.n_cams ? single_off[c] : 0u;
    }
    const size_t smem = (size_t)passes * ((size_t)1 << digit_bits) * 4;
    note_launch("tile_prep_kernel", s), tile_prep_kernel<<<1, 1024, smem, s>>>(tile_diff, tile_single, ts, off, ranges, hist,
                                                          hist_stride, digit_bits, g, capacity);
    return cudaGetLastError();
}

template cudaError_t launch_ranges<uint64_t>(const uint64_t *, uint64_t, const uint64_t *, uint2 *, int, cudaStream_t);
template cudaError_t launch_ranges<uint32_t>(const uint32_t *, uint64_t, const uint64_t *, uint2 *, int, cudaStream_t);

}  // namespace qb
