// qb_sort.cu -- K4: stable LSD radix sort of (u64 key, u32 value) pairs with a
// onesweep schedule (one kernel per digit pass, decoupled look-back across
// tiles), the SortPairs stage of the rasteriser (Sec. 2).
//
// Per sort: one upfront pass reads all keys and builds the digit histograms
// of every pass; a tiny kernel turns them into exclusive bucket offsets.
// Each digit pass then reads and writes the pairs once: a block takes the
// next tile of 4096 keys (tile order = launch order through an atomic
// counter, so every earlier tile belongs to a block that is already
// running), counts its digits, publishes the counts and looks back over
// earlier tiles for their running totals, ranks its keys per warp, and
// scatters keys then values through shared memory so that runs of equal
// digits leave as contiguous stores.  Every look-back spin is bounded; on
// expiry it raises kErrTimeout and still publishes, so no block waits forever.
#include <algorithm>

#include "qb_kernels.cuh"

namespace qb {

constexpr int kSortBlock = 512;
constexpr int kSortWarps = kSortBlock / 32;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortBlock * kSortItems;  // 4096 keys per block
constexpr int kSpinLimit = 1 << 22;
constexpr int kLookWindow = 8;  // status words fetched per look-back step
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagIncl = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1u;
constexpr int kHistStride = 1 << kMaxDigitBits;  // per-pass stride of the histogram table
constexpr size_t kSortHeader = (size_t)kMaxPasses * kHistStride * 4 + 256;

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Elements to sort: the device count when given, treated as zero when it
// exceeds the buffers (an overflow the emit has already flagged).
__device__ __forceinline__ uint64_t device_count(const uint64_t *n_dev, uint64_t n_max) {
    if (!n_dev) return n_max;
    const uint64_t n = *n_dev;
    return n > n_max ? 0 : n;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t *total) {
    __shared__ uint32_t ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < nw ? ws[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t u = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += u;
        }
        ws[lane] = s;
    }
    __syncthreads();
    uint32_t before = wid > 0 ? ws[wid - 1] : 0u;
    *total = ws[nw - 1];
    __syncthreads();
    return incl - v + before;
}

static inline int num_passes(int end_bit, int digit_bits) { return (end_bit + digit_bits - 1) / digit_bits; }

size_t sort_scratch_bytes(uint64_t n, int end_bit, int digit_bits) {
    if (digit_bits < 8 || digit_bits > kMaxDigitBits || end_bit < 1 || end_bit > 64) return 0;
    int passes = num_passes(end_bit, digit_bits);
    if (passes > kMaxPasses) return 0;
    uint64_t tiles = (n + kSortTile - 1) / kSortTile;
    return align256(kSortHeader + (size_t)passes * tiles * ((size_t)1 << digit_bits) * 4);
}

// Upfront histogram of every pass's digit.
template <int RB, typename KeyT>
__global__ void __launch_bounds__(256) sort_hist_kernel(const KeyT *__restrict__ keys, uint64_t n_max,
                                                        const uint64_t *n_dev, int passes, uint32_t *hist) {
    constexpr int R = 1 << RB;
    extern __shared__ uint32_t sh[];
    for (int j = threadIdx.x; j < passes * R; j += blockDim.x) sh[j] = 0u;
    __syncthreads();
    const uint64_t n = device_count(n_dev, n_max);
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const KeyT k = keys[idx];
        for (int p = 0; p < passes; ++p) atomicAdd(&sh[p * R + (int)((k >> (p * RB)) & (R - 1))], 1u);
    }
    // (keys from the depth-first emit are spatially coherent: many lanes of a
    // warp share a digit; the shared-memory atomics serialise them in hardware)
    __syncthreads();
    for (int j = threadIdx.x; j < passes * R; j += blockDim.x) {
        uint32_t v = sh[j];
        if (v) atomicAdd(&hist[(j / R) * kHistStride + (j % R)], v);
    }
}

// Counts -> exclusive bucket offsets, one block per pass.
template <int RB>
__global__ void __launch_bounds__(1024) sort_hist_scan_kernel(uint32_t *hist) {
    constexpr int R = 1 << RB;
    constexpr int PER = (R + 1023) / 1024;
    uint32_t *h = hist + blockIdx.x * kHistStride;
    uint32_t v[PER], s = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int idx = threadIdx.x * PER + k;
        v[k] = idx < R ? h[idx] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t run = block_excl_scan_u32(s, &total);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int idx = threadIdx.x * PER + k;
        if (idx < R) h[idx] = run;
        run += v[k];
    }
}

template <int RB, typename KeyT>
constexpr size_t onesweep_smem() {
    return (size_t)kSortTile * sizeof(KeyT) + (size_t)kSortWarps * (1 << RB) * 2 + (size_t)3 * (1 << RB) * 4;
}

// One digit pass.  Order of work inside a block: load the tile, count its
// digits (shared atomics, order-free), publish the counts and look back at
// once -- so successors never wait for this block's ranking -- then rank the
// keys within each warp in their original order, and scatter keys and values
// through shared memory.
template <int RB, typename KeyT>
__global__ void __launch_bounds__(kSortBlock) onesweep_kernel(const KeyT *__restrict__ kin,
                                                              const uint32_t *__restrict__ vin,
                                                              KeyT *__restrict__ kout, uint32_t *__restrict__ vout,
                                                              uint64_t n_max, const uint64_t *n_dev,
                                                              const uint32_t *__restrict__ bin_off,
                                                              uint32_t *lookback, uint32_t *counter, int shift,
                                                              uint32_t *err) {
    constexpr int R = 1 << RB;
    constexpr uint32_t MASK = R - 1;
    constexpr int PER = (R + kSortBlock - 1) / kSortBlock;
    extern __shared__ __align__(16) uint8_t smem[];
    KeyT *s_keys = reinterpret_cast<KeyT *>(smem);
    uint32_t *s_vals = reinterpret_cast<uint32_t *>(smem);
    uint16_t *s_whist = reinterpret_cast<uint16_t *>(smem + (size_t)kSortTile * sizeof(KeyT));
    uint32_t *s_gbase = reinterpret_cast<uint32_t *>(s_whist + kSortWarps * R);
    uint32_t *s_lstart = s_gbase + R;
    uint32_t *s_bcount = s_lstart + R;
    __shared__ uint32_t s_tile;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(counter, 1u);
    for (int j = tid; j < kSortWarps * R / 2; j += kSortBlock) reinterpret_cast<uint32_t *>(s_whist)[j] = 0u;
    for (int j = tid; j < R; j += kSortBlock) s_bcount[j] = 0u;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t n = device_count(n_dev, n_max);
    const uint64_t tbase = (uint64_t)tile * kSortTile;
    if (tbase >= n) return;  // block-uniform

    // ---- load (warp-striped: item k of lane l at wbase + 32k + l) ----
    const uint64_t wbase = tbase + (uint64_t)wid * (32 * kSortItems);
    KeyT key[kSortItems];
    uint32_t val[kSortItems];
    uint32_t rank[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        uint64_t idx = wbase + 32 * k + lane;
        key[k] = idx < n ? __ldcs(kin + idx) : ~KeyT(0);
    }
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        uint64_t idx = wbase + 32 * k + lane;
        val[k] = idx < n ? __ldcs(vin + idx) : 0u;
    }

    // ---- early digit counts of the tile ----
#pragma unroll
    for (int k = 0; k < kSortItems; ++k)
        if (wbase + 32 * k + lane < n) atomicAdd(&s_bcount[(uint32_t)(key[k] >> shift) & MASK], 1u);
    __syncthreads();

    // ---- publish, look back, publish the inclusive prefix ----
    // One status word per (tile, digit): a 2-bit flag (aggregate = the tile's
    // own count, inclusive = running total through the tile) and a 30-bit
    // count.  Each thread walks back for its digits, kLookWindow words at a
    // time (their addresses do not depend on what is read), adding aggregates
    // until it meets an inclusive total; when the next word is not yet
    // published it polls that word alone, sleeping between polls.
    uint32_t cnt[PER], tsum = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        int d = tid * PER + j;
        cnt[j] = d < R ? s_bcount[d] : 0u;
        tsum += cnt[j];
    }
    uint32_t *lb = lookback + (size_t)tile * R;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        int d = tid * PER + j;
        if (d < R) st_relaxed(lb + d, (tile == 0 ? kFlagIncl : kFlagAgg) | cnt[j]);
    }
    uint32_t btotal;
    uint32_t run = block_excl_scan_u32(tsum, &btotal);  // contains __syncthreads
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        int d = tid * PER + j;
        if (d >= R) continue;
        s_lstart[d] = run;
        run += cnt[j];
        uint32_t acc = 0;
        if (tile > 0) {
            int64_t t = (int64_t)tile - 1;
            int spins = 0;
            bool done = false;
            while (!done && t >= 0) {
                uint32_t sv[kLookWindow];
#pragma unroll
                for (int w = 0; w < kLookWindow; ++w)
                    sv[w] = (t - w >= 0) ? ld_relaxed(lookback + (size_t)(t - w) * R + d) : kFlagIncl;
                int used = 0;
#pragma unroll
                for (int w = 0; w < kLookWindow; ++w) {
                    if (done || used < w) continue;  // stopped at an unpublished word
                    const uint32_t f = sv[w] & ~kCountMask;
                    if (f == 0u) continue;
                    acc += sv[w] & kCountMask;
                    used = w + 1;
                    if (f == kFlagIncl) done = true;
                }
                t -= used;
                if (!done && used == 0) {
                    // the nearest earlier tile has not published this digit yet
                    unsigned ns = 32;
                    while ((ld_relaxed(lookback + (size_t)t * R + d) & ~kCountMask) == 0u) {
                        if (++spins > kSpinLimit) break;
                        __nanosleep(ns);
                        ns = ns < 512 ? 2 * ns : 512;
                    }
                    if (spins > kSpinLimit) {
                        atomicOr(err, kErrTimeout);
                        break;
                    }
                }
            }
            st_relaxed(lb + d, kFlagIncl | ((acc + cnt[j]) & kCountMask));
        }
        s_gbase[d] = bin_off[d] + acc;
    }
    __syncthreads();

    // ---- rank within the warp, in original order ----
    // Lanes holding the same digit are found with one ballot per digit bit.
    uint16_t *wh = s_whist + wid * R;
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const bool valid = wbase + 32 * k + lane < n;
        const uint32_t d = valid ? (uint32_t)(key[k] >> shift) & MASK : (uint32_t)R;
        const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
        uint32_t peers = valid ? vmask : ~vmask;
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const uint32_t bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bb : ~bb;
        }
        const uint32_t pre = valid ? (uint32_t)wh[d] : 0u;
        const uint32_t lower = __popc(peers & lt);
        __syncwarp();
        if (valid && lower == 0) wh[d] = (uint16_t)(pre + __popc(peers));
        __syncwarp();
        rank[k] = pre + lower;
    }
    __syncthreads();

    // ---- per digit: exclusive prefix over the warps ----
    for (int d = tid; d < R; d += kSortBlock) {
        uint32_t r = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            uint32_t c = s_whist[w * R + d];
            s_whist[w * R + d] = (uint16_t)r;
            r += c;
        }
    }
    __syncthreads();

    // ---- keys: scatter to block order in shared memory, then out ----
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        if (wbase + 32 * k + lane < n) {
            uint32_t d = (uint32_t)(key[k] >> shift) & MASK;
            uint32_t lr = s_lstart[d] + s_whist[wid * R + d] + rank[k];
            s_keys[lr] = key[k];
            rank[k] = lr;
        }
    }
    __syncthreads();
    const uint32_t tcount = (uint32_t)min((uint64_t)kSortTile, n - tbase);
    uint32_t dest[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        uint32_t j = tid + k * kSortBlock;
        if (j < tcount) {
            const KeyT kk = s_keys[j];
            uint32_t d = (uint32_t)(kk >> shift) & MASK;
            dest[k] = s_gbase[d] + (j - s_lstart[d]);
            if (dest[k] < n) kout[dest[k]] = kk;  // only false after a look-back timeout
        }
    }
    __syncthreads();
    // ---- values through the same permutation ----
#pragma unroll
    for (int k = 0; k < kSortItems; ++k)
        if (wbase + 32 * k + lane < n) s_vals[rank[k]] = val[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        uint32_t j = tid + k * kSortBlock;
        if (j < tcount && dest[k] < n) vout[dest[k]] = s_vals[j];
    }
}

template <int RB, typename KeyT>
static cudaError_t sort_impl(KeyT *keys, uint32_t *vals, KeyT *keys_alt, uint32_t *vals_alt, uint64_t n_max,
                             const uint64_t *n_dev, int end_bit, void *scratch, uint32_t *err, cudaStream_t s,
                             int *passes_out, bool hist_ready) {
    constexpr int R = 1 << RB;
    const int passes = num_passes(end_bit, RB);
    const uint64_t tiles = (n_max + kSortTile - 1) / kSortTile;
    uint8_t *base = static_cast<uint8_t *>(scratch);
    uint32_t *hist = reinterpret_cast<uint32_t *>(base);
    uint32_t *counters = reinterpret_cast<uint32_t *>(base + (size_t)kMaxPasses * kHistStride * 4);
    uint32_t *lookback = reinterpret_cast<uint32_t *>(base + kSortHeader);
    *passes_out = passes;
    // with hist_ready the caller has already written every pass's exclusive
    // bucket offsets into the histogram table: clear only counters and look-back
    const size_t clear_from = hist_ready ? (size_t)kMaxPasses * kHistStride * 4 : 0;
    cudaError_t e = cudaMemsetAsync(base + clear_from, 0,
                                    kSortHeader - clear_from + (size_t)passes * tiles * R * 4, s);
    if (e != cudaSuccess || n_max == 0) return e;

    static bool attrs_set = false;
    if (!attrs_set) {
        e = cudaFuncSetAttribute(onesweep_kernel<RB, KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)onesweep_smem<RB, KeyT>());
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(sort_hist_kernel<RB, KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kMaxPasses * R * 4);
        if (e != cudaSuccess) return e;
        attrs_set = true;
    }
    if (!hist_ready) {
        uint64_t hblocks = std::min<uint64_t>((n_max + 255) / 256, 152 * 4);
        sort_hist_kernel<RB, KeyT><<<(unsigned)hblocks, 256, (size_t)passes * R * 4, s>>>(keys, n_max, n_dev,
                                                                                            passes, hist);
        sort_hist_scan_kernel<RB><<<passes, 1024, 0, s>>>(hist);
    }
    KeyT *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    for (int p = 0; p < passes; ++p) {
        onesweep_kernel<RB, KeyT><<<(unsigned)tiles, kSortBlock, onesweep_smem<RB, KeyT>(), s>>>(
            kin, vin, kout, vout, n_max, n_dev, hist + p * kHistStride, lookback + (size_t)p * tiles * R,
            counters + p, p * RB, err);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    return cudaGetLastError();
}

template <typename KeyT>
static cudaError_t sort_dispatch(KeyT *keys, uint32_t *vals, KeyT *keys_alt, uint32_t *vals_alt, uint64_t n_max,
                                 const uint64_t *n_dev, int end_bit, int digit_bits, void *scratch, uint32_t *err,
                                 cudaStream_t s, int *passes_out, bool hist_ready) {
    if (end_bit > (int)(8 * sizeof(KeyT))) return cudaErrorInvalidValue;
    switch (digit_bits) {
    case 8:
        return sort_impl<8>(keys, vals, keys_alt, vals_alt, n_max, n_dev, end_bit, scratch, err, s, passes_out,
                            hist_ready);
    case 9:
        return sort_impl<9>(keys, vals, keys_alt, vals_alt, n_max, n_dev, end_bit, scratch, err, s, passes_out,
                            hist_ready);
    case 10:
        return sort_impl<10>(keys, vals, keys_alt, vals_alt, n_max, n_dev, end_bit, scratch, err, s, passes_out,
                             hist_ready);
    case 11:
        return sort_impl<11>(keys, vals, keys_alt, vals_alt, n_max, n_dev, end_bit, scratch, err, s, passes_out,
                             hist_ready);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint64_t n_max,
                       const uint64_t *n_dev, int end_bit, int digit_bits, void *scratch, uint32_t *err,
                       cudaStream_t s, int *passes_out) {
    return sort_dispatch(keys, vals, keys_alt, vals_alt, n_max, n_dev, end_bit, digit_bits, scratch, err, s,
                         passes_out, false);
}

cudaError_t sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, uint64_t n_max,
                       const uint64_t *n_dev, int end_bit, int digit_bits, void *scratch, uint32_t *err,
                       cudaStream_t s, int *passes_out, bool hist_ready) {
    return sort_dispatch(keys, vals, keys_alt, vals_alt, n_max, n_dev, end_bit, digit_bits, scratch, err, s,
                         passes_out, hist_ready);
}

uint32_t *sort_hist_table(void *scratch) { return static_cast<uint32_t *>(scratch); }
int sort_hist_stride() { return kHistStride; }

}  // namespace qb
