// qb_sweep.cuh -- the body of one digit pass of the onesweep radix sort
// (SortPairs, Sec. 2), shared by the plain pass kernel (qb_sort.cu) and the
// QPass emit that performs the tile sort's first pass itself (qb_binning.cu).
//
// A block owns one tile of kSortTile consecutive input positions; its keys arrive
// in registers, warp-striped (item k of lane l of warp w is position
// 32 kSortItems w + 32 k + l of the tile).  The block counts its digits (shared
// atomics, order-free), publishes the counts and looks back over earlier
// tiles for their running totals, ranks its keys per warp in input order,
// and scatters keys then values through shared memory so that runs of equal
// digits leave as contiguous stores.  Tile indices are taken from an atomic
// counter in launch order, so every earlier tile belongs to a block that is
// already running.  Every look-back spin is bounded; on expiry it raises
// kErrTimeout and still publishes, so no block waits forever.
#pragma once

#include <type_traits>

#include "qb_kernels.cuh"

namespace qb {

constexpr int kSortBlock = 256;
constexpr int kSortWarps = kSortBlock / 32;
constexpr int kSortItems = 16;
constexpr int kSortBlocksPerSM = 5;  // resident pass blocks per SM the registers are sized for (32-bit keys)
constexpr int kSortTile = kSortBlock * kSortItems;  // 4096 keys per block
constexpr int kSpinLimit = 1 << 22;
constexpr int kLookWindow = 8;  // status words fetched per look-back step
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagIncl = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1u;
constexpr int kHistStride = 1 << kMaxDigitBits;  // per-pass stride of the histogram table
// scratch: [bucket offset table: kMaxPasses x kHistStride u32][tile counters:
// kMaxPasses u32, padded to 256 B][look-back words: passes x tiles x 2^RB u32]
constexpr size_t kSortCounters = (size_t)kMaxPasses * kHistStride * 4;
constexpr size_t kSortHeader = kSortCounters + 256;

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The error word err[0] is followed by a test-only word, zero in normal use:
// when err[1] > 0, the block of tile 1 of every values-only pass (the last
// pass of a tile sort, whose output only the render reads) finds tile 0's
// status words unpublished and gives up after err[1] polls, so its wait runs
// out deterministically and raises kErrTimeout.  Its scatter positions then
// fall short of the true ones but stay inside [0, n); the sorted values are
// undefined.  Other waits keep the kSpinLimit bound.
__device__ __forceinline__ uint32_t stall_test(const uint32_t *err, uint32_t tile) {
    return tile == 1 ? ld_relaxed(err + 1) : 0u;
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

// Shared memory of one pass: the scatter buffer ((key, value) pairs for 32-bit
// keys; keys, then values, for 64-bit keys), per-warp digit counters, and
// per-digit global base, local start and tile count.
template <int RB, typename KeyT>
constexpr size_t sweep_smem() {
    return (size_t)kSortTile * 8 + (size_t)kSortWarps * (1 << RB) * 2 + (size_t)3 * (1 << RB) * 4;
}

// What a pass writes at each output position.
enum SweepOut : int {
    kOutPairs = 0,   // the key to kout and the value to vout
    kOutValues = 1,  // the value only (the last pass, whose keys the per-tile ranges imply)
    kOutPacked = 2,  // one word to kout: (key >> pack_shift) << vbits | value
};

// One pass over the tile `tile` (positions [tbase, tbase + kSortTile) of n) on the
// digit (key >> shift) & mask, mask < 2^RB.  val(k) gives item k's value; it
// is asked for only at the scatter, after the ranking (so a caller can load
// values late and keep fewer registers live).  bin_off: the pass's exclusive
// bucket offsets; lookback: the pass's status words [tiles][2^RB].  OUT
// (SweepOut) says what is written; kOutPacked (32-bit keys) needs values
// below 2^vbits and keys below 2^(pack_shift + 32 - vbits).
template <int RB, typename KeyT, int OUT, class ValFn>
__device__ __forceinline__ void sweep_tile(const KeyT (&key)[kSortItems], ValFn &&val,
                                           uint32_t n, uint32_t tbase, uint32_t tile,
                                           const uint32_t *__restrict__ bin_off, uint32_t *lookback, int shift,
                                           uint32_t mask, uint32_t *err, KeyT *__restrict__ kout,
                                           uint32_t *__restrict__ vout, uint8_t *smem, int pack_shift = 0,
                                           int vbits = 0) {
    static_assert(OUT != kOutPacked || sizeof(KeyT) == 4, "packed output is for 32-bit keys");
    constexpr bool WRITE_KEYS = OUT != kOutValues;
    constexpr int R = 1 << RB;
    constexpr int PER = (R + kSortBlock - 1) / kSortBlock;
    uint16_t *s_whist = reinterpret_cast<uint16_t *>(smem + (size_t)kSortTile * 8);
    uint32_t *s_gbase = reinterpret_cast<uint32_t *>(s_whist + kSortWarps * R);
    uint32_t *s_lstart = s_gbase + R;
    uint32_t *s_bcount = s_lstart + R;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int j = tid; j < kSortWarps * R / 2; j += kSortBlock) reinterpret_cast<uint32_t *>(s_whist)[j] = 0u;
    for (int j = tid; j < R; j += kSortBlock) s_bcount[j] = 0u;
    __syncthreads();
    const uint32_t wbase = tbase + (uint32_t)wid * (32 * kSortItems);
    // items of this warp that exist: item k of lane l is valid when 32 k + l < wcount
    const int wcount = n > wbase ? (int)min(n - wbase, (uint32_t)(32 * kSortItems)) : 0;
    uint32_t rank[kSortItems];
    auto dig = [&](int k) { return (uint32_t)(key[k] >> shift) & mask; };

    // ---- early digit counts of the tile ----
#pragma unroll
    for (int k = 0; k < kSortItems; ++k)
        if (32 * k + lane < wcount) atomicAdd(&s_bcount[dig(k)], 1u);
    __syncthreads();

    // ---- publish this tile's counts ----
    // One status word per (tile, digit): a 2-bit flag (aggregate = the tile's
    // own count, inclusive = running total through the tile) and a 30-bit
    // count.  (Prefetching the first look-back window here, across the ranking,
    // was measured slower: its registers made the pass spill at five blocks per
    // SM.)
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

    // ---- rank within the warp, in original order ----
    // Lanes holding the same digit are found with one ballot per digit bit:
    // peers &= (bit ? ballot : ~ballot), written as ~(ballot ^ -bit) so that it
    // is one three-input logic operation.  In a warp whose items are not all
    // present, invalid lanes carry the digit R (bit RB), which keeps them apart;
    // a full warp (every warp of every tile but the last) skips that bit.
    uint16_t *wh = s_whist + wid * R;
    const uint32_t lt = lanemask_lt();
    auto rank_items = [&](auto full_tag) {
        constexpr bool FULL = decltype(full_tag)::value;
        constexpr int NB = FULL ? RB : RB + 1;
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const bool valid = FULL || 32 * k + lane < wcount;
            const uint32_t d = valid ? dig(k) : (uint32_t)R;
            uint32_t peers = 0xffffffffu;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const uint32_t bit = (d >> b) & 1u;
                const uint32_t bb = __ballot_sync(0xffffffffu, bit);
                peers &= ~(bb ^ (0u - bit));
            }
            const uint32_t pre = valid ? (uint32_t)wh[d] : 0u;
            const uint32_t lower = __popc(peers & lt);
            __syncwarp();
            if (valid && lower == 0) wh[d] = (uint16_t)(pre + __popc(peers));
            __syncwarp();
            rank[k] = pre + lower;
        }
    };
    if (wcount == 32 * kSortItems) rank_items(std::true_type{});
    else rank_items(std::false_type{});

    // ---- look back for the running totals, publish the inclusive prefix ----
    // Each thread walks back for its digits, kLookWindow words at a time
    // (their addresses do not depend on what is read), adding aggregates until
    // it meets an inclusive total; when the next word is not yet published it
    // polls that word alone, sleeping between polls.
    uint32_t btotal;
    uint32_t run = block_excl_scan_u32(tsum, &btotal);  // contains __syncthreads
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        int d = tid * PER + j;
        if (d >= R) continue;
        const uint32_t lstart = run;
        s_lstart[d] = lstart;
        run += cnt[j];
        uint32_t acc = 0;
        if (tile > 0) {
            int64_t t = (int64_t)tile - 1;
            int spins = 0;
            bool done = false;
            // test-only (values-only passes): tile 0 reads as unpublished
            const uint32_t stall = WRITE_KEYS ? 0u : stall_test(err, tile);
            while (!done && t >= 0) {
                uint32_t sv[kLookWindow];
#pragma unroll
                for (int w = 0; w < kLookWindow; ++w)
                    sv[w] = (t - w >= 0) ? (stall && t - w == 0 ? 0u : ld_relaxed(lookback + (size_t)(t - w) * R + d))
                                         : kFlagIncl;
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
                    const int limit = stall ? (int)min(stall, (uint32_t)kSpinLimit) : kSpinLimit;
                    while (((stall && t == 0 ? 0u : ld_relaxed(lookback + (size_t)t * R + d)) & ~kCountMask) == 0u) {
                        if (++spins > limit) break;
                        __nanosleep(ns);
                        ns = ns < 512 ? 2 * ns : 512;
                    }
                    if (spins > limit) {
                        atomicOr(err, kErrTimeout);
                        break;
                    }
                }
            }
            st_relaxed(lb + d, kFlagIncl | ((acc + cnt[j]) & kCountMask));
        }
        // output position of the tile's j-th key in block order: s_gbase[d] + j
        // (the digit's global base minus its start in the block; mod 2^32)
        s_gbase[d] = bin_off[d] + acc - lstart;
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

    const uint32_t tcount = min(n - tbase, (uint32_t)kSortTile);
    if constexpr (sizeof(KeyT) == 4) {
        // ---- (key, value) pairs to block order in shared memory, then out ----
        uint2 *s_pairs = reinterpret_cast<uint2 *>(smem);
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            if (32 * k + lane < wcount) {
                const uint32_t d = dig(k);
                s_pairs[s_lstart[d] + s_whist[wid * R + d] + rank[k]] = make_uint2((uint32_t)key[k], val(k));
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const uint32_t j = tid + k * kSortBlock;
            if (j < tcount) {
                const uint2 kv = s_pairs[j];
                const uint32_t d = (kv.x >> shift) & mask;
                const uint32_t dest = s_gbase[d] + j;
                if (dest < n) {  // dest >= n only after a look-back timeout
                    if (OUT == kOutPacked) {
                        kout[dest] = (KeyT)(((kv.x >> pack_shift) << vbits) | kv.y);
                    } else {
                        if (WRITE_KEYS) kout[dest] = (KeyT)kv.x;
                        vout[dest] = kv.y;
                    }
                }
            }
        }
    } else {
        // ---- keys: scatter to block order in shared memory, then out ----
        KeyT *s_keys = reinterpret_cast<KeyT *>(smem);
        uint32_t *s_vals = reinterpret_cast<uint32_t *>(smem);
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            if (32 * k + lane < wcount) {
                const uint32_t d = dig(k);
                const uint32_t lr = s_lstart[d] + s_whist[wid * R + d] + rank[k];
                s_keys[lr] = key[k];
                rank[k] = lr;
            }
        }
        __syncthreads();
        uint32_t dest[kSortItems];
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const uint32_t j = tid + k * kSortBlock;
            if (j < tcount) {
                const KeyT kk = s_keys[j];
                const uint32_t d = (uint32_t)(kk >> shift) & mask;
                dest[k] = s_gbase[d] + j;
                if (WRITE_KEYS && dest[k] < n) kout[dest[k]] = kk;
            }
        }
        __syncthreads();
        // ---- values through the same permutation ----
#pragma unroll
        for (int k = 0; k < kSortItems; ++k)
            if (32 * k + lane < wcount) s_vals[rank[k]] = val(k);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const uint32_t j = tid + k * kSortBlock;
            if (j < tcount && dest[k] < n) vout[dest[k]] = s_vals[j];
        }
    }
}

}  // namespace qb
