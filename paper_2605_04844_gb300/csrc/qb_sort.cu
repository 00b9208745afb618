// qb_sort.cu -- K4: stable LSD radix sort of (key, u32 value) pairs with a
// onesweep schedule (one kernel per digit pass, decoupled look-back across
// tiles of 4096 keys), the SortPairs stage of the rasteriser (Sec. 2).  The
// pass body lives in qb_sweep.cuh.
//
// Per sort: one upfront pass reads all keys and builds the digit histograms
// of every pass, and a tiny kernel turns them into exclusive bucket offsets
// (skipped when the caller already has them, as the depth-first tile sort
// does from its per-tile counts).  Each digit pass then reads and writes the
// pairs once.
#include <algorithm>

#include "qb_sweep.cuh"

namespace qb {

static inline int num_passes(int end_bit, int digit_bits) { return (end_bit + digit_bits - 1) / digit_bits; }

static inline uint64_t sort_tiles(uint64_t n) { return (n + kSortTile - 1) / kSortTile; }

size_t sort_scratch_bytes(uint64_t n, int end_bit, int digit_bits) {
    if (digit_bits < 8 || digit_bits > kMaxDigitBits || end_bit < 1 || end_bit > 64) return 0;
    int passes = num_passes(end_bit, digit_bits);
    if (passes > kMaxPasses) return 0;
    return align256(kSortHeader + (size_t)passes * sort_tiles(n) * ((size_t)1 << digit_bits) * 4);
}

uint32_t *sort_hist_table(void *scratch) { return static_cast<uint32_t *>(scratch); }
int sort_hist_stride() { return kHistStride; }

uint32_t *sort_lookback(void *scratch, uint64_t n_cap, int digit_bits, int pass) {
    return reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(scratch) + kSortHeader) +
           (size_t)pass * sort_tiles(n_cap) * ((size_t)1 << digit_bits);
}

uint32_t *sort_counter(void *scratch, int pass) {
    return reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(scratch) + kSortCounters) + pass;
}

cudaError_t sort_clear(void *scratch, uint64_t n_cap, int digit_bits, int first_pass, int end_pass,
                       cudaStream_t s) {
    if (end_pass <= first_pass) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(sort_counter(scratch, first_pass), 0, 4 * (size_t)(end_pass - first_pass), s);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(sort_lookback(scratch, n_cap, digit_bits, first_pass), 0,
                           (size_t)(end_pass - first_pass) * sort_tiles(n_cap) * ((size_t)1 << digit_bits) * 4,
                           s);
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

// One digit pass over pairs already in memory.
template <int RB, typename KeyT, bool WRITE_KEYS>
__global__ void __launch_bounds__(kSortBlock) onesweep_kernel(const KeyT *__restrict__ kin,
                                                              const uint32_t *__restrict__ vin,
                                                              KeyT *__restrict__ kout, uint32_t *__restrict__ vout,
                                                              uint64_t n_max, const uint64_t *n_dev,
                                                              const uint32_t *__restrict__ bin_off,
                                                              uint32_t *lookback, uint32_t *counter, int shift,
                                                              uint32_t *err) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t n = device_count(n_dev, n_max);
    const uint64_t tbase = (uint64_t)tile * kSortTile;
    if (tbase >= n) return;  // block-uniform

    // warp-striped load: item k of lane l at wbase + 32k + l
    const uint64_t wbase = tbase + (uint64_t)wid * (32 * kSortItems);
    KeyT key[kSortItems];
    uint32_t val[kSortItems];
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
    sweep_tile<RB, KeyT, WRITE_KEYS>(key, val, n, tbase, tile, bin_off, lookback, shift, err, kout, vout, smem);
}

template <int RB, typename KeyT, bool WRITE_KEYS>
static cudaError_t set_sweep_attrs() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(onesweep_kernel<RB, KeyT, WRITE_KEYS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_smem<RB, KeyT>());
    if (e == cudaSuccess) done = true;
    return e;
}

template <int RB, typename KeyT>
static cudaError_t launch_pass(const KeyT *kin, const uint32_t *vin, KeyT *kout, uint32_t *vout, uint64_t n_max,
                               const uint64_t *n_dev, const uint32_t *bin_off, uint32_t *lookback,
                               uint32_t *counter, int shift, uint32_t *err, bool write_keys, cudaStream_t s) {
    const unsigned grid = (unsigned)sort_tiles(n_max);
    cudaError_t e;
    if (write_keys) {
        if ((e = set_sweep_attrs<RB, KeyT, true>()) != cudaSuccess) return e;
        note_launch(), onesweep_kernel<RB, KeyT, true><<<grid, kSortBlock, sweep_smem<RB, KeyT>(), s>>>(
            kin, vin, kout, vout, n_max, n_dev, bin_off, lookback, counter, shift, err);
    } else {
        if ((e = set_sweep_attrs<RB, KeyT, false>()) != cudaSuccess) return e;
        note_launch(), onesweep_kernel<RB, KeyT, false><<<grid, kSortBlock, sweep_smem<RB, KeyT>(), s>>>(
            kin, vin, kout, vout, n_max, n_dev, bin_off, lookback, counter, shift, err);
    }
    return cudaGetLastError();
}

template <int RB, typename KeyT>
static cudaError_t sort_impl(KeyT *keys, uint32_t *vals, KeyT *keys_alt, uint32_t *vals_alt, uint64_t n_max,
                             const uint64_t *n_dev, int end_bit, void *scratch, uint32_t *err, cudaStream_t s,
                             int *passes_out, bool hist_ready) {
    constexpr int R = 1 << RB;
    const int passes = num_passes(end_bit, RB);
    uint32_t *hist = sort_hist_table(scratch);
    *passes_out = passes;
    cudaError_t e = cudaSuccess;
    if (!hist_ready) e = cudaMemsetAsync(hist, 0, kSortCounters, s);
    if (e == cudaSuccess) e = sort_clear(scratch, n_max, RB, 0, passes, s);
    if (e != cudaSuccess || n_max == 0) return e;

    if (!hist_ready) {
        static bool attrs = false;
        if (!attrs) {
            e = cudaFuncSetAttribute(sort_hist_kernel<RB, KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kMaxPasses * R * 4);
            if (e != cudaSuccess) return e;
            attrs = true;
        }
        uint64_t hblocks = std::min<uint64_t>((n_max + 255) / 256, 152 * 4);
        note_launch(), sort_hist_kernel<RB, KeyT><<<(unsigned)hblocks, 256, (size_t)passes * R * 4, s>>>(keys, n_max, n_dev,
                                                                                            passes, hist);
        note_launch(), sort_hist_scan_kernel<RB><<<passes, 1024, 0, s>>>(hist);
    }
    KeyT *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    for (int p = 0; p < passes; ++p) {
        e = launch_pass<RB, KeyT>(kin, vin, kout, vout, n_max, n_dev, hist + p * kHistStride,
                                  sort_lookback(scratch, n_max, RB, p), sort_counter(scratch, p), p * RB, err, true,
                                  s);
        if (e != cudaSuccess) return e;
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    return cudaSuccess;
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

// Passes [first_pass, passes) of the depth-first tile sort (bucket offsets
// already in the table).  Pass p writes buffer A when passes - 1 - p is even,
// else B, and reads the other one; the last pass writes values only, into A.
template <int RB>
static cudaError_t tile_passes_impl(uint32_t *kA, uint32_t *vA, uint32_t *kB, uint32_t *vB, uint64_t n_cap,
                                    uint64_t n_max, const uint64_t *n_dev, int passes, int first_pass,
                                    void *scratch, uint32_t *err, cudaStream_t s) {
    cudaError_t e = sort_clear(scratch, n_cap, RB, first_pass, passes, s);
    if (e != cudaSuccess || n_max == 0) return e;
    const uint32_t *hist = sort_hist_table(scratch);
    for (int p = first_pass; p < passes; ++p) {
        const bool to_a = ((passes - 1 - p) & 1) == 0;
        uint32_t *kout = to_a ? kA : kB, *vout = to_a ? vA : vB;
        const uint32_t *kin = to_a ? kB : kA, *vin = to_a ? vB : vA;
        e = launch_pass<RB, uint32_t>(kin, vin, kout, vout, n_max, n_dev, hist + p * kHistStride,
                                      sort_lookback(scratch, n_cap, RB, p), sort_counter(scratch, p), p * RB, err,
                                      p + 1 < passes, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t tile_sort_passes(uint32_t *kA, uint32_t *vA, uint32_t *kB, uint32_t *vB, uint64_t n_cap, uint64_t n_max,
                             const uint64_t *n_dev, int passes, int first_pass, int digit_bits, void *scratch,
                             uint32_t *err, cudaStream_t s) {
    switch (digit_bits) {
    case 8: return tile_passes_impl<8>(kA, vA, kB, vB, n_cap, n_max, n_dev, passes, first_pass, scratch, err, s);
    case 9: return tile_passes_impl<9>(kA, vA, kB, vB, n_cap, n_max, n_dev, passes, first_pass, scratch, err, s);
    case 10: return tile_passes_impl<10>(kA, vA, kB, vB, n_cap, n_max, n_dev, passes, first_pass, scratch, err, s);
    case 11: return tile_passes_impl<11>(kA, vA, kB, vB, n_cap, n_max, n_dev, passes, first_pass, scratch, err, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace qb
