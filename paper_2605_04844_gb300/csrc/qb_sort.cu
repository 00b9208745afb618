// qb_sort.cu -- K4: stable LSD radix sort of (key, u32 value) pairs with a
// onesweep schedule (one kernel per digit pass, decoupled look-back across
// tiles of 4096 keys), the SortPairs stage of the rasteriser (Sec. 2).  The
// pass body lives in qb_sweep.cuh.
//
// Per sort: one upfront pass reads all keys and builds the digit histograms
// of every pass, and a tiny kernel turns them into exclusive bucket offsets
// (skipped when the caller already has them, as the depth-first tile sort
// does from its per-tile counts).  Each digit pass then reads and writes the
// pairs once.  Pass widths are balanced (pass_geo): 13 bits at digits of 8
// bits are sorted as 7 + 6, so no pass carries buckets that are always empty.
#include <algorithm>

#include "qb_sweep.cuh"

namespace qb {

static inline uint64_t sort_tiles(uint64_t n) { return (n + kSortTile - 1) / kSortTile; }

size_t sort_scratch_bytes(uint64_t n, int end_bit, int digit_bits) {
    if (digit_bits < 8 || digit_bits > kMaxDigitBits || end_bit < 1 || end_bit > 64) return 0;
    const PassGeo g = pass_geo(end_bit, digit_bits);
    if (g.passes > kMaxPasses) return 0;
    return align256(kSortHeader + (size_t)g.passes * sort_tiles(n) * ((size_t)1 << digit_bits) * 4);
}

uint32_t *sort_hist_table(void *scratch) { return static_cast<uint32_t *>(scratch); }
int sort_hist_stride() { return kHistStride; }

// Look-back words of pass p: laid out for n_cap pairs and digits of at most
// digit_bits (a pass with fewer bits uses the start of each tile's row).
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

// Upfront histogram of every pass's digit (table stride kHistStride).
template <typename KeyT>
__global__ void __launch_bounds__(256) sort_hist_kernel(const KeyT *__restrict__ keys, uint64_t n_max,
                                                        const uint64_t *n_dev, PassGeo g, uint32_t *hist) {
    extern __shared__ uint32_t sh[];  // passes x 2^bits[p], packed
    int off[kMaxPasses], total = 0;
    for (int p = 0; p < g.passes; ++p) {
        off[p] = total;
        total += 1 << g.bits[p];
    }
    for (int j = threadIdx.x; j < total; j += blockDim.x) sh[j] = 0u;
    __syncthreads();
    const uint64_t n = device_count(n_dev, n_max);
    // Each thread takes 8 consecutive keys and adds a run of equal digits
    // once: keys in emission order repeat their high digits (the tiles of
    // one Gaussian), which would otherwise be conflicting shared atomics.
    constexpr int J = 8;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * J;
    for (uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * J; i0 < n; i0 += stride) {
        KeyT k[J];
        if (sizeof(KeyT) == 4 && i0 + J <= n && (reinterpret_cast<uintptr_t>(keys) & 15) == 0) {
            // two 16-byte loads (i0 is a multiple of 8; callers' buffers may be unaligned)
            const uint4 a = reinterpret_cast<const uint4 *>(keys + i0)[0];
            const uint4 b = reinterpret_cast<const uint4 *>(keys + i0)[1];
            k[0] = (KeyT)a.x, k[1] = (KeyT)a.y, k[2] = (KeyT)a.z, k[3] = (KeyT)a.w;
            k[4] = (KeyT)b.x, k[5] = (KeyT)b.y, k[6] = (KeyT)b.z, k[7] = (KeyT)b.w;
        } else {
#pragma unroll
            for (int j = 0; j < J; ++j) k[j] = i0 + j < n ? keys[i0 + j] : KeyT(0);
        }
        const int m = (int)(n - i0 < (uint64_t)J ? n - i0 : (uint64_t)J);
        for (int p = 0; p < g.passes; ++p) {
            const KeyT msk = (KeyT(1) << g.bits[p]) - 1;
            const int sh_p = g.shift[p];
            int run_d = (int)((k[0] >> sh_p) & msk);
            uint32_t run_c = 1;
#pragma unroll
            for (int j = 1; j < J; ++j) {
                if (j >= m) break;
                const int d = (int)((k[j] >> sh_p) & msk);
                if (d == run_d) {
                    ++run_c;
                } else {
                    atomicAdd(&sh[off[p] + run_d], run_c);
                    run_d = d;
                    run_c = 1;
                }
            }
            atomicAdd(&sh[off[p] + run_d], run_c);
        }
    }
    __syncthreads();
    for (int p = 0; p < g.passes; ++p)
        for (int d = threadIdx.x; d < (1 << g.bits[p]); d += blockDim.x) {
            const uint32_t v = sh[off[p] + d];
            if (v) atomicAdd(&hist[p * kHistStride + d], v);
        }
}

// Counts -> exclusive bucket offsets, one block per pass.
__global__ void __launch_bounds__(1024) sort_hist_scan_kernel(uint32_t *hist, PassGeo g) {
    const int R = 1 << g.bits[blockIdx.x];
    const int per = (R + 1023) / 1024;
    uint32_t *h = hist + blockIdx.x * kHistStride;
    uint32_t v[2], s = 0;  // R <= 2048
    for (int k = 0; k < 2; ++k) {
        const int idx = threadIdx.x * per + k;
        v[k] = (k < per && idx < R) ? h[idx] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t run = block_excl_scan_u32(s, &total);
    for (int k = 0; k < 2; ++k) {
        const int idx = threadIdx.x * per + k;
        if (k < per && idx < R) h[idx] = run;
        run += v[k];
    }
}

// One digit pass over pairs already in memory.  OUT: what it writes
// (SweepOut).  PACKED_IN: kin holds packed words (key bits above vbits, the
// value below) and vin is not read.
template <int RB, typename KeyT, int OUT, bool PACKED_IN>
__global__ void __launch_bounds__(kSortBlock, sizeof(KeyT) == 4 ? kSortBlocksPerSM : 3) onesweep_kernel(const KeyT *__restrict__ kin,
                                                              const uint32_t *__restrict__ vin,
                                                              KeyT *__restrict__ kout, uint32_t *__restrict__ vout,
                                                              uint64_t n_max, const uint64_t *n_dev,
                                                              const uint32_t *__restrict__ bin_off,
                                                              uint32_t *lookback, uint32_t *counter, int shift,
                                                              uint32_t mask, uint32_t *err, int pack_shift, int vbits) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t n = (uint32_t)device_count(n_dev, n_max);  // <= 2^30
    const uint32_t tbase = tile * kSortTile;
    if (tbase >= n) return;  // block-uniform

    // warp-striped load: item k of lane l at wbase + 32k + l; the values are
    // read only at the scatter, after the ranking
    const uint32_t wbase = tbase + (uint32_t)wid * (32 * kSortItems);
    KeyT key[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const uint32_t idx = wbase + 32 * k + lane;
        key[k] = idx < n ? __ldcs(kin + idx) : KeyT(0);
    }
    if constexpr (PACKED_IN) {
        const uint32_t vmask = (1u << vbits) - 1u;
        auto val = [&](int k) -> uint32_t { return (uint32_t)key[k] & vmask; };
        sweep_tile<RB, KeyT, OUT>(key, val, n, tbase, tile, bin_off, lookback, shift, mask, err, kout, vout, smem,
                                  pack_shift, vbits);
    } else {
        auto val = [&](int k) -> uint32_t { return __ldcs(vin + wbase + 32 * k + lane); };
        sweep_tile<RB, KeyT, OUT>(key, val, n, tbase, tile, bin_off, lookback, shift, mask, err, kout, vout, smem,
                                  pack_shift, vbits);
    }
}

template <int RB, typename KeyT, int OUT, bool PACKED_IN>
static cudaError_t launch_pass_t(const KeyT *kin, const uint32_t *vin, KeyT *kout, uint32_t *vout, uint64_t n_max,
                                 const uint64_t *n_dev, const uint32_t *bin_off, uint32_t *lookback,
                                 uint32_t *counter, int shift, uint32_t mask, uint32_t *err, int pack_shift, int vbits,
                                 const char *name, cudaStream_t s) {
    constexpr size_t smem = sweep_smem<RB, KeyT>();
    cudaError_t e = ensure_dyn_smem((const void *)onesweep_kernel<RB, KeyT, OUT, PACKED_IN>, smem);
    if (e != cudaSuccess) return e;
    note_launch(name, s),
        onesweep_kernel<RB, KeyT, OUT, PACKED_IN><<<(unsigned)sort_tiles(n_max), kSortBlock, smem, s>>>(
            kin, vin, kout, vout, n_max, n_dev, bin_off, lookback, counter, shift, mask, err, pack_shift, vbits);
    return cudaGetLastError();
}

// One pass on the digit bits [shift, shift + bits), bits <= 11, writing keys
// and values (write_keys) or values only.
template <typename KeyT>
static cudaError_t launch_pass(const KeyT *kin, const uint32_t *vin, KeyT *kout, uint32_t *vout, uint64_t n_max,
                               const uint64_t *n_dev, const uint32_t *bin_off, uint32_t *lookback,
                               uint32_t *counter, int shift, int bits, uint32_t *err, bool write_keys,
                               const char *name, cudaStream_t s) {
    const uint32_t mask = (1u << bits) - 1u;
#define QB_PASS_CASE(RB)                                                                                           \
    case RB:                                                                                                       \
        return write_keys ? launch_pass_t<RB, KeyT, kOutPairs, false>(kin, vin, kout, vout, n_max, n_dev, bin_off, \
                                                                      lookback, counter, shift, mask, err, 0, 0,   \
                                                                      name, s)                                     \
                          : launch_pass_t<RB, KeyT, kOutValues, false>(kin, vin, kout, vout, n_max, n_dev,        \
                                                                       bin_off, lookback, counter, shift, mask,    \
                                                                       err, 0, 0, name, s);
    switch (bits < 4 ? 4 : bits) {
        QB_PASS_CASE(4)
        QB_PASS_CASE(5)
        QB_PASS_CASE(6)
        QB_PASS_CASE(7)
        QB_PASS_CASE(8)
        QB_PASS_CASE(9)
        QB_PASS_CASE(10)
        QB_PASS_CASE(11)
    default: return cudaErrorInvalidValue;
    }
#undef QB_PASS_CASE
}

template <typename KeyT>
static cudaError_t sort_impl(KeyT *keys, uint32_t *vals, KeyT *keys_alt, uint32_t *vals_alt, uint64_t n_max,
                             const uint64_t *n_dev, int end_bit, int digit_bits, void *scratch, uint32_t *err,
                             cudaStream_t s, int *passes_out, bool hist_ready) {
    if (end_bit > (int)(8 * sizeof(KeyT)) || digit_bits < 8 || digit_bits > kMaxDigitBits) return cudaErrorInvalidValue;
    const PassGeo g = pass_geo(end_bit, digit_bits);
    if (g.passes > kMaxPasses) return cudaErrorInvalidValue;
    uint32_t *hist = sort_hist_table(scratch);
    *passes_out = g.passes;
    cudaError_t e = cudaSuccess;
    if (!hist_ready) e = cudaMemsetAsync(hist, 0, kSortCounters, s);
    if (e == cudaSuccess) e = sort_clear(scratch, n_max, digit_bits, 0, g.passes, s);
    if (e != cudaSuccess || n_max == 0) return e;

    if (!hist_ready) {
        e = ensure_dyn_smem((const void *)sort_hist_kernel<KeyT>, (size_t)kMaxPasses * kHistStride * 4);
        if (e != cudaSuccess) return e;
        size_t smem = 0;
        for (int p = 0; p < g.passes; ++p) smem += (size_t)4 << g.bits[p];
        uint64_t hblocks = std::min<uint64_t>((n_max + 8 * 256 - 1) / (8 * 256), 152 * 4);
        note_launch("sort_hist_kernel", s), sort_hist_kernel<KeyT><<<(unsigned)hblocks, 256, smem, s>>>(keys, n_max, n_dev, g, hist);
        note_launch("sort_hist_scan_kernel", s), sort_hist_scan_kernel<<<g.passes, 1024, 0, s>>>(hist, g);
    }
    KeyT *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    for (int p = 0; p < g.passes; ++p) {
        e = launch_pass<KeyT>(kin, vin, kout, vout, n_max, n_dev, hist + p * kHistStride,
                              sort_lookback(scratch, n_max, digit_bits, p), sort_counter(scratch, p), g.shift[p],
                              g.bits[p], err, true, "onesweep_kernel", s);
        if (e != cudaSuccess) return e;
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    return cudaSuccess;
}

cudaError_t sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint64_t n_max,
                       const uint64_t *n_dev, int end_bit, int digit_bits, void *scratch, uint32_t *err,
                       cudaStream_t s, int *passes_out) {
    return sort_impl(keys, vals, keys_alt, vals_alt, n_max, n_dev, end_bit, digit_bits, scratch, err, s, passes_out,
                     false);
}

cudaError_t sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, uint64_t n_max,
                       const uint64_t *n_dev, int end_bit, int digit_bits, void *scratch, uint32_t *err,
                       cudaStream_t s, int *passes_out, bool hist_ready) {
    return sort_impl(keys, vals, keys_alt, vals_alt, n_max, n_dev, end_bit, digit_bits, scratch, err, s, passes_out,
                     hist_ready);
}

// The two passes of a tile sort whose values fit beside the second digit in
// one word: the first pass writes (key >> shift1) << vbits | value, one 4-byte
// word instead of a key and a value, and the second reads that word alone
// (digit above vbits, value below), 20 bytes of traffic per pair over the two
// passes instead of 28.
template <int RB0, int RB1>
static cudaError_t packed_passes(const uint32_t *kA, const uint32_t *vA, uint32_t *kB, uint32_t *vOut,
                                 uint64_t n_cap, uint64_t n_max, const uint64_t *n_dev, const PassGeo &g,
                                 int digit_bits, void *scratch, uint32_t *err, cudaStream_t s) {
    const uint32_t *hist = sort_hist_table(scratch);
    const int vbits = 32 - RB1;
    cudaError_t e = launch_pass_t<RB0, uint32_t, kOutPacked, false>(
        kA, vA, kB, nullptr, n_max, n_dev, hist, sort_lookback(scratch, n_cap, digit_bits, 0), sort_counter(scratch, 0),
        g.shift[0], (1u << RB0) - 1u, err, g.shift[1], vbits, "tile_sort_pass", s);
    if (e != cudaSuccess) return e;
    return launch_pass_t<RB1, uint32_t, kOutValues, true>(
        kB, nullptr, nullptr, vOut, n_max, n_dev, hist + kHistStride, sort_lookback(scratch, n_cap, digit_bits, 1),
        sort_counter(scratch, 1), vbits, (1u << RB1) - 1u, err, 0, vbits, "tile_sort_pass_values", s);
}

// Passes [first_pass, passes) of the depth-first tile sort on bits
// [0, end_bit) (bucket offsets already in the table).  Pass p writes buffer A
// when passes - 1 - p is even, else B, and reads the other one; the last pass
// writes values only, into A.  Every value is below val_bound: a sort of two
// passes from the first whose values fit in 32 - (second digit's bits) bits
// takes the packed form (packed_passes; B's value buffer is then not used).
cudaError_t tile_sort_passes(uint32_t *kA, uint32_t *vA, uint32_t *kB, uint32_t *vB, uint64_t n_cap, uint64_t n_max,
                             const uint64_t *n_dev, int end_bit, int first_pass, int digit_bits, void *scratch,
                             uint32_t *err, cudaStream_t s, uint64_t val_bound) {
    const PassGeo g = pass_geo(end_bit, digit_bits);
    cudaError_t e = sort_clear(scratch, n_cap, digit_bits, first_pass, g.passes, s);
    if (e != cudaSuccess || n_max == 0) return e;
    if (first_pass == 0 && g.passes == 2 && val_bound <= (1ull << (32 - g.bits[1]))) {
        // pass 0 reads A and writes B, pass 1 reads B and writes A's values;
        // tile ids of 9 to 16 bits: first digits of 5 to 8 bits, the second
        // of the same width or one bit less
        const int b0 = g.bits[0], b1 = g.bits[1];
#define QB_PACKED_CASE(B0)                                                                                   \
    if (b0 == B0 && b1 == B0)                                                                                \
        return packed_passes<B0, B0>(kA, vA, kB, vA, n_cap, n_max, n_dev, g, digit_bits, scratch, err, s);  \
    if (b0 == B0 && b1 == B0 - 1)                                                                            \
        return packed_passes<B0, B0 - 1>(kA, vA, kB, vA, n_cap, n_max, n_dev, g, digit_bits, scratch, err, s);
        QB_PACKED_CASE(5)
        QB_PACKED_CASE(6)
        QB_PACKED_CASE(7)
        QB_PACKED_CASE(8)
#undef QB_PACKED_CASE
    }
    const uint32_t *hist = sort_hist_table(scratch);
    for (int p = first_pass; p < g.passes; ++p) {
        const bool to_a = pass_writes_a(g.passes, p);
        uint32_t *kout = to_a ? kA : kB, *vout = to_a ? vA : vB;
        const uint32_t *kin = to_a ? kB : kA, *vin = to_a ? vB : vA;
        e = launch_pass<uint32_t>(kin, vin, kout, vout, n_max, n_dev, hist + p * kHistStride,
                                  sort_lookback(scratch, n_cap, digit_bits, p), sort_counter(scratch, p), g.shift[p],
                                  g.bits[p], err, p + 1 < g.passes,
                                  p + 1 < g.passes ? "tile_sort_pass" : "tile_sort_pass_values", s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace qb
