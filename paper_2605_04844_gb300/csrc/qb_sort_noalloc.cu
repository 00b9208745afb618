// qb_sort_noalloc.cu -- a variant of the pair sort for callers that may not
// allocate device memory.
//
// Some callers cannot call cudaMalloc: a plug-in inside a host application
// whose allocator owns all device memory, a render loop that must not stall
// on an allocation (cudaMalloc can synchronise the device), or code that
// must keep its device footprint fixed after start-up.  For them the sort's
// scratch (digit histograms, look-back words, tile counters and the error
// word) lives in one file-scope __device__ array of fixed size instead of a
// caller-supplied buffer.  The array is part of the library image, so every
// GPU that loads the library holds it until the process exits.
#include <cstdio>

#include "qb_kernels.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB of sort scratch
constexpr size_t kNoAllocErrOffset = kNoAllocScratchBytes;  // then one 256-byte error block

__device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes + 256];

qb_status noalloc_fail(qb_status s, const char *msg) {
    qb::set_last_error(msg);
    return s;
}

// The array's device address on the current device.  In host code the
// symbol name is only a host-side stand-in, so the kernels must be given this
// address instead.  It is looked up on every call (a cheap query once the
// module is loaded), so nothing stale survives a cudaDeviceReset.
cudaError_t noalloc_scratch(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" {

size_t qb_sort_pairs_noalloc_max_scratch(void) { return kNoAllocScratchBytes; }

qb_status qb_sort_pairs_noalloc(uint64_t *d_keys, uint32_t *d_vals, uint64_t *d_keys_alt, uint32_t *d_vals_alt,
                                uint64_t n, int32_t end_bit, int32_t digit_bits, int32_t *result_in_alt,
                                qb_stream_t stream) {
    if (n > (1ull << 30)) return noalloc_fail(QB_ERR_INVALID_ARG, "n must be <= 2^30");
    if (digit_bits < 8 || digit_bits > qb::kMaxDigitBits)
        return noalloc_fail(QB_ERR_INVALID_ARG, "digit_bits must be 8..11");
    if (end_bit < 1 || end_bit > 64) return noalloc_fail(QB_ERR_INVALID_ARG, "end_bit must be 1..64");
    if (!result_in_alt) return noalloc_fail(QB_ERR_INVALID_ARG, "result_in_alt is NULL");
    if (n > 0 && (!d_keys || !d_vals || !d_keys_alt || !d_vals_alt))
        return noalloc_fail(QB_ERR_INVALID_ARG, "NULL buffer");
    const size_t need = qb::sort_scratch_bytes(n, end_bit, digit_bits);
    if (need == 0) return noalloc_fail(QB_ERR_INVALID_ARG, "unsupported sort configuration");
    if (need > kNoAllocScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "sort of %llu pairs on %d bits with %d-bit digits needs %zu bytes of scratch, more than the "
                 "%zu bytes of the static scratch array; use qb_sort_pairs with a caller-owned buffer",
                 (unsigned long long)n, end_bit, digit_bits, need, kNoAllocScratchBytes);
        return noalloc_fail(QB_ERR_INVALID_ARG, msg);
    }
    void *base = nullptr;
    cudaError_t e = noalloc_scratch(&base);
    if (e != cudaSuccess) return noalloc_fail(QB_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *err = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(base) + kNoAllocErrOffset);
    // the array keeps the previous call's contents: the error word and the
    // test-only word after it are cleared here, and sort_pairs clears the
    // histograms, counters and look-back words
    e = cudaMemsetAsync(err, 0, 8, s);
    if (e != cudaSuccess) return noalloc_fail(QB_ERR_CUDA, cudaGetErrorString(e));
    int passes = 0;
    e = qb::sort_pairs(d_keys, d_vals, d_keys_alt, d_vals_alt, n, nullptr, end_bit, digit_bits, base, err, s,
                       &passes);
    if (e != cudaSuccess) return noalloc_fail(QB_ERR_CUDA, cudaGetErrorString(e));
    *result_in_alt = passes & 1;
    uint32_t flags = 0;
    e = cudaMemcpyAsync(&flags, err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(QB_ERR_CUDA, cudaGetErrorString(e));
    if (flags & qb::kErrTimeout) return noalloc_fail(QB_ERR_TIMEOUT, "sort look-back reached its iteration limit");
    return QB_OK;
}

}  // extern "C"
