// qb_api.cu -- the extern "C" entry points of libquadbox (include/quadbox.h).
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "qb_kernels.cuh"

using namespace qb;

namespace {

thread_local std::string g_err;

qb_status fail(qb_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define QB_CUDA(call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(QB_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int tile_bits_for(int tiles) {
    int b = 0;
    while ((1ll << b) < (long long)tiles) ++b;
    return b;
}

bool make_layout(int n, int W, int H, uint64_t cap, Layout &L) {
    if (n < 0 || W <= 0 || H <= 0 || W > (1 << 15) || H > (1 << 15) || cap > (1ull << 30)) return false;
    const int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile;
    const int tiles = tx * ty;
    const int key_bits = kDepthBits + tile_bits_for(tiles);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t N = (size_t)n;
    L.xy = take(8 * N);
    L.shape = take(8 * N);
    L.conic_o = take(16 * N);
    L.rgbd = take(16 * N);
    L.box = take(16 * N);
    L.r3 = take(4 * N);
    L.meta = take(4 * N);
    L.counts = take(4 * N);
    L.offsets = take(4 * N);
    L.counts_e = take(4 * N);
    L.chunk_first = take(4 * chunk_table_size(cap));
    L.segs = take(64 * N);
    L.scan_part = take(8 * scan_partials_count(n));
    L.keys0 = take(8 * cap);
    L.keys1 = take(8 * cap);
    L.vals0 = take(4 * cap);
    L.vals1 = take(4 * cap);
    size_t sb = 0;
    for (int d = 8; d <= kMaxDigitBits; ++d) {
        size_t b = sort_scratch_bytes(cap, key_bits, d);
        if (b > sb) sb = b;
    }
    L.sort_scratch_bytes = sb;
    L.sort_scratch = take(sb);
    L.dkeys0 = take(4 * N);
    L.dkeys1 = take(4 * N);
    L.dvals0 = take(4 * N);
    L.dvals1 = take(4 * N);
    size_t db = 0;
    for (int d = 8; d <= kMaxDigitBits; ++d) {
        size_t b = sort_scratch_bytes(N, kDepthBits, d);
        if (b > db) db = b;
    }
    L.dsort_scratch = take(db);
    L.ranges = take(8 * (size_t)tiles);
    L.tile_counts = take(4 * ((size_t)tiles + 1));  // + the tile histogram's block counter
    L.tile_diff = take(4 * (size_t)(tx + 1) * (ty + 1));
    L.tile_single = take(4 * (size_t)tiles);
    L.order_cnt = take(4 * 2 * (size_t)kOrderBuckets);
    L.order_list = take(4 * 2 * (size_t)kOrderBuckets * tiles);
    L.tfinal = take(4 * (size_t)W * H);
    L.ncontrib = take(4 * (size_t)W * H);
    L.neval = take(4 * (size_t)W * H);
    L.gscreen = take(72 * N);
    L.state = take(256);
    L.total = off;
    return true;
}

template <typename T>
T *at(const qb_frame *f, size_t off) {
    return reinterpret_cast<T *>(static_cast<uint8_t *>(f->workspace) + off);
}

CamDev to_cam(const qb_camera &c) {
    CamDev d;
    for (int i = 0; i < 12; ++i) d.V[i] = c.viewmat[i];
    d.fx = c.fx;
    d.fy = c.fy;
    d.cx = c.cx;
    d.cy = c.cy;
    d.limx = 1.3f * c.tan_fovx;
    d.limy = 1.3f * c.tan_fovy;
    d.campos[0] = c.campos[0];
    d.campos[1] = c.campos[1];
    d.campos[2] = c.campos[2];
    d.znear = c.znear;
    d.W = c.width;
    d.H = c.height;
    return d;
}

// A single frame is a set of one camera.
TileSet frame_tileset(const qb_frame *f) {
    TileSet ts;
    std::memset(&ts, 0, sizeof(ts));
    ts.n_cams = 1;
    ts.total_tiles = (uint32_t)(f->tiles_x * f->tiles_y);
    ts.cam[0].W = f->width;
    ts.cam[0].H = f->height;
    ts.cam[0].tiles_x = f->tiles_x;
    ts.cam[0].tiles_y = f->tiles_y;
    ts.cam[0].tile_base = 0;
    ts.cam[0].pix_base = 0;
    return ts;
}

CamSet frame_camset(const qb_camera &c) {
    CamSet cs;
    std::memset(&cs, 0, sizeof(cs));
    cs.n_cams = 1;
    cs.cam[0] = to_cam(c);
    return cs;
}

qb_status check_frame(const qb_frame *f, Layout &L) {
    if (!f || !f->workspace) return fail(QB_ERR_INVALID_ARG, "frame is NULL or not initialised");
    if (!make_layout(f->n, f->width, f->height, f->pair_capacity, L))
        return fail(QB_ERR_INVALID_ARG, "frame has invalid sizes");
    return QB_OK;
}

qb_status check_scene(const qb_frame *f, const qb_scene *s) {
    if (!s) return fail(QB_ERR_INVALID_ARG, "scene is NULL");
    if (s->n != f->n) return fail(QB_ERR_INVALID_ARG, "scene.n (%d) != frame.n (%d)", s->n, f->n);
    if (s->sh_degree < 0 || s->sh_degree > 3) return fail(QB_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (s->n > 0 && (!s->means || !s->scales || !s->quats || !s->opacities || !s->sh))
        return fail(QB_ERR_INVALID_ARG, "scene has a NULL array");
    return QB_OK;
}

qb_status check_camera(const qb_frame *f, const qb_camera *c) {
    if (!c) return fail(QB_ERR_INVALID_ARG, "camera is NULL");
    if (c->width != f->width || c->height != f->height)
        return fail(QB_ERR_INVALID_ARG, "camera size %dx%d != frame size %dx%d", c->width, c->height, f->width,
                    f->height);
    if (!(c->fx > 0.f) || !(c->fy > 0.f) || !(c->tan_fovx > 0.f) || !(c->tan_fovy > 0.f))
        return fail(QB_ERR_INVALID_ARG, "camera focal lengths and fov tangents must be positive");
    return QB_OK;
}

}  // namespace

namespace qb {
void set_last_error(const char *msg) { g_err = msg; }
static std::atomic<uint64_t> g_launches{0};
static std::atomic<qb_launch_hook> g_hook{nullptr};
static std::atomic<void *> g_hook_user{nullptr};
void note_launch(const char *kernel, cudaStream_t s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    const qb_launch_hook h = g_hook.load(std::memory_order_acquire);
    if (h) h(kernel, (qb_stream_t)s, g_hook_user.load(std::memory_order_relaxed));
}

cudaError_t ensure_dyn_smem(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> set;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t &have = set[{func, dev}];
    if (bytes <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}
}  // namespace qb

extern "C" {

const char *qb_last_error(void) { return g_err.c_str(); }

const char *qb_version(void) { return "libquadbox 0.1 sm_103a"; }

uint64_t qb_kernel_launches(void) { return qb::g_launches.load(std::memory_order_relaxed); }

void qb_set_launch_hook(qb_launch_hook hook, void *user) {
    qb::g_hook_user.store(user, std::memory_order_relaxed);
    qb::g_hook.store(hook, std::memory_order_release);
}

size_t qb_frame_workspace_bytes(int32_t n, int32_t width, int32_t height, uint64_t pair_capacity) {
    Layout L;
    if (!make_layout(n, width, height, pair_capacity, L)) return 0;
    return L.total;
}

qb_status qb_frame_init(qb_frame *frame, int32_t n, int32_t width, int32_t height, uint64_t pair_capacity,
                        void *d_workspace, size_t workspace_bytes, qb_stream_t stream) {
    if (!frame) return fail(QB_ERR_INVALID_ARG, "frame is NULL");
    Layout L;
    if (!make_layout(n, width, height, pair_capacity, L))
        return fail(QB_ERR_INVALID_ARG, "invalid frame sizes n=%d %dx%d capacity=%llu", n, width, height,
                    (unsigned long long)pair_capacity);
    if (!d_workspace) return fail(QB_ERR_INVALID_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0)
        return fail(QB_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (workspace_bytes < L.total)
        return fail(QB_ERR_INVALID_ARG, "workspace too small: %zu < %zu", workspace_bytes, L.total);
    std::memset(frame, 0, sizeof(*frame));
    frame->n = n;
    frame->width = width;
    frame->height = height;
    frame->tiles_x = (width + kTile - 1) / kTile;
    frame->tiles_y = (height + kTile - 1) / kTile;
    frame->pair_capacity = pair_capacity;
    frame->workspace = d_workspace;
    frame->workspace_bytes = workspace_bytes;
    frame->key_bits = kDepthBits + tile_bits_for(frame->tiles_x * frame->tiles_y);
    frame->n_pairs = UINT64_MAX;
    frame->sort_digit_bits = 8;
    frame->render_batch = 128;
    frame->sort_mode = QB_SORT_DEPTH_FIRST;
    QB_CUDA(cudaMemsetAsync(at<uint8_t>(frame, L.state), 0, 256, (cudaStream_t)stream));
    return QB_OK;
}

qb_status qb_frame_arrays_get(const qb_frame *frame, qb_frame_arrays *out) {
    Layout L;
    qb_status st = check_frame(frame, L);
    if (st != QB_OK) return st;
    if (!out) return fail(QB_ERR_INVALID_ARG, "out is NULL");
    const bool alt = frame->sorted_in_alt != 0 && frame->stage >= 3;
    out->xy = at<float>(frame, L.xy);
    out->conic_o = at<float>(frame, L.conic_o);
    out->rgbd = at<float>(frame, L.rgbd);
    out->box = at<float>(frame, L.box);
    out->r3 = at<float>(frame, L.r3);
    out->meta = at<int32_t>(frame, L.meta);
    out->counts = at<uint32_t>(frame, L.counts);
    out->offsets = at<uint32_t>(frame, L.offsets);
    out->keys = at<uint64_t>(frame, alt ? L.keys1 : L.keys0);
    out->tile_keys = at<uint32_t>(frame, alt ? L.keys1 : L.keys0);
    out->vals = at<uint32_t>(frame, alt ? L.vals1 : L.vals0);
    out->depth_order = at<uint32_t>(frame, frame->depth_in_alt ? L.dvals1 : L.dvals0);
    out->ranges = at<uint32_t>(frame, L.ranges);
    out->t_final = at<float>(frame, L.tfinal);
    out->n_contrib = at<int32_t>(frame, L.ncontrib);
    out->n_eval = at<int32_t>(frame, L.neval);
    out->n_pairs = at<uint64_t>(frame, L.state);
    out->err_flags = at<uint32_t>(frame, L.state + 8);
    out->order_counts = at<uint32_t>(frame, L.order_cnt);
    out->order_lists = at<uint32_t>(frame, L.order_list);
    return QB_OK;
}

qb_status qb_frame_tile_keys(const qb_frame *frame, uint32_t *d_out, uint64_t n_out, qb_stream_t stream) {
    Layout L;
    qb_status st = check_frame(frame, L);
    if (st != QB_OK) return st;
    if (frame->stage < 3) return fail(QB_ERR_STATE, "qb_frame_tile_keys before qb_sort");
    if (!d_out && n_out > 0) return fail(QB_ERR_INVALID_ARG, "output pointer is NULL");
    QB_CUDA(launch_expand_ranges(at<uint2>(frame, L.ranges), frame->tiles_x * frame->tiles_y, d_out, n_out,
                                 (cudaStream_t)stream));
    return QB_OK;
}

qb_status qb_frame_check(qb_frame *frame, qb_stream_t stream) {
    Layout L;
    qb_status st = check_frame(frame, L);
    if (st != QB_OK) return st;
    uint32_t flags = 0;
    QB_CUDA(cudaMemcpyAsync(&flags, at<uint32_t>(frame, L.state + 8), 4, cudaMemcpyDeviceToHost,
                            (cudaStream_t)stream));
    QB_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (flags) QB_CUDA(cudaMemsetAsync(at<uint32_t>(frame, L.state + 8), 0, 4, (cudaStream_t)stream));
    if (flags & kErrCapacity) return fail(QB_ERR_CAPACITY, "pair capacity exceeded on the device");
    if (flags & kErrTimeout) return fail(QB_ERR_TIMEOUT, "a device spin-wait reached its iteration limit");
    return QB_OK;
}

qb_status qb_preprocess(qb_frame *frame, const qb_scene *scene, const qb_camera *camera, int32_t mode,
                        qb_stream_t stream) {
    Layout L;
    qb_status st = check_frame(frame, L);
    if (st != QB_OK) return st;
    if ((st = check_scene(frame, scene)) != QB_OK) return st;
    if ((st = check_camera(frame, camera)) != QB_OK) return st;
    const int base_mode = mode & 0xff;
    if (base_mode < QB_BIN_AABB3S || base_mode > QB_BIN_DUALBOX || (mode & ~(0xff | QB_BIN_NO_CLAMP)))
        return fail(QB_ERR_INVALID_ARG, "invalid binning mode %d", mode);
    PreArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = scene->n;
    a.means = scene->means;
    a.scales = scene->scales;
    a.quats = scene->quats;
    a.opac = scene->opacities;
    a.sh = scene->sh;
    a.raw = scene->params_raw != 0;
    a.sh_vec4 = reinterpret_cast<uintptr_t>(scene->sh) % 16 == 0;
    a.quat_vec4 = reinterpret_cast<uintptr_t>(scene->quats) % 16 == 0;
    a.cams = frame_camset(*camera);
    a.mode = base_mode;
    a.clamp3s = (mode & QB_BIN_NO_CLAMP) == 0;
    a.xy = at<float2>(frame, L.xy);
    a.shape = at<float2>(frame, L.shape);
    a.conic_o = at<float4>(frame, L.conic_o);
    a.rgbd = at<float4>(frame, L.rgbd);
    a.box = at<float4>(frame, L.box);
    a.r3 = at<float>(frame, L.r3);
    a.meta = at<int>(frame, L.meta);
    a.counts = at<uint32_t>(frame, L.counts);
    a.tile_diff = nullptr;
    a.tile_single = nullptr;
    a.segs = at<uint4>(frame, L.segs);
    std::memset(a.diff_off, 0, sizeof(a.diff_off));
    std::memset(a.single_off, 0, sizeof(a.single_off));
    if (frame->sort_mode < QB_SORT_DEPTH_FIRST || frame->sort_mode > QB_SORT_FULL_KEY)
        return fail(QB_ERR_INVALID_ARG, "invalid sort_mode %d", frame->sort_mode);
    const int eff = frame->sort_mode;
    // the fused emit needs the per-tile counts before it runs: from the
    // preprocess's difference arrays (also when the grid is too large for the
    // histogram of the unfused path)
    const bool fused = eff == QB_SORT_DEPTH_FIRST &&
                       (frame->emit_fused != 0 || frame->tiles_x * frame->tiles_y > kTileCountMax);
    if (fused) {
        a.tile_diff = at<int>(frame, L.tile_diff);
        a.tile_single = at<int>(frame, L.tile_single);
        // the two count arrays are adjacent in the workspace: clear them together
        QB_CUDA(cudaMemsetAsync(a.tile_diff, 0, L.tile_single - L.tile_diff + 4 * (size_t)frame->tiles_x * frame->tiles_y,
                                (cudaStream_t)stream));
    }
    if (eff != QB_SORT_FULL_KEY) {  // the depth-order sort's keys, written by the preprocess
        a.depth_keys = at<uint32_t>(frame, L.dkeys0);
        a.depth_vals = at<uint32_t>(frame, L.dvals0);
    }
    QB_CUDA(launch_preprocess(a, scene->sh_degree, (cudaStream_t)stream));
    // requested sort | effective sort << 8 | fused emit << 16, as the counts were made for
    frame->reserved[0] = frame->sort_mode | (eff << 8) | ((fused ? 1 : 0) << 16);
    frame->bin_mode = mode;
    frame->sh_degree = scene->sh_degree;
    frame->stage = 1;
    frame->n_pairs = UINT64_MAX;
    return QB_OK;
}

qb_status qb_bin_emit(qb_frame *frame, uint64_t *n_pairs_out, qb_stream_t stream) {
    Layout L;
    qb_status st = check_frame(frame, L);
    if (st != QB_OK) return st;
    if (frame->stage < 1) return fail(QB_ERR_STATE, "qb_bin_emit before qb_preprocess");
    if (frame->sort_mode < QB_SORT_DEPTH_FIRST || frame->sort_mode > QB_SORT_FULL_KEY)
        return fail(QB_ERR_INVALID_ARG, "invalid sort_mode %d", frame->sort_mode);
    if (frame->sort_mode != (frame->reserved[0] & 0xff))
        return fail(QB_ERR_STATE, "sort_mode changed between qb_preprocess and qb_bin_emit");
    const int eff = (frame->reserved[0] >> 8) & 0xff;
    const bool fused = (frame->reserved[0] >> 16) & 1;
    if (frame->sort_digit_bits < 8 || frame->sort_digit_bits > kMaxDigitBits)
        return fail(QB_ERR_INVALID_ARG, "sort_digit_bits must be 8..11");
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t *d_np = at<uint64_t>(frame, L.state);
    uint32_t *err = at<uint32_t>(frame, L.state + 8);
    const bool depth_first = eff != QB_SORT_FULL_KEY;  // Gaussians emitted in depth order
    const uint32_t *perm = nullptr;
    if (depth_first) {
        // emission order = Gaussians sorted by (depth, index)
        uint32_t *dk0 = at<uint32_t>(frame, L.dkeys0), *dk1 = at<uint32_t>(frame, L.dkeys1);
        uint32_t *dv0 = at<uint32_t>(frame, L.dvals0), *dv1 = at<uint32_t>(frame, L.dvals1);
        // (keys and indices in dk0 / dv0 from the preprocess)
        int passes = 0;
        if (frame->n > 0)
            QB_CUDA(sort_pairs(dk0, dv0, dk1, dv1, (uint64_t)frame->n, nullptr, kDepthBits, kDepthDigitBits,
                               at<void>(frame, L.dsort_scratch), err, s, &passes));
        frame->depth_in_alt = passes & 1;
        perm = frame->depth_in_alt ? dv1 : dv0;
    }
    QB_CUDA(launch_scan(at<uint32_t>(frame, L.counts), perm, frame->n, at<uint32_t>(frame, L.offsets),
                        at<uint64_t>(frame, L.scan_part), d_np, err, s, at<uint32_t>(frame, L.counts_e),
                        at<uint32_t>(frame, L.chunk_first), (uint32_t)chunk_table_size(frame->pair_capacity)));
    if (eff == QB_SORT_DEPTH_FIRST && fused) {
        // per-tile counts -> ranges and the tile sort's bucket offsets
        const int tile_bits = frame->key_bits - kDepthBits;
        const uint32_t zero_off[1] = {0u};
        QB_CUDA(launch_tile_prep(at<int>(frame, L.tile_diff), at<int>(frame, L.tile_single), frame_tileset(frame),
                                 zero_off, zero_off,
                                 at<uint2>(frame, L.ranges), sort_hist_table(at<void>(frame, L.sort_scratch)),
                                 sort_hist_stride(), frame->sort_digit_bits, tile_bits, frame->pair_capacity, s));
        frame->reserved[1] = frame->sort_digit_bits;  // digit width the offsets were made for
    }
    frame->n_pairs = UINT64_MAX;
    if (n_pairs_out) {
        uint64_t P = 0;
        QB_CUDA(cudaMemcpyAsync(&P, d_np, sizeof(P), cudaMemcpyDeviceToHost, s));
        QB_CUDA(cudaStreamSynchronize(s));
        *n_pairs_out = P;
        if (P > frame->pair_capacity) {
            frame->stage = 1;
            return fail(QB_ERR_CAPACITY, "%llu pairs exceed the capacity of %llu", (unsigned long long)P,
                        (unsigned long long)frame->pair_capacity);
        }
        frame->n_pairs = P;
    }
    EmitArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = frame->n;
    a.n_per_cam = frame->n > 0 ? frame->n : 1;
    a.ts = frame_tileset(frame);
    a.perm = perm;
    a.xy = at<float2>(frame, L.xy);
    a.box = at<float4>(frame, L.box);
    a.r3 = at<float>(frame, L.r3);
    a.meta = at<int>(frame, L.meta);
    a.rgbd = at<float4>(frame, L.rgbd);
    a.counts = at<uint32_t>(frame, L.counts);
    a.offsets = at<uint32_t>(frame, L.offsets);
    a.counts_e = at<uint32_t>(frame, L.counts_e);
    a.chunk_first = at<uint32_t>(frame, L.chunk_first);
    a.vals = at<uint32_t>(frame, L.vals0);
    a.n_pairs = d_np;
    a.n_pairs_host = frame->n_pairs;
    a.capacity = frame->pair_capacity;
    a.mode = frame->bin_mode & 0xff;
    a.clamp3s = (frame->bin_mode & QB_BIN_NO_CLAMP) == 0;
    a.err = err;
    a.segs = at<uint4>(frame, L.segs);
    if (depth_first) {
        // QPass emit in depth order; in the QPass modes it also performs the
        // tile sort's first digit pass (qb_sort runs the remaining ones)
        void *scratch = at<void>(frame, L.sort_scratch);
        const int rb = frame->sort_digit_bits;
        const int tile_bits = frame->key_bits - kDepthBits;
        const int passes = tile_bits > 0 ? (tile_bits + rb - 1) / rb : 0;
        uint32_t *kA = at<uint32_t>(frame, L.keys0), *vA = at<uint32_t>(frame, L.vals0);
        uint32_t *kB = at<uint32_t>(frame, L.keys1), *vB = at<uint32_t>(frame, L.vals1);
        if (fused && passes > 0 && a.mode != QB_BIN_QUADBOX_NAIVE) {
            const bool to_a = pass_writes_a(passes, 0);
            QB_CUDA(sort_clear(scratch, frame->pair_capacity, rb, 0, 1, s));
            QB_CUDA(launch_emit_sweep(a, pass_geo(tile_bits, rb).bits[0], passes > 1, to_a ? kA : kB, to_a ? vA : vB,
                                      sort_hist_table(scratch),
                                      sort_lookback(scratch, frame->pair_capacity, rb, 0), sort_counter(scratch, 0),
                                      s));
            frame->reserved[2] = 1;  // first pass left to qb_sort
        } else {
            // plain emit into the buffer the first pass reads (or the final one)
            const bool into_a = passes == 0 || !pass_writes_a(passes, 0);
            a.vals = into_a ? vA : vB;
            QB_CUDA(launch_emit<uint32_t>(a, into_a ? kA : kB, s));
            frame->reserved[2] = 0;
        }
        frame->reserved[1] = frame->sort_digit_bits;  // digit width the buffers were chosen for
    } else {
        QB_CUDA(launch_emit<uint64_t>(a, at<uint64_t>(frame, L.keys0), s));
    }
    frame->stage = 2;
    return QB_OK;
}

qb_status qb_sort(qb_frame *frame, qb_stream_t stream) {
    Layout L;
    qb_status st = check_frame(frame, L);
    if (st != QB_OK) return st;
    if (frame->stage < 2) return fail(QB_ERR_STATE, "qb_sort before qb_bin_emit");
    if (frame->sort_digit_bits < 8 || frame->sort_digit_bits > kMaxDigitBits)
        return fail(QB_ERR_INVALID_ARG, "sort_digit_bits must be 8..11");
    cudaStream_t s = (cudaStream_t)stream;
    const bool known = frame->n_pairs != UINT64_MAX;
    const uint64_t n_max = known ? frame->n_pairs : frame->pair_capacity;
    const uint64_t *n_dev = known ? nullptr : at<uint64_t>(frame, L.state);
    int passes = 0;
    const int ntiles = frame->tiles_x * frame->tiles_y;
    uint32_t *err = at<uint32_t>(frame, L.state + 8);
    const int eff = (frame->reserved[0] >> 8) & 0xff;
    const bool fused = (frame->reserved[0] >> 16) & 1;
    if (eff == QB_SORT_DEPTH_FIRST) {
        // pairs were emitted in depth order: a stable sort on the tile id alone
        // (bucket offsets and ranges came from the per-tile counts in qb_bin_emit)
        if (frame->sort_digit_bits != frame->reserved[1])
            return fail(QB_ERR_STATE, "sort_digit_bits changed between qb_bin_emit and qb_sort");
        const int tile_bits = frame->key_bits - kDepthBits;
        const int rb = frame->sort_digit_bits;
        passes = tile_bits > 0 ? (tile_bits + rb - 1) / rb : 0;
        if (!fused) {
            // per-tile counts from the emitted tile ids -> ranges and every
            // pass's bucket offsets
            const uint32_t *src = at<uint32_t>(frame, passes > 0 && pass_writes_a(passes, 0) ? L.keys1 : L.keys0);
            uint32_t *counts = at<uint32_t>(frame, L.tile_counts);
            QB_CUDA(launch_tile_count(src, n_max, n_dev, ntiles, counts, at<uint2>(frame, L.ranges),
                                      sort_hist_table(at<void>(frame, L.sort_scratch)), sort_hist_stride(), rb,
                                      tile_bits, s));
        }
        if (passes > 0)
            QB_CUDA(tile_sort_passes(at<uint32_t>(frame, L.keys0), at<uint32_t>(frame, L.vals0),
                                     at<uint32_t>(frame, L.keys1), at<uint32_t>(frame, L.vals1), frame->pair_capacity,
                                     n_max, n_dev, tile_bits, frame->reserved[2], rb, at<void>(frame, L.sort_scratch),
                                     err, s, (uint64_t)frame->n));
        frame->sorted_in_alt = 0;  // the values end in vals0; the tile of each is given by the ranges
        (void)ntiles;
    } else {
        QB_CUDA(sort_pairs(at<uint64_t>(frame, L.keys0), at<uint32_t>(frame, L.vals0), at<uint64_t>(frame, L.keys1),
                           at<uint32_t>(frame, L.vals1), n_max, n_dev, frame->key_bits, frame->sort_digit_bits,
                           at<void>(frame, L.sort_scratch), err, s, &passes));
        frame->sorted_in_alt = passes & 1;
        const uint64_t *sorted = at<uint64_t>(frame, frame->sorted_in_alt ? L.keys1 : L.keys0);
        QB_CUDA(launch_ranges<uint64_t>(sorted, n_max, n_dev, at<uint2>(frame, L.ranges), ntiles, s));
    }
    frame->stage = 3;
    return QB_OK;
}

static qb_status render_fwd_impl(qb_frame *frame, const float *bg, float *d_img, unsigned long long *counts,
                                 qb_stream_t stream) {
    Layout L;
    qb_status st = check_frame(frame, L);
    if (st != QB_OK) return st;
    if (frame->stage < 3) return fail(QB_ERR_STATE, "qb_render_fwd before qb_sort");
    if (!d_img) return fail(QB_ERR_INVALID_ARG, "image pointer is NULL");
    RenderArgs a;
    std::memset(&a, 0, sizeof(a));
    a.ranges = at<uint2>(frame, L.ranges);
    a.vals = at<uint32_t>(frame, frame->sorted_in_alt ? L.vals1 : L.vals0);
    a.xy = at<float2>(frame, L.xy);
    a.shape = at<float2>(frame, L.shape);
    a.conic_o = at<float4>(frame, L.conic_o);
    a.rgbd = at<float4>(frame, L.rgbd);
    a.ts = frame_tileset(frame);
    a.queue = nullptr;
    a.tiles_per_fetch = 1;
    a.blocks_per_sm = 0;
    for (int c = 0; c < 3; ++c) a.bg[c] = bg ? bg[c] : 0.f;
    a.img = d_img;
    a.tfinal = at<float>(frame, L.tfinal);
    a.ncontrib = at<int>(frame, L.ncontrib);
    a.neval = at<int>(frame, L.neval);
    a.counts = counts;
    // heaviest tiles first: every tile filed by a work estimate, then blocks
    // take the tiles in that order (the last blocks to start are short ones);
    // the render files every tile again by the backward's work
    const size_t ntiles = a.ts.total_tiles;
    uint32_t *cnt = at<uint32_t>(frame, L.order_cnt), *list = at<uint32_t>(frame, L.order_list);
    a.order = TileOrder{cnt, list};
    a.order_out = TileOrder{cnt + kOrderBuckets, list + (size_t)kOrderBuckets * ntiles};
    QB_CUDA(cudaMemsetAsync(cnt, 0, 4 * 2 * (size_t)kOrderBuckets, (cudaStream_t)stream));
    QB_CUDA(launch_tile_work(a, (cudaStream_t)stream));
    QB_CUDA(launch_render(a, frame->render_batch, (cudaStream_t)stream));
    frame->stage = 4;
    return QB_OK;
}

qb_status qb_render_fwd(qb_frame *frame, const float *bg, float *d_img, qb_stream_t stream) {
    return render_fwd_impl(frame, bg, d_img, nullptr, stream);
}

qb_status qb_render_fwd_counted(qb_frame *frame, const float *bg, float *d_img, uint64_t *d_counts,
                                qb_stream_t stream) {
    if (!d_counts) return fail(QB_ERR_INVALID_ARG, "counts pointer is NULL");
    if (reinterpret_cast<uintptr_t>(d_counts) % 8 != 0) return fail(QB_ERR_INVALID_ARG, "counts must be 8-byte aligned");
    return render_fwd_impl(frame, bg, d_img, reinterpret_cast<unsigned long long *>(d_counts), stream);
}

qb_status qb_render_bwd(qb_frame *frame, const qb_scene *scene, const qb_camera *camera, const float *bg,
                        const float *d_dL_dimg, qb_scene_grads *grads, double *d_grad_screen, qb_stream_t stream) {
    Layout L;
    qb_status st = check_frame(frame, L);
    if (st != QB_OK) return st;
    if (frame->stage < 4) return fail(QB_ERR_STATE, "qb_render_bwd before qb_render_fwd");
    if ((st = check_scene(frame, scene)) != QB_OK) return st;
    if ((st = check_camera(frame, camera)) != QB_OK) return st;
    if (scene->sh_degree != frame->sh_degree) return fail(QB_ERR_INVALID_ARG, "sh_degree differs from forward");
    if (!d_dL_dimg || !grads) return fail(QB_ERR_INVALID_ARG, "dL_dimg or grads is NULL");
    if (frame->n > 0 && (!grads->means || !grads->scales || !grads->quats || !grads->opacities || !grads->sh))
        return fail(QB_ERR_INVALID_ARG, "a gradient array is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    double *gscreen = d_grad_screen;
    if (!gscreen) {
        gscreen = at<double>(frame, L.gscreen);
        QB_CUDA(cudaMemsetAsync(gscreen, 0, 72 * (size_t)frame->n, s));
    }
    BwdArgs b;
    std::memset(&b, 0, sizeof(b));
    b.ranges = at<uint2>(frame, L.ranges);
    b.vals = at<uint32_t>(frame, frame->sorted_in_alt ? L.vals1 : L.vals0);
    b.xy = at<float2>(frame, L.xy);
    b.shape = at<float2>(frame, L.shape);
    b.conic_o = at<float4>(frame, L.conic_o);
    b.rgbd = at<float4>(frame, L.rgbd);
    b.ts = frame_tileset(frame);
    b.queue = nullptr;
    b.tiles_per_fetch = 1;
    b.blocks_per_sm = 0;
    for (int c = 0; c < 3; ++c) b.bg[c] = bg ? bg[c] : 0.f;
    b.dL_dimg = d_dL_dimg;
    b.tfinal = at<float>(frame, L.tfinal);
    b.ncontrib = at<int>(frame, L.ncontrib);
    b.g_screen = gscreen;
    // tiles by decreasing last-contributor count (the backward's work per
    // tile, filed by the forward render)
    b.order = TileOrder{at<uint32_t>(frame, L.order_cnt) + kOrderBuckets,
                        at<uint32_t>(frame, L.order_list) + (size_t)kOrderBuckets * b.ts.total_tiles};
    QB_CUDA(launch_render_bwd(b, s));
    PreBwdArgs p;
    std::memset(&p, 0, sizeof(p));
    p.n = scene->n;
    p.means = scene->means;
    p.scales = scene->scales;
    p.quats = scene->quats;
    p.opac = scene->opacities;
    p.sh = scene->sh;
    p.raw = scene->params_raw != 0;
    p.cams = frame_camset(*camera);
    p.meta = at<int>(frame, L.meta);
    p.g_screen = gscreen;
    p.gm = grads->means;
    p.gs = grads->scales;
    p.gq = grads->quats;
    p.go = grads->opacities;
    p.gsh = grads->sh;
    p.sh_vec4 = reinterpret_cast<uintptr_t>(scene->sh) % 16 == 0;
    p.gsh_vec4 = reinterpret_cast<uintptr_t>(grads->sh) % 16 == 0;
    QB_CUDA(launch_preprocess_bwd(p, scene->sh_degree, s));
    return QB_OK;
}

qb_status qb_l1_loss_grad(const float *d_img, const float *d_target, float *d_dL, uint64_t n, float scale,
                          double *d_loss, qb_stream_t stream) {
    if (n > 0 && (!d_img || !d_target || !d_dL)) return fail(QB_ERR_INVALID_ARG, "an array is NULL");
    QB_CUDA(launch_l1_grad(d_img, d_target, d_dL, n, scale, d_loss, (cudaStream_t)stream));
    return QB_OK;
}

qb_status qb_adam_step(float *d_param, const float *d_grad, float *d_m, float *d_v, uint64_t n, float lr, float beta1,
                       float beta2, float eps, int32_t step, qb_stream_t stream) {
    if (n > 0 && (!d_param || !d_grad || !d_m || !d_v)) return fail(QB_ERR_INVALID_ARG, "an array is NULL");
    if (step < 1) return fail(QB_ERR_INVALID_ARG, "step must be >= 1 (got %d)", step);
    if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return fail(QB_ERR_INVALID_ARG, "need 0 <= beta1, beta2 < 1 and eps > 0");
    QB_CUDA(launch_adam(d_param, d_grad, d_m, d_v, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream));
    return QB_OK;
}

size_t qb_sort_scratch_bytes(uint64_t n, int32_t end_bit, int32_t digit_bits) {
    if (n > (1ull << 30)) return 0;
    size_t b = sort_scratch_bytes(n, end_bit, digit_bits);
    return b ? b + 256 : 0;  // + the error word
}

qb_status qb_sort_pairs(uint64_t *d_keys, uint32_t *d_vals, uint64_t *d_keys_alt, uint32_t *d_vals_alt, uint64_t n,
                        int32_t end_bit, int32_t digit_bits, void *d_scratch, size_t scratch_bytes,
                        int32_t *result_in_alt, qb_stream_t stream) {
    if (n > (1ull << 30)) return fail(QB_ERR_INVALID_ARG, "n must be <= 2^30");
    if (digit_bits < 8 || digit_bits > kMaxDigitBits) return fail(QB_ERR_INVALID_ARG, "digit_bits must be 8..11");
    if (end_bit < 1 || end_bit > 64) return fail(QB_ERR_INVALID_ARG, "end_bit must be 1..64");
    if (!result_in_alt) return fail(QB_ERR_INVALID_ARG, "result_in_alt is NULL");
    size_t need = qb_sort_scratch_bytes(n, end_bit, digit_bits);
    if (need == 0) return fail(QB_ERR_INVALID_ARG, "unsupported sort configuration");
    if (n > 0 && (!d_keys || !d_vals || !d_keys_alt || !d_vals_alt || !d_scratch))
        return fail(QB_ERR_INVALID_ARG, "NULL buffer");
    if (scratch_bytes < need) return fail(QB_ERR_INVALID_ARG, "scratch too small: %zu < %zu", scratch_bytes, need);
    if (reinterpret_cast<uintptr_t>(d_scratch) % 256 != 0)
        return fail(QB_ERR_INVALID_ARG, "scratch must be 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t *base = static_cast<uint8_t *>(d_scratch);
    uint32_t *err = reinterpret_cast<uint32_t *>(base + need - 256);
    // the error word and the test-only word after it (qb_sweep.cuh) start at zero
    QB_CUDA(cudaMemsetAsync(err, 0, 8, s));
    int passes = 0;
    QB_CUDA(sort_pairs(d_keys, d_vals, d_keys_alt, d_vals_alt, n, nullptr, end_bit, digit_bits, d_scratch, err, s,
                       &passes));
    *result_in_alt = passes & 1;
    uint32_t flags = 0;
    QB_CUDA(cudaMemcpyAsync(&flags, err, 4, cudaMemcpyDeviceToHost, s));
    QB_CUDA(cudaStreamSynchronize(s));
    if (flags & kErrTimeout) return fail(QB_ERR_TIMEOUT, "sort look-back reached its iteration limit");
    return QB_OK;
}

}  // extern "C"
