// qb_batch.cu -- many cameras of one scene rendered together (include/quadbox.h,
// qb_render_batch).  The cameras are taken in groups for the preprocess: one
// launch projects the scene into every camera of a group (one grid row per
// camera), so the scene's parameters and SH coefficients are read once per
// group.  Each camera's pairs are then binned like a single frame -- depth
// order of its records, scan, QPass emit with camera-local tile ids, the
// shared-memory tile histogram (ranges and bucket offsets) and the two-pass
// tile sort -- into the camera's own slot of sorted values.  Last, one
// persistent render takes tiles of every camera of the batch from one global
// work queue, so cameras of uneven resolution balance across the whole GPU
// and no camera's tail leaves SMs idle before the next one starts.
//
// The per-camera geometry the render needs (tile and pixel bases, the slot of
// sorted values, the first record) is fixed when the batch is initialised and
// lives in a device table in the workspace.  Nothing synchronises the host,
// so a whole call can be captured in a CUDA graph.  The records, the sorted
// values, the ranges and the per-pixel state of every camera stay in the
// workspace for qb_render_batch_bwd, whose render backward is one persistent
// launch over all cameras' tiles as well.
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "qb_kernels.cuh"

using namespace qb;

namespace {

qb_status bfail(qb_status s, const char *msg) {
    set_last_error(msg);
    return s;
}

#define QB_BCUDA(call)                                                    \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return bfail(QB_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)

struct Geo {  // per-camera geometry of a batch
    int tx[QB_MAX_CAMERAS], ty[QB_MAX_CAMERAS];
    uint64_t tile_base[QB_MAX_CAMERAS + 1];
    uint64_t pix_base[QB_MAX_CAMERAS + 1];
    int max_tile_bits, max_tiles;
};

int bits_for(uint64_t v) {  // bits to hold values < v
    int b = 0;
    while ((1ull << b) < v) ++b;
    return b;
}

bool make_geo(int n_cams, const int32_t *W, const int32_t *H, Geo &g) {
    if (n_cams < 1 || n_cams > QB_MAX_CAMERAS || !W || !H) return false;
    g.tile_base[0] = 0;
    g.pix_base[0] = 0;
    g.max_tile_bits = 1;
    g.max_tiles = 1;
    for (int k = 0; k < n_cams; ++k) {
        if (W[k] <= 0 || H[k] <= 0 || W[k] > (1 << 15) || H[k] > (1 << 15)) return false;
        g.tx[k] = (W[k] + kTile - 1) / kTile;
        g.ty[k] = (H[k] + kTile - 1) / kTile;
        const int tiles = g.tx[k] * g.ty[k];
        if (tiles > kTileCountMax) return false;  // beyond the tile histogram's shared memory
        g.tile_base[k + 1] = g.tile_base[k] + (uint64_t)tiles;
        g.pix_base[k + 1] = g.pix_base[k] + (uint64_t)W[k] * H[k];
        g.max_tiles = tiles > g.max_tiles ? tiles : g.max_tiles;
        const int tb = bits_for((uint64_t)tiles);
        g.max_tile_bits = tb > g.max_tile_bits ? tb : g.max_tile_bits;
    }
    return g.tile_base[n_cams] < (1ull << 32);
}

// Cameras binned at the same time: each has its own scratch set and side
// stream (forked from the caller's stream after the group's preprocess and
// joined before the next one), so one camera's small, latency-bound kernels
// overlap another's.
constexpr int kBatchStreams = 4;  // 8 measured no faster on the 64-camera case

struct BLayout {
    size_t xy, shape, conic_o, rgbd, box, r3, meta, counts;  // [n_cams * n] records
    size_t cam_table;                                 // [n_cams] CamTile
    size_t slots;                                     // [n_cams][cap] sorted values per camera
    size_t ranges;                                    // [total tiles]
    size_t tfinal, ncontrib, neval;                   // [total pixels]
    size_t segs, dk0, dk1, dv0, dv1;                  // [group * n] group scratch
    // one camera's binning scratch, kBatchStreams sets set_stride bytes apart:
    size_t keysA, keysB, valsT;                       // [cap] pairs
    size_t offsets, counts_e, chunk_first, scan_part, dsort, sort, tile_counts;
    size_t set_stride;
    size_t gscreen;                                   // [n_cams * n][9]
    size_t queue, state;
    size_t total;
};

bool make_blayout(int n, int n_cams, int group, uint64_t cap, const Geo &g, BLayout &L) {
    if (n < 0 || group < 1 || group > QB_GROUP_MAX || cap > (1ull << 30)) return false;
    const size_t recs = (size_t)n_cams * n, grecs = (size_t)group * n;
    if (grecs > (size_t)INT32_MAX || recs >= (1ull << 32)) return false;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.xy = take(8 * recs);
    L.shape = take(8 * recs);
    L.conic_o = take(16 * recs);
    L.rgbd = take(16 * recs);
    L.box = take(16 * recs);
    L.r3 = take(4 * recs);
    L.meta = take(4 * recs);
    L.counts = take(4 * recs);
    L.cam_table = take(sizeof(CamTile) * (size_t)n_cams);
    L.slots = take(4 * (size_t)n_cams * cap);
    L.ranges = take(8 * g.tile_base[n_cams]);
    L.tfinal = take(4 * g.pix_base[n_cams]);
    L.ncontrib = take(4 * g.pix_base[n_cams]);
    L.neval = take(4 * g.pix_base[n_cams]);
    L.segs = take(64 * grecs);
    L.dk0 = take(4 * grecs);
    L.dk1 = take(4 * grecs);
    L.dv0 = take(4 * grecs);
    L.dv1 = take(4 * grecs);
    const size_t set0 = off;
    L.keysA = take(4 * cap);
    L.keysB = take(4 * cap);
    L.valsT = take(4 * cap);
    L.offsets = take(4 * (size_t)n);
    L.counts_e = take(4 * (size_t)n);
    L.chunk_first = take(4 * chunk_table_size(cap));
    L.scan_part = take(8 * scan_partials_count(n));
    size_t db = 0, sb = 0;
    for (int d = 8; d <= kMaxDigitBits; ++d) {
        const size_t b1 = sort_scratch_bytes((uint64_t)n, kDepthBits, d);
        const size_t b2 = sort_scratch_bytes(cap, g.max_tile_bits, d);
        db = b1 > db ? b1 : db;
        sb = b2 > sb ? b2 : sb;
    }
    L.dsort = take(db);
    L.sort = take(sb);
    L.tile_counts = take(4 * ((size_t)g.max_tiles + 1));
    L.set_stride = off - set0;
    off += (kBatchStreams - 1) * L.set_stride;  // the other sets
    L.gscreen = take(72 * recs);
    L.queue = take(256);
    L.state = take(8 * (size_t)n_cams + 256);
    L.total = off;
    return true;
}

// Side streams and events of a batch, keyed by its workspace, created by
// qb_batch_init and destroyed by qb_batch_release.
struct SideStreams {
    int device;
    cudaStream_t side[kBatchStreams];
    cudaEvent_t fork, join[kBatchStreams];
};
std::mutex g_side_mu;
std::map<const void *, SideStreams> g_side;

cudaError_t side_create(const void *ws, SideStreams &out) {
    std::lock_guard<std::mutex> lock(g_side_mu);
    auto it = g_side.find(ws);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (it != g_side.end() && it->second.device == dev) {
        out = it->second;
        return cudaSuccess;
    }
    SideStreams ss;
    std::memset(&ss, 0, sizeof(ss));
    ss.device = dev;
    for (int i = 0; i < kBatchStreams && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&ss.side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss.join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    g_side[ws] = ss;
    out = ss;
    return cudaSuccess;
}

bool side_find(const void *ws, SideStreams &out) {
    std::lock_guard<std::mutex> lock(g_side_mu);
    auto it = g_side.find(ws);
    if (it == g_side.end()) return false;
    out = it->second;
    return true;
}

template <typename T>
T *bat(const qb_batch *b, size_t off) {
    return reinterpret_cast<T *>(static_cast<uint8_t *>(b->workspace) + off);
}

uint32_t *err_word(const qb_batch *b, const BLayout &L) {
    return reinterpret_cast<uint32_t *>(bat<uint8_t>(b, L.state) + 8 * (size_t)b->n_cams);
}

CamDev cam_dev(const qb_camera &c) {
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

// Camera k's entry of the render's table: global tile and pixel bases, its
// slot of sorted values, and the first record of its group (the emitted
// values are record indices within the group).
CamTile cam_tile(const qb_batch *b, const Geo &g, int k) {
    CamTile t;
    std::memset(&t, 0, sizeof(t));
    t.W = b->widths[k];
    t.H = b->heights[k];
    t.tiles_x = g.tx[k];
    t.tiles_y = g.ty[k];
    t.tile_base = (uint32_t)g.tile_base[k];
    t.rec_base = (uint32_t)((size_t)(k - k % b->group) * b->n);
    t.pix_base = g.pix_base[k];
    t.vals_base = (uint64_t)k * b->pair_capacity;
    return t;
}

// A group of cameras: camera set for the preprocess, and a tile set whose
// cameras all start at tile 0 (each camera is binned on its own tiles).
struct GroupView {
    int k0, k1, ncam;
    uint64_t rec0;  // first record
    CamSet cs;
    TileSet ts;
};

void group_view(const qb_batch *b, const Geo &g, const qb_camera *cams, int gi, GroupView &v) {
    std::memset(&v, 0, sizeof(v));
    v.k0 = gi * b->group;
    v.k1 = v.k0 + b->group < b->n_cams ? v.k0 + b->group : b->n_cams;
    v.ncam = v.k1 - v.k0;
    v.rec0 = (uint64_t)v.k0 * b->n;
    v.cs.n_cams = v.ncam;
    v.ts.n_cams = v.ncam;
    for (int c = 0; c < v.ncam; ++c) {
        const int k = v.k0 + c;
        if (cams) v.cs.cam[c] = cam_dev(cams[k]);
        v.ts.cam[c].W = b->widths[k];
        v.ts.cam[c].H = b->heights[k];
        v.ts.cam[c].tiles_x = g.tx[k];
        v.ts.cam[c].tiles_y = g.ty[k];
        v.ts.cam[c].tile_base = 0;
        v.ts.cam[c].pix_base = g.pix_base[k];
        v.ts.total_tiles = v.ts.total_tiles > (uint32_t)(g.tx[k] * g.ty[k]) ? v.ts.total_tiles
                                                                           : (uint32_t)(g.tx[k] * g.ty[k]);
    }
}

// The whole batch as one tile set for the persistent render and backward
// (the cameras themselves come from the device table).
TileSet batch_tileset(const qb_batch *b, const Geo &g) {
    TileSet ts;
    std::memset(&ts, 0, sizeof(ts));
    ts.n_cams = b->n_cams;
    ts.total_tiles = (uint32_t)g.tile_base[b->n_cams];
    return ts;
}

qb_status check_batch(const qb_batch *b, Geo &g, BLayout &L) {
    if (!b || !b->workspace) return bfail(QB_ERR_INVALID_ARG, "batch is NULL or not initialised");
    if (!make_geo(b->n_cams, b->widths, b->heights, g) ||
        !make_blayout(b->n, b->n_cams, b->group, b->pair_capacity, g, L))
        return bfail(QB_ERR_INVALID_ARG, "batch has invalid sizes");
    return QB_OK;
}

qb_status check_batch_inputs(const qb_batch *b, const qb_scene *scene, const qb_camera *cams) {
    if (!scene || scene->n != b->n) return bfail(QB_ERR_INVALID_ARG, "scene is NULL or scene.n != batch.n");
    if (scene->sh_degree < 0 || scene->sh_degree > 3) return bfail(QB_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (scene->n > 0 && (!scene->means || !scene->scales || !scene->quats || !scene->opacities || !scene->sh))
        return bfail(QB_ERR_INVALID_ARG, "scene has a NULL array");
    if (!cams) return bfail(QB_ERR_INVALID_ARG, "cameras are NULL");
    for (int k = 0; k < b->n_cams; ++k) {
        if (cams[k].width != b->widths[k] || cams[k].height != b->heights[k])
            return bfail(QB_ERR_INVALID_ARG, "camera size differs from qb_batch_init");
        if (!(cams[k].fx > 0.f) || !(cams[k].fy > 0.f) || !(cams[k].tan_fovx > 0.f) || !(cams[k].tan_fovy > 0.f))
            return bfail(QB_ERR_INVALID_ARG, "camera focal lengths and fov tangents must be positive");
    }
    return QB_OK;
}

qb_tune tune_or_default(const qb_tune *t) {
    qb_tune d{2, 128, 8, 0};
    if (!t) return d;
    return *t;
}

}  // namespace

extern "C" {

size_t qb_batch_workspace_bytes(int32_t n, int32_t n_cams, const int32_t *widths, const int32_t *heights,
                                int32_t group, uint64_t pair_capacity) {
    Geo local;
    BLayout L;
    if (!make_geo(n_cams, widths, heights, local)) return 0;
    if (!make_blayout(n, n_cams, group, pair_capacity, local, L)) return 0;
    return L.total;
}

qb_status qb_batch_init(qb_batch *batch, int32_t n, int32_t n_cams, const int32_t *widths, const int32_t *heights,
                        int32_t group, uint64_t pair_capacity, void *d_workspace, size_t workspace_bytes,
                        qb_stream_t stream) {
    if (!batch) return bfail(QB_ERR_INVALID_ARG, "batch is NULL");
    Geo g;
    BLayout L;
    if (!make_geo(n_cams, widths, heights, g))
        return bfail(QB_ERR_INVALID_ARG, "invalid camera sizes (1..256 cameras of 1..32768 pixels a side, at most "
                                         "24576 tiles each)");
    if (!make_blayout(n, n_cams, group, pair_capacity, g, L)) return bfail(QB_ERR_INVALID_ARG, "invalid batch sizes");
    if (!d_workspace || reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0)
        return bfail(QB_ERR_INVALID_ARG, "workspace must be non-NULL and 256-byte aligned");
    if (workspace_bytes < L.total) return bfail(QB_ERR_INVALID_ARG, "workspace too small");
    std::memset(batch, 0, sizeof(*batch));
    batch->n = n;
    batch->n_cams = n_cams;
    batch->group = group;
    batch->n_groups = (n_cams + group - 1) / group;
    batch->pair_capacity = pair_capacity;
    batch->workspace = d_workspace;
    batch->workspace_bytes = workspace_bytes;
    for (int k = 0; k < n_cams; ++k) {
        batch->widths[k] = widths[k];
        batch->heights[k] = heights[k];
        batch->image_offset[k] = 3 * g.pix_base[k];
    }
    batch->total_floats = 3 * g.pix_base[n_cams];
    cudaStream_t s = (cudaStream_t)stream;
    QB_BCUDA(cudaMemsetAsync(bat<uint8_t>(batch, L.state), 0, 8 * (size_t)n_cams + 256, s));
    // the render's camera table: fixed by the cameras' sizes and the capacity
    std::vector<CamTile> table((size_t)n_cams);
    for (int k = 0; k < n_cams; ++k) table[(size_t)k] = cam_tile(batch, g, k);
    QB_BCUDA(cudaMemcpyAsync(bat<void>(batch, L.cam_table), table.data(), sizeof(CamTile) * table.size(),
                             cudaMemcpyHostToDevice, s));
    QB_BCUDA(cudaStreamSynchronize(s));  // the host table goes out of scope
    SideStreams ss;
    QB_BCUDA(side_create(d_workspace, ss));
    return QB_OK;
}

qb_status qb_batch_release(qb_batch *batch) {
    if (!batch || !batch->workspace) return bfail(QB_ERR_INVALID_ARG, "batch is NULL or not initialised");
    SideStreams ss;
    bool found;
    {
        std::lock_guard<std::mutex> lock(g_side_mu);
        auto it = g_side.find(batch->workspace);
        found = it != g_side.end();
        if (found) {
            ss = it->second;
            g_side.erase(it);
        }
    }
    if (found) {
        for (int i = 0; i < kBatchStreams; ++i) {
            QB_BCUDA(cudaStreamSynchronize(ss.side[i]));
            QB_BCUDA(cudaStreamDestroy(ss.side[i]));
            QB_BCUDA(cudaEventDestroy(ss.join[i]));
        }
        QB_BCUDA(cudaEventDestroy(ss.fork));
    }
    batch->workspace = nullptr;
    return QB_OK;
}

qb_status qb_render_batch(qb_batch *b, const qb_scene *scene, const qb_camera *cams, int32_t mode,
                          const qb_tune *tune_in, const float *bg, float *d_images, qb_stream_t stream) {
    Geo geo;
    BLayout L;
    qb_status st = check_batch(b, geo, L);
    if (st != QB_OK) return st;
    if ((st = check_batch_inputs(b, scene, cams)) != QB_OK) return st;
    if (!d_images) return bfail(QB_ERR_INVALID_ARG, "image buffer is NULL");
    const int base_mode = mode & 0xff;
    if (base_mode < QB_BIN_AABB3S || base_mode > QB_BIN_DUALBOX || (mode & ~(0xff | QB_BIN_NO_CLAMP)))
        return bfail(QB_ERR_INVALID_ARG, "invalid binning mode");
    const qb_tune t = tune_or_default(tune_in);
    if (t.sort_digit_bits < 8 || t.sort_digit_bits > kMaxDigitBits || t.tiles_per_fetch < 1 ||
        t.tiles_per_fetch > 8 || t.blocks_per_sm < 0)
        return bfail(QB_ERR_INVALID_ARG, "invalid tuning");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = b->n;
    const uint64_t cap = b->pair_capacity;
    const int rb = t.sort_digit_bits;
    uint64_t *npairs = bat<uint64_t>(b, L.state);
    uint32_t *err = err_word(b, L);
    SideStreams ss;
    const bool forked = side_find(b->workspace, ss);
    for (int gi = 0; gi < b->n_groups; ++gi) {
        GroupView v;
        group_view(b, geo, cams, gi, v);
        // ---- preprocess over the group's (camera, Gaussian) records ----
        PreArgs a;
        std::memset(&a, 0, sizeof(a));
        a.n = n;
        a.means = scene->means;
        a.scales = scene->scales;
        a.quats = scene->quats;
        a.opac = scene->opacities;
        a.sh = scene->sh;
        a.raw = scene->params_raw != 0;
        a.sh_vec4 = reinterpret_cast<uintptr_t>(scene->sh) % 16 == 0;
        a.quat_vec4 = reinterpret_cast<uintptr_t>(scene->quats) % 16 == 0;
        a.cams = v.cs;
        a.mode = base_mode;
        a.clamp3s = (mode & QB_BIN_NO_CLAMP) == 0;
        a.xy = bat<float2>(b, L.xy) + v.rec0;
        a.shape = bat<float2>(b, L.shape) + v.rec0;
        a.conic_o = bat<float4>(b, L.conic_o) + v.rec0;
        a.rgbd = bat<float4>(b, L.rgbd) + v.rec0;
        a.box = bat<float4>(b, L.box) + v.rec0;
        a.r3 = bat<float>(b, L.r3) + v.rec0;
        a.meta = bat<int>(b, L.meta) + v.rec0;
        a.counts = bat<uint32_t>(b, L.counts) + v.rec0;
        a.segs = bat<uint4>(b, L.segs);
        a.depth_keys = bat<uint32_t>(b, L.dk0);  // the depth-order sort's keys and record indices
        a.depth_vals = bat<uint32_t>(b, L.dv0);
        QB_BCUDA(launch_preprocess(a, scene->sh_degree, s));
        // ---- each camera binned like a frame, into its own slot; camera c on
        // side stream c % kBatchStreams with that stream's scratch set ----
        const int nside = forked ? (v.ncam < kBatchStreams ? v.ncam : kBatchStreams) : 0;
        if (nside > 0) {
            QB_BCUDA(cudaEventRecord(ss.fork, s));
            for (int i = 0; i < nside; ++i) QB_BCUDA(cudaStreamWaitEvent(ss.side[i], ss.fork, 0));
        }
        for (int c = 0; c < v.ncam; ++c) {
            const int k = v.k0 + c;
            const int set = nside > 0 ? c % nside : 0;
            const cudaStream_t cs = nside > 0 ? ss.side[set] : s;
            const size_t so = (size_t)set * L.set_stride;
            uint32_t *keysA = bat<uint32_t>(b, L.keysA + so), *keysB = bat<uint32_t>(b, L.keysB + so);
            uint32_t *valsT = bat<uint32_t>(b, L.valsT + so);
            void *sort_scratch = bat<void>(b, L.sort + so);
            const size_t r0 = (size_t)c * n;  // the camera's records within the group
            uint32_t *dk0 = bat<uint32_t>(b, L.dk0) + r0, *dk1 = bat<uint32_t>(b, L.dk1) + r0;
            uint32_t *dv0 = bat<uint32_t>(b, L.dv0) + r0, *dv1 = bat<uint32_t>(b, L.dv1) + r0;
            int passes = 0;
            if (n > 0)
                QB_BCUDA(sort_pairs(dk0, dv0, dk1, dv1, (uint64_t)n, nullptr, kDepthBits, kDepthDigitBits,
                                    bat<void>(b, L.dsort + so), err, cs, &passes));
            const uint32_t *perm = (passes & 1) ? dv1 : dv0;  // group record indices in depth order
            QB_BCUDA(launch_scan(a.counts, perm, n, bat<uint32_t>(b, L.offsets + so),
                                 bat<uint64_t>(b, L.scan_part + so), npairs + k, err, cs,
                                 bat<uint32_t>(b, L.counts_e + so), bat<uint32_t>(b, L.chunk_first + so),
                                 (uint32_t)chunk_table_size(cap)));
            const int ntiles = geo.tx[k] * geo.ty[k];
            const int tile_bits = bits_for((uint64_t)ntiles);
            const int tpasses = tile_bits > 0 ? (tile_bits + rb - 1) / rb : 0;
            uint32_t *slot = bat<uint32_t>(b, L.slots) + (size_t)k * cap;
            // plain emit into the buffer pair the first pass reads (or the final one)
            const bool into_a = tpasses == 0 || !pass_writes_a(tpasses, 0);
            EmitArgs e;
            std::memset(&e, 0, sizeof(e));
            e.n = n;
            e.n_per_cam = n > 0 ? n : 1;
            e.perm = perm;
            e.xy = a.xy;
            e.box = a.box;
            e.r3 = a.r3;
            e.meta = a.meta;
            e.rgbd = a.rgbd;
            e.counts = a.counts;
            e.offsets = bat<uint32_t>(b, L.offsets + so);
            e.counts_e = bat<uint32_t>(b, L.counts_e + so);
            e.chunk_first = bat<uint32_t>(b, L.chunk_first + so);
            e.segs = bat<uint4>(b, L.segs);
            e.vals = into_a ? slot : valsT;
            e.n_pairs = npairs + k;
            e.n_pairs_host = UINT64_MAX;
            e.capacity = cap;
            e.mode = base_mode;
            e.clamp3s = a.clamp3s;
            e.err = err;
            e.ts = v.ts;
            QB_BCUDA(launch_emit<uint32_t>(e, into_a ? keysA : keysB, cs));
            // per-tile counts -> the camera's ranges and every pass's bucket
            // offsets; then the tile sort, whose last pass writes the slot
            uint2 *ranges = bat<uint2>(b, L.ranges) + geo.tile_base[k];
            QB_BCUDA(launch_tile_count(into_a ? keysA : keysB, cap, npairs + k, ntiles,
                                       bat<uint32_t>(b, L.tile_counts + so), ranges, sort_hist_table(sort_scratch),
                                       sort_hist_stride(), rb, tile_bits, cs));
            if (tpasses > 0)
                QB_BCUDA(tile_sort_passes(keysA, slot, keysB, valsT, cap, cap, npairs + k, tile_bits, 0, rb,
                                          sort_scratch, err, cs, (uint64_t)b->group * (uint64_t)b->n));
        }
        for (int i = 0; i < nside; ++i) {  // join before the next group's preprocess reuses the group scratch
            QB_BCUDA(cudaEventRecord(ss.join[i], ss.side[i]));
            QB_BCUDA(cudaStreamWaitEvent(s, ss.join[i], 0));
        }
    }
    // ---- one persistent render over every camera's tiles ----
    QB_BCUDA(cudaMemsetAsync(bat<uint32_t>(b, L.queue), 0, 4, s));
    RenderArgs r;
    std::memset(&r, 0, sizeof(r));
    r.ranges = bat<uint2>(b, L.ranges);
    r.vals = bat<uint32_t>(b, L.slots);
    r.xy = bat<float2>(b, L.xy);
    r.shape = bat<float2>(b, L.shape);
    r.conic_o = bat<float4>(b, L.conic_o);
    r.rgbd = bat<float4>(b, L.rgbd);
    for (int c = 0; c < 3; ++c) r.bg[c] = bg ? bg[c] : 0.f;
    r.img = d_images;
    r.tfinal = bat<float>(b, L.tfinal);
    r.ncontrib = bat<int>(b, L.ncontrib);
    r.neval = bat<int>(b, L.neval);
    r.ts = batch_tileset(b, geo);
    r.cam_table = bat<CamTile>(b, L.cam_table);
    r.queue = bat<uint32_t>(b, L.queue);
    r.tiles_per_fetch = t.tiles_per_fetch;
    r.blocks_per_sm = t.blocks_per_sm;
    QB_BCUDA(launch_render(r, t.render_batch, s));
    b->sh_degree = scene->sh_degree;
    b->bin_mode = mode;
    b->stage = 1;
    b->reserved[0] = t.tiles_per_fetch;
    b->reserved[1] = t.blocks_per_sm;
    return QB_OK;
}

qb_status qb_render_batch_bwd(qb_batch *b, const qb_scene *scene, const qb_camera *cams, const float *bg,
                              const float *d_dL_dimages, qb_scene_grads *grads, qb_stream_t stream) {
    Geo geo;
    BLayout L;
    qb_status st = check_batch(b, geo, L);
    if (st != QB_OK) return st;
    if ((st = check_batch_inputs(b, scene, cams)) != QB_OK) return st;
    if (b->stage < 1) return bfail(QB_ERR_STATE, "qb_render_batch_bwd before qb_render_batch");
    if (scene->sh_degree != b->sh_degree) return bfail(QB_ERR_INVALID_ARG, "sh_degree differs from the forward");
    if (!d_dL_dimages || !grads) return bfail(QB_ERR_INVALID_ARG, "dL_dimages or grads is NULL");
    if (b->n > 0 && (!grads->means || !grads->scales || !grads->quats || !grads->opacities || !grads->sh))
        return bfail(QB_ERR_INVALID_ARG, "a gradient array is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = b->n;
    // ---- one persistent render backward over every camera's tiles ----
    double *gscreen = bat<double>(b, L.gscreen);
    QB_BCUDA(cudaMemsetAsync(gscreen, 0, 72 * (size_t)b->n_cams * n, s));
    QB_BCUDA(cudaMemsetAsync(bat<uint32_t>(b, L.queue), 0, 4, s));
    BwdArgs r;
    std::memset(&r, 0, sizeof(r));
    r.ranges = bat<uint2>(b, L.ranges);
    r.vals = bat<uint32_t>(b, L.slots);
    r.xy = bat<float2>(b, L.xy);
    r.shape = bat<float2>(b, L.shape);
    r.conic_o = bat<float4>(b, L.conic_o);
    r.rgbd = bat<float4>(b, L.rgbd);
    for (int c = 0; c < 3; ++c) r.bg[c] = bg ? bg[c] : 0.f;
    r.dL_dimg = d_dL_dimages;
    r.tfinal = bat<float>(b, L.tfinal);
    r.ncontrib = bat<int>(b, L.ncontrib);
    r.g_screen = gscreen;
    r.ts = batch_tileset(b, geo);
    r.cam_table = bat<CamTile>(b, L.cam_table);
    r.queue = bat<uint32_t>(b, L.queue);
    r.tiles_per_fetch = b->reserved[0] > 0 ? b->reserved[0] : 1;
    r.blocks_per_sm = b->reserved[1];
    QB_BCUDA(launch_render_bwd(r, s));
    // ---- the chain to the scene parameters, one launch per group ----
    for (int gi = 0; gi < b->n_groups; ++gi) {
        GroupView v;
        group_view(b, geo, cams, gi, v);
        PreBwdArgs p;
        std::memset(&p, 0, sizeof(p));
        p.n = n;
        p.means = scene->means;
        p.scales = scene->scales;
        p.quats = scene->quats;
        p.opac = scene->opacities;
        p.sh = scene->sh;
        p.raw = scene->params_raw != 0;
        p.cams = v.cs;
        p.meta = bat<int>(b, L.meta) + v.rec0;
        p.g_screen = gscreen + 9 * v.rec0;
        p.gm = grads->means;
        p.gs = grads->scales;
        p.gq = grads->quats;
        p.go = grads->opacities;
        p.gsh = grads->sh;
        p.sh_vec4 = reinterpret_cast<uintptr_t>(scene->sh) % 16 == 0;
        p.gsh_vec4 = reinterpret_cast<uintptr_t>(grads->sh) % 16 == 0;
        QB_BCUDA(launch_preprocess_bwd(p, scene->sh_degree, s));
    }
    return QB_OK;
}

qb_status qb_batch_check(qb_batch *b, uint64_t *pairs_out, qb_stream_t stream) {
    Geo geo;
    BLayout L;
    qb_status st = check_batch(b, geo, L);
    if (st != QB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t flags = 0;
    uint8_t *state = bat<uint8_t>(b, L.state);
    QB_BCUDA(cudaMemcpyAsync(&flags, err_word(b, L), 4, cudaMemcpyDeviceToHost, s));
    if (pairs_out)
        QB_BCUDA(cudaMemcpyAsync(pairs_out, state, 8 * (size_t)b->n_cams, cudaMemcpyDeviceToHost, s));
    QB_BCUDA(cudaStreamSynchronize(s));
    if (flags) QB_BCUDA(cudaMemsetAsync(err_word(b, L), 0, 4, s));
    if (flags & kErrCapacity) return bfail(QB_ERR_CAPACITY, "a camera's pairs exceeded the pair capacity");
    if (flags & kErrTimeout) return bfail(QB_ERR_TIMEOUT, "a device spin-wait reached its iteration limit");
    return QB_OK;
}

}  // extern "C"
