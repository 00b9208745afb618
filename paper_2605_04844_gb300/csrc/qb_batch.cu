// qb_batch.cu -- many cameras of one scene rendered together (include/quadbox.h,
// qb_render_batch).  The cameras are taken in groups; for a group every stage
// of the rasteriser runs once over all of its (camera, Gaussian) records:
// preprocess (one grid row per camera), depth order of the records, scan,
// QPass emit with tile ids global over the group, a stable sort on those ids
// (per-pass digit histograms, every pass writing keys), the ranges from the
// sorted ids, and a persistent render that takes tiles of any of the group's
// cameras from one work queue.  (The group's ~10^5 tiles are too many for the
// shared-memory tile histogram of the single-frame path, and counting them
// from the preprocess by atomics on difference arrays cost more than the
// sort's own histograms and a ranges pass.)  Nothing synchronises the host, so a whole call can be
// captured in a CUDA graph.  The records, the sorted values, the ranges and
// the per-pixel state of every camera stay in the workspace for
// qb_render_batch_bwd.
#include <cstring>

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
};

bool make_geo(int n_cams, const int32_t *W, const int32_t *H, Geo &g) {
    if (n_cams < 1 || n_cams > QB_MAX_CAMERAS || !W || !H) return false;
    g.tile_base[0] = 0;
    g.pix_base[0] = 0;
    for (int k = 0; k < n_cams; ++k) {
        if (W[k] <= 0 || H[k] <= 0 || W[k] > (1 << 15) || H[k] > (1 << 15)) return false;
        g.tx[k] = (W[k] + kTile - 1) / kTile;
        g.ty[k] = (H[k] + kTile - 1) / kTile;
        g.tile_base[k + 1] = g.tile_base[k] + (uint64_t)g.tx[k] * g.ty[k];
        g.pix_base[k + 1] = g.pix_base[k] + (uint64_t)W[k] * H[k];
    }
    return true;
}

int bits_for(uint64_t v) {  // bits to hold values < v
    int b = 0;
    while ((1ull << b) < v) ++b;
    return b;
}

struct BLayout {
    size_t xy, conic_o, rgbd, box, r3, meta, counts;  // [n_cams * n]
    size_t slots;                                     // [n_groups][cap] sorted values
    size_t ranges;                                    // [total tiles]
    size_t tfinal, ncontrib, neval;                   // [total pixels]
    size_t keysA, keysB, valsT;                       // [cap] group scratch
    size_t offsets, segs, scan_part, dk0, dk1, dv0, dv1;  // [group * n]
    size_t dsort, sort, gscreen, queue, state;
    size_t total;
};

bool make_blayout(int n, int n_cams, int group, uint64_t cap, const Geo &g, BLayout &L) {
    if (n < 0 || group < 1 || group > QB_GROUP_MAX || cap > (1ull << 30)) return false;
    const int n_groups = (n_cams + group - 1) / group;
    const size_t recs = (size_t)n_cams * n, grecs = (size_t)group * n;
    int max_tile_bits = 1;
    for (int g0 = 0; g0 < n_cams; g0 += group) {
        const int g1 = g0 + group < n_cams ? g0 + group : n_cams;
        const int tb = bits_for(g.tile_base[g1] - g.tile_base[g0]);
        max_tile_bits = tb > max_tile_bits ? tb : max_tile_bits;
    }
    if ((size_t)group * n > (size_t)INT32_MAX) return false;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.xy = take(8 * recs);
    L.conic_o = take(16 * recs);
    L.rgbd = take(16 * recs);
    L.box = take(16 * recs);
    L.r3 = take(4 * recs);
    L.meta = take(4 * recs);
    L.counts = take(4 * recs);
    L.slots = take(4 * (size_t)n_groups * cap);
    L.ranges = take(8 * g.tile_base[n_cams]);
    L.tfinal = take(4 * g.pix_base[n_cams]);
    L.ncontrib = take(4 * g.pix_base[n_cams]);
    L.neval = take(4 * g.pix_base[n_cams]);
    L.keysA = take(4 * cap);
    L.keysB = take(4 * cap);
    L.valsT = take(4 * cap);
    L.offsets = take(4 * grecs);
    L.segs = take(64 * grecs);
    L.scan_part = take(8 * scan_partials_count((int)grecs));
    L.dk0 = take(4 * grecs);
    L.dk1 = take(4 * grecs);
    L.dv0 = take(4 * grecs);
    L.dv1 = take(4 * grecs);
    size_t db = 0, sb = 0;
    for (int d = 8; d <= kMaxDigitBits; ++d) {
        size_t b1 = sort_scratch_bytes(grecs, kDepthBits, d), b2 = sort_scratch_bytes(cap, max_tile_bits, d);
        db = b1 > db ? b1 : db;
        sb = b2 > sb ? b2 : sb;
    }
    L.dsort = take(db);
    L.sort = take(sb);
    L.gscreen = take(72 * grecs);
    L.queue = take(256);
    L.state = take(8 * (size_t)n_groups + 256);
    L.total = off;
    return true;
}

template <typename T>
T *bat(const qb_batch *b, size_t off) {
    return reinterpret_cast<T *>(static_cast<uint8_t *>(b->workspace) + off);
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

// Per-group views: camera set, tile set (tile ids local to the group, pixel
// bases global), count-array offsets.
struct GroupView {
    int k0, k1, ncam;
    uint64_t rec0;      // first record
    uint64_t tile0;     // first global tile
    uint32_t ntiles;
    int tile_bits;
    CamSet cs;
    TileSet ts;
};

void group_view(const qb_batch *b, const Geo &g, const qb_camera *cams, int gi, GroupView &v) {
    std::memset(&v, 0, sizeof(v));
    v.k0 = gi * b->group;
    v.k1 = v.k0 + b->group < b->n_cams ? v.k0 + b->group : b->n_cams;
    v.ncam = v.k1 - v.k0;
    v.rec0 = (uint64_t)v.k0 * b->n;
    v.tile0 = g.tile_base[v.k0];
    v.ntiles = (uint32_t)(g.tile_base[v.k1] - g.tile_base[v.k0]);
    v.tile_bits = bits_for(v.ntiles);
    v.cs.n_cams = v.ncam;
    v.ts.n_cams = v.ncam;
    v.ts.total_tiles = v.ntiles;
    for (int c = 0; c < v.ncam; ++c) {
        const int k = v.k0 + c;
        if (cams) v.cs.cam[c] = cam_dev(cams[k]);
        v.ts.cam[c].W = b->widths[k];
        v.ts.cam[c].H = b->heights[k];
        v.ts.cam[c].tiles_x = g.tx[k];
        v.ts.cam[c].tiles_y = g.ty[k];
        v.ts.cam[c].tile_base = (uint32_t)(g.tile_base[k] - v.tile0);
        v.ts.cam[c].pix_base = g.pix_base[k];
    }
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
    if (!make_geo(n_cams, widths, heights, g) || !make_blayout(n, n_cams, group, pair_capacity, g, L))
        return bfail(QB_ERR_INVALID_ARG, "invalid batch sizes");
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
    QB_BCUDA(cudaMemsetAsync(bat<uint8_t>(batch, L.state), 0, 8 * (size_t)batch->n_groups + 256,
                             (cudaStream_t)stream));
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
    uint64_t *npairs = bat<uint64_t>(b, L.state);
    uint32_t *err = reinterpret_cast<uint32_t *>(bat<uint8_t>(b, L.state) + 8 * (size_t)b->n_groups);
    for (int gi = 0; gi < b->n_groups; ++gi) {
        GroupView v;
        group_view(b, geo, cams, gi, v);
        const int nrec = v.ncam * n;
        // ---- preprocess over (camera, Gaussian) records ----
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
        a.conic_o = bat<float4>(b, L.conic_o) + v.rec0;
        a.rgbd = bat<float4>(b, L.rgbd) + v.rec0;
        a.box = bat<float4>(b, L.box) + v.rec0;
        a.r3 = bat<float>(b, L.r3) + v.rec0;
        a.meta = bat<int>(b, L.meta) + v.rec0;
        a.counts = bat<uint32_t>(b, L.counts) + v.rec0;
        a.segs = bat<uint4>(b, L.segs);
        uint32_t *dk0 = bat<uint32_t>(b, L.dk0), *dk1 = bat<uint32_t>(b, L.dk1);
        uint32_t *dv0 = bat<uint32_t>(b, L.dv0), *dv1 = bat<uint32_t>(b, L.dv1);
        a.depth_keys = dk0;  // the depth-order sort's keys, written by the preprocess
        a.depth_vals = dv0;
        QB_BCUDA(launch_preprocess(a, scene->sh_degree, s));
        // ---- depth order of the records, scan in that order ----
        int passes = 0;
        if (nrec > 0)
            QB_BCUDA(sort_pairs(dk0, dv0, dk1, dv1, (uint64_t)nrec, nullptr, kDepthBits, kDepthDigitBits, bat<void>(b, L.dsort),
                                err, s, &passes));
        const uint32_t *perm = (passes & 1) ? dv1 : dv0;
        QB_BCUDA(launch_scan(a.counts, perm, nrec, bat<uint32_t>(b, L.offsets), bat<uint64_t>(b, L.scan_part),
                             npairs + gi, err, s));
        // ---- QPass emit of (group tile id, record) pairs in depth order,
        // stable sort on the tile id (every pass writes keys and values), and
        // the ranges from the sorted tile ids.  The emit writes the buffer
        // pair from which the last pass lands in (keysA, this group's slot).
        const PassGeo tg = pass_geo(v.tile_bits, t.sort_digit_bits);
        const int tpasses = v.tile_bits > 0 ? tg.passes : 0;
        uint2 *ranges = bat<uint2>(b, L.ranges) + v.tile0;
        uint32_t *slot = bat<uint32_t>(b, L.slots) + (size_t)gi * b->pair_capacity;
        uint32_t *valsT = bat<uint32_t>(b, L.valsT);
        uint32_t *keysA = bat<uint32_t>(b, L.keysA), *keysB = bat<uint32_t>(b, L.keysB);
        void *sort_scratch = bat<void>(b, L.sort);
        const bool into_a = tpasses % 2 == 0;
        EmitArgs e;
        std::memset(&e, 0, sizeof(e));
        e.n = nrec;
        e.n_per_cam = n > 0 ? n : 1;
        e.perm = perm;
        e.xy = a.xy;
        e.box = a.box;
        e.r3 = a.r3;
        e.meta = a.meta;
        e.rgbd = a.rgbd;
        e.counts = a.counts;
        e.offsets = bat<uint32_t>(b, L.offsets);
        e.vals = into_a ? slot : valsT;
        e.n_pairs = npairs + gi;
        e.n_pairs_host = UINT64_MAX;
        e.capacity = b->pair_capacity;
        e.mode = base_mode;
        e.clamp3s = a.clamp3s;
        e.err = err;
        e.ts = v.ts;
        e.segs = bat<uint4>(b, L.segs);
        QB_BCUDA(launch_emit<uint32_t>(e, into_a ? keysA : keysB, s));
        if (tpasses > 0) {
            int done = 0;
            QB_BCUDA(sort_pairs(into_a ? keysA : keysB, into_a ? slot : valsT, into_a ? keysB : keysA,
                                into_a ? valsT : slot, b->pair_capacity, npairs + gi, v.tile_bits, t.sort_digit_bits,
                                sort_scratch, err, s, &done, false));
        }
        QB_BCUDA(launch_ranges<uint32_t>(keysA, b->pair_capacity, npairs + gi, ranges, (int)v.ts.total_tiles, s));
        // ---- persistent render over the group's tiles ----
        QB_BCUDA(cudaMemsetAsync(bat<uint32_t>(b, L.queue), 0, 4, s));
        RenderArgs r;
        std::memset(&r, 0, sizeof(r));
        r.ranges = ranges;
        r.vals = slot;
        r.xy = a.xy;
        r.conic_o = a.conic_o;
        r.rgbd = a.rgbd;
        for (int c = 0; c < 3; ++c) r.bg[c] = bg ? bg[c] : 0.f;
        r.img = d_images;
        r.tfinal = bat<float>(b, L.tfinal);
        r.ncontrib = bat<int>(b, L.ncontrib);
        r.neval = bat<int>(b, L.neval);
        r.ts = v.ts;
        r.queue = bat<uint32_t>(b, L.queue);
        r.tiles_per_fetch = t.tiles_per_fetch;
        r.blocks_per_sm = t.blocks_per_sm;
        QB_BCUDA(launch_render(r, t.render_batch, s));
    }
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
    for (int gi = 0; gi < b->n_groups; ++gi) {
        GroupView v;
        group_view(b, geo, cams, gi, v);
        const size_t nrec = (size_t)v.ncam * n;
        double *gscreen = bat<double>(b, L.gscreen);
        QB_BCUDA(cudaMemsetAsync(gscreen, 0, 72 * nrec, s));
        QB_BCUDA(cudaMemsetAsync(bat<uint32_t>(b, L.queue), 0, 4, s));
        BwdArgs r;
        std::memset(&r, 0, sizeof(r));
        r.ranges = bat<uint2>(b, L.ranges) + v.tile0;
        r.vals = bat<uint32_t>(b, L.slots) + (size_t)gi * b->pair_capacity;
        r.xy = bat<float2>(b, L.xy) + v.rec0;
        r.conic_o = bat<float4>(b, L.conic_o) + v.rec0;
        r.rgbd = bat<float4>(b, L.rgbd) + v.rec0;
        for (int c = 0; c < 3; ++c) r.bg[c] = bg ? bg[c] : 0.f;
        r.dL_dimg = d_dL_dimages;
        r.tfinal = bat<float>(b, L.tfinal);
        r.ncontrib = bat<int>(b, L.ncontrib);
        r.g_screen = gscreen;
        r.ts = v.ts;
        r.queue = bat<uint32_t>(b, L.queue);
        r.tiles_per_fetch = b->reserved[0] > 0 ? b->reserved[0] : 1;
        r.blocks_per_sm = b->reserved[1];
        QB_BCUDA(launch_render_bwd(r, s));
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
        p.g_screen = gscreen;
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
    QB_BCUDA(cudaMemcpyAsync(&flags, state + 8 * (size_t)b->n_groups, 4, cudaMemcpyDeviceToHost, s));
    if (pairs_out)
        QB_BCUDA(cudaMemcpyAsync(pairs_out, state, 8 * (size_t)b->n_groups, cudaMemcpyDeviceToHost, s));
    QB_BCUDA(cudaStreamSynchronize(s));
    if (flags) QB_BCUDA(cudaMemsetAsync(state + 8 * (size_t)b->n_groups, 0, 4, s));
    if (flags & kErrCapacity) return bfail(QB_ERR_CAPACITY, "a group's pairs exceeded the pair capacity");
    if (flags & kErrTimeout) return bfail(QB_ERR_TIMEOUT, "a device spin-wait reached its iteration limit");
    return QB_OK;
}

}  // extern "C"
