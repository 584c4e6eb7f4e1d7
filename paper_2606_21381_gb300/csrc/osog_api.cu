// C ABI of libosog: plans, argument checks, workspace layout, launch
// sequencing, CUDA-graph cache of the batched path, per-kernel timing.
#include <math.h>
#include <string.h>

#include <mutex>
#include <string>
#include <algorithm>
#include <vector>

#include "osog_fft.cuh"
#include "osog_kernels.h"

using namespace osog;

struct osog_plan {
    int H = 0, W = 0;
    Geometry geo{};
    float2 *tw_w = nullptr;   // twiddle tables of the W-point transform (W entries)
    float2 *tw_h = nullptr;   // twiddle tables of the H-point transform (H entries)
    int32_t *status = nullptr;
    int32_t *status_host = nullptr;  // pinned
    int64_t launches = 0;
    // per-kernel timing
    bool prof = false;
    std::vector<cudaEvent_t> ev;  // pairs (start, stop)
    std::vector<int> ev_cls;
    int ev_used = 0;
    int32_t prof_launches[OSOG_KERNEL_CLASS_COUNT] = {};
    // autotuned choices per batch shape (scenes, particles, modalities)
    struct Tuned {
        int S;
        int64_t n;
        int K;
        int ppp, persistent, band_rows, raster;
    };
    std::vector<Tuned> tuned;
    // cached graph of the last batched launch sequence
    cudaGraphExec_t gexec = nullptr;
    std::vector<unsigned char> gkey;
    int64_t graph_kernels = 0;
    // forward states left by osog_render_keep, by workspace
    struct Kept {
        void *ws;
        size_t ws_bytes;
        const float *soa;
        int64_t ld;
        int32_t n;
        osog_optics_t optics;
    };
    std::vector<Kept> kept;
    std::mutex kept_lock;  // autograd may run the adjoint on a thread of its own
    // device array of the four differentiable optics scalars, or null
    const float *optics_dyn = nullptr;
    // particle-band pairs reserved per particle by single-scene calls and by
    // the workspace queries (osog_plan_set_pairs_per_particle)
    int ppp = 8;
};

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    return fail(OSOG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool pow2_in_range(int v) { return v >= 32 && v <= 2048 && (v & (v - 1)) == 0; }

int popcount3(uint32_t m) { return (int)(m & 1u) + (int)((m >> 1) & 1u) + (int)((m >> 2) & 1u); }

constexpr int kDefaultPairs = 8;
constexpr int kMaxTimed = 8192;
constexpr size_t kMaxKept = 64;  // forward states remembered per plan

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Layout {
    size_t rec, rrec, rect, cnt, band_off, pairs, pair_rect, G, Q, colrange, ctr, total;
};

// Workspace regions for a launch group of up to S scenes, n records,
// nchunks binning chunks and pair_total band slots.
Layout make_layout(const Geometry &geo, int64_t n, int64_t nchunks, int S, int K,
                   int64_t pair_total) {
    Layout l;
    size_t o = 0;
    l.rec = o;
    o = align256(o + (size_t)n * sizeof(PRec));
    l.rrec = o;
    o = align256(o + (size_t)n * sizeof(RRec));
    l.rect = o;
    o = align256(o + (size_t)n * sizeof(Rect));
    l.cnt = o;
    o = align256(o + (size_t)nchunks * geo.nbands * sizeof(int32_t));
    l.band_off = o;
    o = align256(o + (size_t)S * (geo.nbands + 1) * sizeof(int32_t));
    l.pairs = o;
    o = align256(o + (size_t)pair_total * sizeof(int32_t));
    l.pair_rect = o;
    o = align256(o + (size_t)pair_total * sizeof(Rect));
    l.G = o;
    o = align256(o + (size_t)S * geo.H * geo.W * sizeof(float2));
    l.Q = o;
    o = align256(o + (size_t)S * K * geo.H * geo.W * sizeof(float2));
    l.colrange = o;
    o = align256(o + (size_t)S * sizeof(int2));
    l.ctr = o;
    o = align256(o + (size_t)(2 + 2 * S) * sizeof(int32_t));
    l.total = o;
    return l;
}

Work carve(void *ws, const Layout &l, int32_t *status) {
    char *b = static_cast<char *>(ws);
    Work w;
    w.rec = reinterpret_cast<PRec *>(b + l.rec);
    w.rrec = reinterpret_cast<RRec *>(b + l.rrec);
    w.rect = reinterpret_cast<Rect *>(b + l.rect);
    w.cnt = reinterpret_cast<int32_t *>(b + l.cnt);
    w.band_off = reinterpret_cast<int32_t *>(b + l.band_off);
    w.pairs = reinterpret_cast<int32_t *>(b + l.pairs);
    w.pair_rect = reinterpret_cast<Rect *>(b + l.pair_rect);
    w.G = reinterpret_cast<float2 *>(b + l.G);
    w.Q = reinterpret_cast<float2 *>(b + l.Q);
    w.colrange = reinterpret_cast<int2 *>(b + l.colrange);
    w.slotmap = nullptr;
    w.slotmap_ppp = 0;
    w.status = status;
    return w;
}

bool finite_all(std::initializer_list<double> v) {
    for (double x : v)
        if (!isfinite(x)) return false;
    return true;
}

int check_optics(const osog_plan *p, const osog_optics_t *o) {
    if (!o) return fail(OSOG_ERR_INVALID_ARG, "optics is NULL");
    if (o->H != p->H || o->W != p->W)
        return fail(OSOG_ERR_INVALID_ARG, "optics H, W differ from the plan's");
    if (!finite_all({o->dx_um, o->lambda_um, o->NA, o->n_medium, o->defocus_um, o->oblique_frac,
                     o->oblique_angle, o->shear_px, o->shear_angle, o->bias_phase, o->bevel_slope}))
        return fail(OSOG_ERR_INVALID_ARG, "optics has a non-finite field");
    if (!(o->dx_um > 0) || !(o->lambda_um > 0) || !(o->NA > 0) || !(o->n_medium >= o->NA))
        return fail(OSOG_ERR_INVALID_ARG, "optics needs dx > 0, lambda > 0, 0 < NA <= n_medium");
    if (!(o->bevel_slope > 0)) return fail(OSOG_ERR_INVALID_ARG, "bevel_slope must be > 0");
    if (o->modes == 0 || (o->modes & ~7u)) return fail(OSOG_ERR_INVALID_ARG, "modes must be in 1..7");
    return OSOG_OK;
}

// Launch helper: optional event bracketing and the launch counter.
template <typename F>
int run_kernel(osog_plan *p, int cls, cudaStream_t st, F &&launch) {
    bool timed = false;
    if (p->prof) {
        p->prof_launches[cls]++;
        if (p->ev_used < kMaxTimed) {
            if ((size_t)(2 * p->ev_used + 2) > p->ev.size()) {
                cudaEvent_t a, b;
                if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
                    return fail(OSOG_ERR_CUDA, "cudaEventCreate failed");
                p->ev.push_back(a);
                p->ev.push_back(b);
                p->ev_cls.push_back(0);
            }
            cudaEventRecord(p->ev[2 * p->ev_used], st);
            timed = true;
        }
    }
    cudaError_t e = launch();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (timed) {
        cudaEventRecord(p->ev[2 * p->ev_used + 1], st);
        p->ev_cls[p->ev_used] = cls;
        p->ev_used++;
    }
    p->launches++;
    return OSOG_OK;
}

enum Stage { kFull, kOpdOnly, kFromMap, kBinOnly };

// The forward raster and row pass of a launch group: either the strip pass
// rasterises its own rows (the default), or (tiles) the tile raster writes
// every pixel's fixed-point phase and absorption words into the region of Q
// (the filtered spectra, unused until the column pass) and the strip pass
// forms the exit wave from them.  The words are the same either way.
int raster_and_strip(osog_plan *p, StripArgs &sa, cudaStream_t st, bool tiles = false) {
    if (!tiles)
        return run_kernel(p, OSOG_KERNEL_STRIP_FORWARD, st,
                          [&] { return launch_strip_forward(sa, kStripRender, st); });
    RasterArgs ra{};
    ra.geo = sa.geo;
    ra.w = sa.w;
    ra.P = reinterpret_cast<uint2 *>(sa.w.Q);
    ra.S = sa.S;
    ra.TW = raster_tile_cols(sa.geo);
    for (int s = 0; s < sa.S; ++s) ra.sc[s] = sa.sc[s];
    int rc = run_kernel(p, OSOG_KERNEL_RASTER, st, [&] { return launch_raster_tiles(ra, st); });
    if (rc) return rc;
    sa.phase = ra.P;
    return run_kernel(p, OSOG_KERNEL_STRIP_FORWARD, st,
                      [&] { return launch_strip_forward(sa, kStripFromPhase, st); });
}

// Per-call choices of the batched path (see osog_tuning_t).
struct GroupOpts {
    int ppp = kDefaultPairs;  // replaced by the plan's reservation
    bool persistent = false;
    int band_rows = 0;
    int wait_polls = 0;       // persistent launch: 0 = the default limit
    int wait_extra = 0;       // failure-detection test (osog_tuning_t.test_wait_extra)
    bool raster_tiles = false;  // the raster in a kernel of its own
    std::vector<int32_t> *band_off_out = nullptr;  // kBinOnly: host copy of band_off
    const float4 *planes = nullptr;                 // kind-2 particles (single scene)
    const int32_t *plane_off = nullptr;
    int32_t n_planes = 0;
};

// The plan's geometry with the binning band height replaced by band_rows
// (0 keeps it).  False if band_rows is not a multiple of the strip height
// that divides H into at most kMaxBands bands.
bool band_geometry(const Geometry &base, int band_rows, Geometry &g) {
    g = base;
    if (band_rows <= 0) return true;
    if (band_rows % base.R || base.H % band_rows || base.H / band_rows > kMaxBands) return false;
    g.BH = band_rows;
    g.nbands = base.H / band_rows;
    return true;
}

// One launch group: up to kMaxScenes scenes whose records start at soa.
int enqueue_group(osog_plan *p, const float *soa, int64_t ld, const int32_t *counts, int S,
                  const osog_optics_t *optics, int K, const GroupOpts &opt, void *ws,
                  size_t ws_bytes, float *images, const float *opd_att, float *opd_out,
                  Stage stage, cudaStream_t st) {
    Geometry geo;
    if (!band_geometry(p->geo, opt.band_rows, geo))
        return fail(OSOG_ERR_INVALID_ARG, "band_rows must be a multiple of the strip height "
                                          "dividing H into at most 64 bands");
    const int pairs_per_particle = opt.ppp;
    GroupDev gd{};
    gd.S = S;
    gd.K = K;
    int64_t n = 0, chunks = 0, pairs = 0;
    for (int s = 0; s < S; ++s) {
        SceneDev sc = scene_dev(optics[s]);
        sc.p0 = (int32_t)n;
        sc.n = counts[s];
        sc.chunk0 = (int32_t)chunks;
        sc.pair0 = (int32_t)pairs;
        sc.pair_cap = (int32_t)((int64_t)counts[s] * pairs_per_particle);
        gd.sc[s] = sc;
        n += counts[s];
        chunks += (counts[s] + kChunk - 1) / kChunk;
        pairs += (int64_t)counts[s] * pairs_per_particle;
        int k = 0;
        for (int bit = 0; bit < 3; ++bit)
            if (optics[s].modes & (1u << bit)) gd.md[s][k++] = mode_dev(optics[s], 1u << bit, p->optics_dyn);
    }
    if (pairs > INT32_MAX || n > INT32_MAX) return fail(OSOG_ERR_INVALID_ARG, "too many particles");
    gd.nchunks = (int32_t)chunks;
    const Layout l = make_layout(geo, n, chunks, S, stage == kFull || stage == kFromMap ? K : 0, pairs);
    if (l.total > ws_bytes) return fail(OSOG_ERR_WORKSPACE, "workspace too small");
    Work w = carve(ws, l, p->status);
    if (opt.planes) {  // the planes' pixel-affine bounds follow the regions above
        const size_t coef = align256(l.total);
        if (coef + (size_t)opt.n_planes * sizeof(float4) > ws_bytes)
            return fail(OSOG_ERR_WORKSPACE, "workspace too small for the planes");
        w.planes = opt.planes;
        w.plane_off = opt.plane_off;
        w.n_planes = opt.n_planes;
        w.plane_coef = reinterpret_cast<float4 *>(static_cast<char *>(ws) + coef);
    }
    int rc;
    if (stage != kFromMap && stage != kBinOnly && S == 1 && gd.nchunks == 1) {
        // one scene of one chunk: the three binning passes in one launch
        rc = run_kernel(p, OSOG_KERNEL_BIN_COUNT, st,
                        [&] { return launch_bin_single(soa, ld, gd, geo, w, st); });
        if (rc) return rc;
    } else {
        if (stage != kFromMap) {
            rc = run_kernel(p, OSOG_KERNEL_BIN_COUNT, st,
                            [&] { return launch_bin_count(soa, ld, gd, geo, w, st); });
            if (rc) return rc;
        }
        // The scan also bounds the columns that any pupil passes.
        rc = run_kernel(p, OSOG_KERNEL_BIN_SCAN, st, [&] { return launch_bin_scan(gd, geo, w, st); });
        if (rc) return rc;
        if (stage == kBinOnly) {  // autotuner dry run: the per-band pair totals only
            opt.band_off_out->resize((size_t)S * (geo.nbands + 1));
            cudaError_t e = cudaMemcpyAsync(opt.band_off_out->data(), w.band_off,
                                            sizeof(int32_t) * opt.band_off_out->size(),
                                            cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            return e == cudaSuccess ? OSOG_OK : cuda_fail(e, "autotune dry run");
        }
        if (stage != kFromMap) {
            rc = run_kernel(p, OSOG_KERNEL_BIN_FILL, st, [&] { return launch_bin_fill(gd, geo, w, st); });
            if (rc) return rc;
        }
    }
    StripArgs sa{};
    sa.geo = geo;
    sa.w = w;
    sa.tw = p->tw_w;
    sa.opd_att = reinterpret_cast<const float2 *>(opd_att);
    sa.opd_out = reinterpret_cast<float2 *>(opd_out);
    sa.S = S;
    for (int s = 0; s < S; ++s) sa.sc[s] = gd.sc[s];
    ColumnArgs ca{};
    ca.geo = geo;
    ca.w = w;
    ca.tw = p->tw_h;
    ca.S = S;
    ca.K = K;
    for (int s = 0; s < S; ++s)
        for (int k = 0; k < K; ++k) ca.md[s][k] = gd.md[s][k];
    ca.wait_polls = opt.wait_polls;
    ca.wait_extra = opt.wait_extra;
    InverseArgs ia{};
    ia.geo = geo;
    ia.w = w;
    ia.tw = p->tw_w;
    ia.images = images;
    ia.S = S;
    ia.K = K;
    if (opt.persistent && stage == kFull && geo.H == geo.W) {
        PersistArgs pa{};
        pa.sa = sa;
        pa.ca = ca;
        pa.ia = ia;
        pa.ctr = reinterpret_cast<int32_t *>(static_cast<char *>(ws) + l.ctr);
        pa.total = S * (geo.nstrips + geo.nblocks + K * geo.nstrips);
        pa.wait_polls = opt.wait_polls > 0 ? opt.wait_polls : (1 << 24);
        pa.wait_extra = opt.wait_extra > 0 ? opt.wait_extra : 0;
        cudaError_t e = cudaMemsetAsync(pa.ctr, 0, sizeof(int32_t) * (2 + 2 * S), st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
        return run_kernel(p, OSOG_KERNEL_PERSISTENT, st, [&] { return launch_persistent(pa, st); });
    }
    if (stage == kFull) {
        rc = raster_and_strip(p, sa, st, opt.raster_tiles);
    } else {
        const StripMode sm = stage == kOpdOnly ? kStripOpdOnly : kStripFromMap;
        rc = run_kernel(p, OSOG_KERNEL_STRIP_FORWARD, st, [&] { return launch_strip_forward(sa, sm, st); });
    }
    if (rc || stage == kOpdOnly) return rc;
    rc = run_kernel(p, OSOG_KERNEL_COLUMN, st, [&] { return launch_column(ca, st); });
    if (rc) return rc;
    return run_kernel(p, OSOG_KERNEL_STRIP_INVERSE, st, [&] { return launch_strip_inverse(ia, st); });
}

int check_ws(void *ws, size_t need, size_t have) {
    if (!ws && need) return fail(OSOG_ERR_WORKSPACE, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(OSOG_ERR_WORKSPACE, "workspace not 256-byte aligned");
    if (have < need) return fail(OSOG_ERR_WORKSPACE, "workspace too small");
    return OSOG_OK;
}

size_t ws_need(const osog_plan *p, int64_t n_total, int K, int S, int pairs_pp) {
    const int Sg = S < kMaxScenes ? S : kMaxScenes;
    const int64_t chunks = (n_total + kChunk - 1) / kChunk + S;
    return make_layout(p->geo, n_total, chunks, Sg, K, n_total * pairs_pp).total;
}

// Workspace of the adjoint: the forward regions (one scene, K modalities)
// followed by the slot map, the per-(band slot, strip) particle partials and
// the per-block optics partials.
struct BwdLayout {
    Layout fwd;
    size_t slotmap, part, opart, total;
};

BwdLayout make_bwd_layout(const Geometry &geo, int64_t n, int64_t chunks, int K, int ppp) {
    BwdLayout b;
    const int64_t pairs = n * ppp;
    b.fwd = make_layout(geo, n, chunks, 1, K, pairs);
    size_t o = b.fwd.total;
    b.slotmap = o;
    o = align256(o + (size_t)n * ppp * sizeof(int32_t));
    b.part = o;
    o = align256(o + (size_t)pairs * (geo.BH / geo.R) * 8 * sizeof(float));
    b.opart = o;
    o = align256(o + (size_t)geo.nblocks * 4 * sizeof(float));
    b.total = o;
    return b;
}

// One scene's forward pass laid out for the adjoint: the launch group, the
// carved work regions and the adjoint's partial buffers.
struct BwdState {
    BwdLayout bl;
    GroupDev gd;
    SceneDev sc;
    Work w;
    float *part, *opart;
    int K;
    int64_t chunks;
};

int bwd_setup(osog_plan *p, const float *soa, int64_t ld, int32_t n, const osog_optics_t *optics,
              void *ws, size_t ws_bytes, BwdState &b) {
    if (!p) return fail(OSOG_ERR_INVALID_ARG, "plan is NULL");
    int rc = check_optics(p, optics);
    if (rc) return rc;
    if (n < 0 || (int64_t)n > ld) return fail(OSOG_ERR_INVALID_ARG, "need 0 <= n <= ld");
    if (n > 0 && !soa) return fail(OSOG_ERR_INVALID_ARG, "soa is NULL");
    b.K = popcount3(optics->modes);
    b.chunks = (n + kChunk - 1) / kChunk;
    const int ppp = p->ppp;
    b.bl = make_bwd_layout(p->geo, n, b.chunks, b.K, ppp);
    rc = check_ws(ws, b.bl.total, ws_bytes);
    if (rc) return rc;
    b.gd = GroupDev{};
    b.gd.S = 1;
    b.gd.K = b.K;
    b.gd.nchunks = (int32_t)b.chunks;
    b.sc = scene_dev(*optics);
    b.sc.p0 = 0;
    b.sc.n = n;
    b.sc.chunk0 = 0;
    b.sc.pair0 = 0;
    b.sc.pair_cap = (int32_t)((int64_t)n * ppp);
    b.gd.sc[0] = b.sc;
    for (int bit = 0, k = 0; bit < 3; ++bit)
        if (optics->modes & (1u << bit)) b.gd.md[0][k++] = mode_dev(*optics, 1u << bit, p->optics_dyn);
    b.w = carve(ws, b.bl.fwd, p->status);
    b.w.slotmap = reinterpret_cast<int32_t *>(static_cast<char *>(ws) + b.bl.slotmap);
    b.w.slotmap_ppp = ppp;
    b.part = reinterpret_cast<float *>(static_cast<char *>(ws) + b.bl.part);
    b.opart = reinterpret_cast<float *>(static_cast<char *>(ws) + b.bl.opart);
    return OSOG_OK;
}

int bwd_check_grads(const float *grad_image, const float *grad_soa, const float *grad_optics,
                    int32_t n) {
    if (n > 0 && !grad_soa) return fail(OSOG_ERR_INVALID_ARG, "grad_soa is NULL");
    if (!grad_image || !grad_optics) return fail(OSOG_ERR_INVALID_ARG, "grad_image or grad_optics is NULL");
    return OSOG_OK;
}

// Forward pass into the adjoint's layout: binning (with the slot map), the
// strip and column passes up to the filtered columns Q_m, and, when image is
// given, the inverse strip pass that writes the images.
int bwd_forward(osog_plan *p, const float *soa, int64_t ld, const BwdState &b, float *image,
                cudaStream_t st) {
    const Geometry &geo = p->geo;
    int rc;
    if (b.gd.nchunks == 1) {  // one chunk: the three binning passes in one launch
        rc = run_kernel(p, OSOG_KERNEL_BIN_COUNT, st,
                        [&] { return launch_bin_single(soa, ld, b.gd, geo, b.w, st); });
        if (rc) return rc;
    } else {
        rc = run_kernel(p, OSOG_KERNEL_BIN_COUNT, st,
                        [&] { return launch_bin_count(soa, ld, b.gd, geo, b.w, st); });
        if (rc) return rc;
        rc = run_kernel(p, OSOG_KERNEL_BIN_SCAN, st, [&] { return launch_bin_scan(b.gd, geo, b.w, st); });
        if (rc) return rc;
        rc = run_kernel(p, OSOG_KERNEL_BIN_FILL, st, [&] { return launch_bin_fill(b.gd, geo, b.w, st); });
        if (rc) return rc;
    }
    StripArgs sa{};
    sa.geo = geo;
    sa.w = b.w;
    sa.tw = p->tw_w;
    sa.S = 1;
    sa.sc[0] = b.sc;
    rc = raster_and_strip(p, sa, st);
    if (rc) return rc;
    ColumnArgs ca{};
    ca.geo = geo;
    ca.w = b.w;
    ca.tw = p->tw_h;
    ca.S = 1;
    ca.K = b.K;
    for (int k = 0; k < b.K; ++k) ca.md[0][k] = b.gd.md[0][k];
    rc = run_kernel(p, OSOG_KERNEL_COLUMN, st, [&] { return launch_column(ca, st); });
    if (rc || !image) return rc;
    InverseArgs ia{};
    ia.geo = geo;
    ia.w = b.w;
    ia.tw = p->tw_w;
    ia.images = image;
    ia.S = 1;
    ia.K = b.K;
    return run_kernel(p, OSOG_KERNEL_STRIP_INVERSE, st, [&] { return launch_strip_inverse(ia, st); });
}

// The adjoint passes over a forward state left in the workspace by
// bwd_forward: dL/dI -> dL/dQ_m (rows), -> dL/dG and the optics partials
// (columns), -> per-(band slot, strip) particle partials (strips), and the
// fixed-order sums into grad_soa and grad_optics.
int bwd_adjoint(osog_plan *p, const BwdState &b, const float *grad_image, float *grad_soa,
                int64_t ld, float *grad_optics, cudaStream_t st) {
    const Geometry &geo = p->geo;
    BwdRowsArgs ra{};
    ra.geo = geo;
    ra.w = b.w;
    ra.tw = p->tw_w;
    ra.grad_image = grad_image;
    ra.S = 1;
    ra.K = b.K;
    int rc = run_kernel(p, OSOG_KERNEL_BWD_ROWS, st, [&] { return launch_bwd_rows(ra, st); });
    if (rc) return rc;
    BwdColumnArgs bc{};
    bc.geo = geo;
    bc.w = b.w;
    bc.tw = p->tw_h;
    bc.opart = b.opart;
    bc.S = 1;
    bc.K = b.K;
    for (int k = 0; k < b.K; ++k) bc.md[0][k] = b.gd.md[0][k];
    rc = run_kernel(p, OSOG_KERNEL_BWD_COLUMN, st, [&] { return launch_bwd_column(bc, st); });
    if (rc) return rc;
    BwdStripArgs bs{};
    bs.geo = geo;
    bs.w = b.w;
    bs.tw = p->tw_w;
    bs.part = b.part;
    bs.S = 1;
    bs.sc[0] = b.sc;
    rc = run_kernel(p, OSOG_KERNEL_BWD_STRIP, st, [&] { return launch_bwd_strip(bs, st); });
    if (rc) return rc;
    BwdReduceArgs br{};
    br.geo = geo;
    br.w = b.w;
    br.part = b.part;
    br.opart = b.opart;
    br.grad_soa = grad_soa;
    br.ld = ld;
    br.grad_optics = grad_optics;
    br.S = 1;
    br.nchunks = (int32_t)b.chunks;
    br.sc[0] = b.sc;
    return run_kernel(p, OSOG_KERNEL_BWD_REDUCE, st, [&] { return launch_bwd_reduce(br, st); });
}

// Field-by-field equality (the struct has padding).
bool same_optics(const osog_optics_t &a, const osog_optics_t &b) {
    return a.H == b.H && a.W == b.W && a.dx_um == b.dx_um && a.lambda_um == b.lambda_um &&
           a.NA == b.NA && a.n_medium == b.n_medium && a.defocus_um == b.defocus_um &&
           a.modes == b.modes && a.oblique_frac == b.oblique_frac &&
           a.oblique_angle == b.oblique_angle && a.shear_px == b.shear_px &&
           a.shear_angle == b.shear_angle && a.bias_phase == b.bias_phase &&
           a.bevel_slope == b.bevel_slope;
}

// Drop every kept forward state of the plan.
void forget_all_kept(osog_plan *p) {
    std::lock_guard<std::mutex> guard(p->kept_lock);
    p->kept.clear();
}

// Drop the forward states that osog_render_keep left in workspace ws (any
// other call that writes ws invalidates them).
void forget_kept(osog_plan *p, const void *ws) {
    std::lock_guard<std::mutex> guard(p->kept_lock);
    for (size_t i = p->kept.size(); i-- > 0;)
        if (p->kept[i].ws == ws) p->kept.erase(p->kept.begin() + i);
}

}  // namespace

extern "C" {

const char *osog_last_error(void) { return g_err.c_str(); }

int osog_plan_create(osog_plan_t **out, int32_t H, int32_t W) {
    if (!out) return fail(OSOG_ERR_INVALID_ARG, "plan pointer is NULL");
    *out = nullptr;
    if (!pow2_in_range(H) || !pow2_in_range(W))
        return fail(OSOG_ERR_UNSUPPORTED_SIZE, "H and W must be powers of two in [32, 2048]");
    osog_plan *p = new osog_plan();
    p->H = H;
    p->W = W;
    p->geo = make_geometry(H, W);
    cudaError_t e = cudaMalloc(&p->tw_w, sizeof(float2) * (W + H));
    if (e == cudaSuccess) e = cudaMalloc(&p->status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&p->status_host, sizeof(int32_t));
    if (e == cudaSuccess) {
        std::vector<float2> tw(W + H);
        fill_twiddles(W, tw.data());
        fill_twiddles(H, tw.data() + W);
        p->tw_h = p->tw_w + W;
        e = cudaMemcpy(p->tw_w, tw.data(), sizeof(float2) * (W + H), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(p->status, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = prepare_kernels(H, W);
    if (e == cudaSuccess) e = prepare_backward(H, W);
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "osog_plan_create");
        osog_plan_destroy(p);
        return rc;
    }
    *out = p;
    return OSOG_OK;
}

void osog_plan_destroy(osog_plan_t *p) {
    if (!p) return;
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    cudaFree(p->tw_w);
    cudaFree(p->status);
    cudaFreeHost(p->status_host);
    delete p;
}

size_t osog_workspace_size(const osog_plan_t *p, int32_t n_max, int32_t K, int32_t batch) {
    if (!p || n_max < 0 || K < 0 || K > 3 || batch < 1) return 0;
    return ws_need(p, n_max, K, batch, p->ppp);
}

static int render_stage(osog_plan_t *p, const float *soa, int64_t ld, int32_t n,
                        const osog_optics_t *optics, float *image, const float *opd_att,
                        float *opd_out, void *ws, size_t ws_bytes, osog_stream_t stream,
                        Stage stage) {
    if (!p) return fail(OSOG_ERR_INVALID_ARG, "plan is NULL");
    forget_kept(p, ws);
    int rc = check_optics(p, optics);
    if (rc) return rc;
    if (n < 0 || (int64_t)n > ld) return fail(OSOG_ERR_INVALID_ARG, "need 0 <= n <= ld");
    if (stage != kFromMap && n > 0 && !soa) return fail(OSOG_ERR_INVALID_ARG, "soa is NULL");
    if (stage == kFromMap && !opd_att) return fail(OSOG_ERR_INVALID_ARG, "opd_att is NULL");
    if (stage == kOpdOnly && !opd_out) return fail(OSOG_ERR_INVALID_ARG, "opd_att output is NULL");
    if (stage != kOpdOnly && !image) return fail(OSOG_ERR_INVALID_ARG, "image is NULL");
    const int K = popcount3(optics->modes);
    const int nn = stage == kFromMap ? 0 : n;
    rc = check_ws(ws, ws_need(p, nn, stage == kOpdOnly ? 0 : K, 1, p->ppp), ws_bytes);
    if (rc) return rc;
    GroupOpts o;
    o.ppp = p->ppp;
    return enqueue_group(p, soa, ld, &nn, 1, optics, K, o, ws, ws_bytes, image,
                         opd_att, opd_out, stage, reinterpret_cast<cudaStream_t>(stream));
}

int osog_render(osog_plan_t *p, const float *soa, int64_t ld, int32_t n,
                const osog_optics_t *optics, float *image, void *ws, size_t ws_bytes,
                osog_stream_t stream) {
    return render_stage(p, soa, ld, n, optics, image, nullptr, nullptr, ws, ws_bytes, stream, kFull);
}

size_t osog_polyhedra_workspace_size(const osog_plan_t *p, int32_t n_max, int32_t K,
                                     int32_t n_planes) {
    if (!p || n_max < 0 || K < 1 || K > 3 || n_planes < 0) return 0;
    return align256(ws_need(p, n_max, K, 1, p->ppp)) + (size_t)n_planes * sizeof(float4);
}

int osog_render_polyhedra(osog_plan_t *p, const float *soa, int64_t ld, int32_t n,
                          const float *planes, const int32_t *plane_offsets, int32_t n_planes,
                          const osog_optics_t *optics, float *image, void *ws, size_t ws_bytes,
                          osog_stream_t stream) {
    if (!p) return fail(OSOG_ERR_INVALID_ARG, "plan is NULL");
    forget_kept(p, ws);
    int rc = check_optics(p, optics);
    if (rc) return rc;
    if (n < 0 || (int64_t)n > ld) return fail(OSOG_ERR_INVALID_ARG, "need 0 <= n <= ld");
    if (n > 0 && !soa) return fail(OSOG_ERR_INVALID_ARG, "soa is NULL");
    if (!image) return fail(OSOG_ERR_INVALID_ARG, "image is NULL");
    if (n_planes < 0 || (n_planes > 0 && !planes) || !plane_offsets)
        return fail(OSOG_ERR_INVALID_ARG, "planes / plane_offsets missing");
    if (reinterpret_cast<uintptr_t>(planes) & 15)
        return fail(OSOG_ERR_INVALID_ARG, "planes must be 16-byte aligned");
    const int K = popcount3(optics->modes);
    rc = check_ws(ws, osog_polyhedra_workspace_size(p, n, K, n_planes), ws_bytes);
    if (rc) return rc;
    GroupOpts o;
    o.ppp = p->ppp;
    o.planes = reinterpret_cast<const float4 *>(planes);
    o.plane_off = plane_offsets;
    o.n_planes = n_planes;
    return enqueue_group(p, soa, ld, &n, 1, optics, K, o, ws, ws_bytes, image, nullptr, nullptr,
                         kFull, reinterpret_cast<cudaStream_t>(stream));
}

// Workspace of the incoherent DIC render: the one-scene, one-modality
// regions, then a float [H][W] intensity buffer and the complex [H][W]
// optical transfer function table (column-blocked like Q).
struct DicLayout {
    Layout l;
    size_t img, otf, total;
};

DicLayout dic_layout(const Geometry &geo, int64_t n, int ppp) {
    DicLayout d;
    d.l = make_layout(geo, n, (n + kChunk - 1) / kChunk + 1, 1, 1, n * ppp);
    size_t o = d.l.total;
    d.img = o;
    o = align256(o + (size_t)geo.H * geo.W * sizeof(float));
    d.otf = o;
    o = align256(o + (size_t)geo.H * geo.W * sizeof(float2));
    d.total = o;
    return d;
}

size_t osog_dic_incoherent_workspace_size(const osog_plan_t *p, int32_t n_max) {
    if (!p || n_max < 0) return 0;
    return dic_layout(p->geo, n_max, p->ppp).total;
}

int osog_render_dic_incoherent(osog_plan_t *p, const float *soa, int64_t ld, int32_t n,
                               const osog_optics_t *optics, float *image, void *ws,
                               size_t ws_bytes, osog_stream_t stream) {
    if (!p) return fail(OSOG_ERR_INVALID_ARG, "plan is NULL");
    forget_kept(p, ws);
    int rc = check_optics(p, optics);
    if (rc) return rc;
    if (n < 0 || (int64_t)n > ld) return fail(OSOG_ERR_INVALID_ARG, "need 0 <= n <= ld");
    if (n > 0 && !soa) return fail(OSOG_ERR_INVALID_ARG, "soa is NULL");
    if (!image) return fail(OSOG_ERR_INVALID_ARG, "image is NULL");
    const Geometry &geo = p->geo;
    const DicLayout dl = dic_layout(geo, n, p->ppp);
    rc = check_ws(ws, dl.total, ws_bytes);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const Work w = carve(ws, dl.l, p->status);
    float *J = reinterpret_cast<float *>(static_cast<char *>(ws) + dl.img);
    float2 *otf = reinterpret_cast<float2 *>(static_cast<char *>(ws) + dl.otf);

    GroupDev gd{};
    gd.S = 1;
    gd.K = 1;
    gd.sc[0] = scene_dev(*optics);  // no particles until step 3
    StripArgs sa{};
    sa.geo = geo;
    sa.w = w;
    sa.tw = p->tw_w;
    sa.S = 1;
    ColumnArgs ca{};
    ca.geo = geo;
    ca.w = w;
    ca.tw = p->tw_h;
    ca.S = 1;
    ca.K = 1;
    InverseArgs ia{};
    ia.geo = geo;
    ia.w = w;
    ia.tw = p->tw_w;
    ia.S = 1;
    ia.K = 1;
    // Each step bounds its modality's columns (all of them for every op but
    // the pupil) before the render kernels run.
    auto use_mode = [&](const ModeDev &md) {
        gd.md[0][0] = md;
        ca.md[0][0] = md;
        sa.sc[0] = gd.sc[0];
        return run_kernel(p, OSOG_KERNEL_BIN_SCAN, st, [&] { return launch_bin_scan(gd, geo, w, st); });
    };
    auto column = [&] { return run_kernel(p, OSOG_KERNEL_COLUMN, st, [&] { return launch_column(ca, st); }); };
    auto inverse = [&] {
        return run_kernel(p, OSOG_KERNEL_STRIP_INVERSE, st, [&] { return launch_strip_inverse(ia, st); });
    };
    auto strip = [&](StripMode m) {
        if (m == kStripRender) return raster_and_strip(p, sa, st);
        return run_kernel(p, OSOG_KERNEL_STRIP_FORWARD, st, [&] { return launch_strip_forward(sa, m, st); });
    };

    // 1. |h|^2: unit spectrum times the brightfield pupil (NA, defocus),
    //    inverse transform, squared modulus (h = IDFT2(P) / (H W)).
    const ModeDev bf = mode_dev(*optics, OSOG_MODE_BRIGHTFIELD, p->optics_dyn);
    ca.unit_input = 1;
    ia.images = J;
    ia.real_out = 0;
    if ((rc = use_mode(bf)) || (rc = column()) || (rc = inverse())) return rc;
    // 2. OTF = DFT2(|h|^2), kept as a table (its DC term is sum |h|^2).
    ModeDev sp{};
    sp.op = kOpSpectrum;
    sp.tab = otf;
    sp.scale = 1.f;
    ca.unit_input = 0;
    sa.opd_att = reinterpret_cast<const float2 *>(J);
    if ((rc = use_mode(sp)) || (rc = strip(kStripFromReal)) || (rc = column())) return rc;
    // 3. J = |D|^2, D = IDFT2(DFT2(U) 2i sin(k . ds + theta)) / (H W): the
    //    exit wave sheared and interfered on every frequency (Eq. 5).
    ModeDev dic = mode_dev(*optics, OSOG_MODE_DIC, p->optics_dyn);
    dic.op = kOpAllPass;
    dic.dz = 0.f;
    dic.fixed_dz = 1;  // the defocus is in |h|^2 (step 1), also when bound
    const int64_t chunks = (n + kChunk - 1) / kChunk;
    gd.nchunks = (int32_t)chunks;
    gd.sc[0].n = n;
    gd.sc[0].pair_cap = (int32_t)((int64_t)n * p->ppp);
    if ((rc = run_kernel(p, OSOG_KERNEL_BIN_COUNT, st,
                         [&] { return launch_bin_count(soa, ld, gd, geo, w, st); })))
        return rc;
    if ((rc = use_mode(dic))) return rc;
    if ((rc = run_kernel(p, OSOG_KERNEL_BIN_FILL, st, [&] { return launch_bin_fill(gd, geo, w, st); })))
        return rc;
    if ((rc = strip(kStripRender)) || (rc = column()) || (rc = inverse())) return rc;
    // 4. I = IDFT2(DFT2(J) OTF / OTF(0)) / (H W): J blurred by the unit-sum
    //    intensity PSF; the result is real.
    ModeDev tb{};
    tb.op = kOpTable;
    tb.tab = otf;
    tb.scale = (float)(1.0 / ((double)geo.H * geo.W));
    gd.nchunks = 0;
    gd.sc[0].n = 0;
    gd.sc[0].pair_cap = 0;
    ia.images = image;
    ia.real_out = 1;
    if ((rc = use_mode(tb)) || (rc = strip(kStripFromReal)) || (rc = column()) || (rc = inverse()))
        return rc;
    return OSOG_OK;
}

int osog_render_opd(osog_plan_t *p, const float *soa, int64_t ld, int32_t n,
                    const osog_optics_t *optics, float *opd_att, void *ws, size_t ws_bytes,
                    osog_stream_t stream) {
    return render_stage(p, soa, ld, n, optics, nullptr, nullptr, opd_att, ws, ws_bytes, stream,
                        kOpdOnly);
}

int osog_optics_from_opd(osog_plan_t *p, const float *opd_att, const osog_optics_t *optics,
                         float *image, void *ws, size_t ws_bytes, osog_stream_t stream) {
    return render_stage(p, nullptr, 0, 0, optics, image, opd_att, nullptr, ws, ws_bytes, stream,
                        kFromMap);
}

static int batch_enqueue(osog_plan_t *p, const float *soa_all, int64_t ld, const int32_t *offsets,
                         int32_t S, const osog_optics_t *optics, float *images, int K,
                         const GroupOpts &opt, void *ws, size_t ws_bytes, cudaStream_t st,
                         Stage stage = kFull, int *ppp_needed = nullptr) {
    const size_t img_scene = (size_t)K * p->H * p->W;
    for (int g0 = 0; g0 < S; g0 += kMaxScenes) {
        const int Sg = S - g0 < kMaxScenes ? S - g0 : kMaxScenes;
        int32_t counts[kMaxScenes];
        for (int s = 0; s < Sg; ++s) counts[s] = offsets[g0 + s + 1] - offsets[g0 + s];
        const float *soa_g = soa_all ? soa_all + offsets[g0] : nullptr;
        std::vector<int32_t> offs;
        GroupOpts o = opt;
        o.band_off_out = &offs;
        int rc = enqueue_group(p, soa_g, ld, counts, Sg, optics + g0, K, o, ws, ws_bytes,
                               images + (size_t)g0 * img_scene, nullptr, nullptr, stage, st);
        if (rc) return rc;
        if (stage == kBinOnly && ppp_needed) {
            const int nb = (int)(offs.size() / Sg) - 1;
            for (int s = 0; s < Sg; ++s)
                if (counts[s] > 0) {
                    const int64_t tot = offs[(size_t)s * (nb + 1) + nb];
                    const int need = (int)((tot + counts[s] - 1) / counts[s]);
                    if (need > *ppp_needed) *ppp_needed = need;
                }
        }
    }
    return OSOG_OK;
}

int osog_batch_submit(osog_plan_t *p, const float *soa_all, int64_t ld, const int32_t *offsets,
                      int32_t S, const osog_optics_t *optics, float *images,
                      const osog_tuning_t *tuning, void *ws, size_t ws_bytes,
                      osog_stream_t stream) {
    if (!p) return fail(OSOG_ERR_INVALID_ARG, "plan is NULL");
    forget_kept(p, ws);
    if (S < 1 || !offsets || !optics || !images)
        return fail(OSOG_ERR_INVALID_ARG, "need S >= 1 and non-NULL offsets, optics, images");
    for (int s = 0; s < S; ++s) {
        if (offsets[s + 1] < offsets[s] || offsets[s] < 0)
            return fail(OSOG_ERR_INVALID_ARG, "offsets must be non-decreasing and >= 0");
        int rc = check_optics(p, optics + s);
        if (rc) return rc;
        if (optics[s].modes != optics[0].modes)
            return fail(OSOG_ERR_INVALID_ARG, "all scenes must select the same modes");
    }
    if ((int64_t)offsets[S] > ld) return fail(OSOG_ERR_INVALID_ARG, "offsets[S] > ld");
    const int64_t n_total = (int64_t)offsets[S] - offsets[0];
    if (n_total > 0 && !soa_all) return fail(OSOG_ERR_INVALID_ARG, "soa_all is NULL");
    const int K = popcount3(optics[0].modes);
    // Options: explicit tuning fields first, then the autotuned values for
    // this batch shape, then the defaults.
    GroupOpts opt;
    opt.ppp = p->ppp;
    for (const auto &t : p->tuned)
        if (t.S == S && t.n == n_total && t.K == K) {
            opt.ppp = t.ppp;
            opt.persistent = t.persistent > 0;
            opt.band_rows = t.band_rows;
            opt.raster_tiles = t.raster > 0;
        }
    bool use_graph = true;
    if (tuning) {
        if (tuning->pairs_per_particle > 0) opt.ppp = tuning->pairs_per_particle;
        if (tuning->persistent != 0) opt.persistent = tuning->persistent > 0;
        if (tuning->band_rows > 0) opt.band_rows = tuning->band_rows;
        opt.wait_polls = tuning->wait_polls;
        opt.wait_extra = tuning->test_wait_extra;
        if (tuning->raster != 0) opt.raster_tiles = tuning->raster > 0;
        use_graph = tuning->use_graph > 0;
    }
    const int ppp = opt.ppp;
    int rc = check_ws(ws, ws_need(p, n_total, K, S, ppp), ws_bytes);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (st) cudaStreamIsCapturing(st, &cs);
    if (!use_graph || p->prof || !st || cs != cudaStreamCaptureStatusNone)
        return batch_enqueue(p, soa_all, ld, offsets, S, optics, images, K, opt, ws, ws_bytes, st);

    // Key of the launch sequence: every argument that ends up in a kernel.
    std::vector<unsigned char> key;
    auto put = [&key](const void *d, size_t b) {
        const unsigned char *c = static_cast<const unsigned char *>(d);
        key.insert(key.end(), c, c + b);
    };
    put(&soa_all, sizeof soa_all);
    put(&ld, sizeof ld);
    put(&S, sizeof S);
    put(offsets, sizeof(int32_t) * (S + 1));
    put(optics, sizeof(osog_optics_t) * S);
    put(&images, sizeof images);
    put(&ws, sizeof ws);
    put(&ws_bytes, sizeof ws_bytes);
    put(&opt.ppp, sizeof opt.ppp);
    put(&opt.persistent, sizeof opt.persistent);
    put(&opt.band_rows, sizeof opt.band_rows);
    put(&opt.wait_polls, sizeof opt.wait_polls);
    put(&opt.wait_extra, sizeof opt.wait_extra);
    put(&opt.raster_tiles, sizeof opt.raster_tiles);
    put(&p->optics_dyn, sizeof p->optics_dyn);
    if (!(p->gexec && key == p->gkey)) {
        const int64_t before = p->launches;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        rc = batch_enqueue(p, soa_all, ld, offsets, S, optics, images, K, opt, ws, ws_bytes, st);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(st, &g);
        p->graph_kernels = p->launches - before;
        p->launches = before;
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        if (p->gexec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(p->gexec, g, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(p->gexec);
                p->gexec = nullptr;
            }
        }
        if (!p->gexec) {
            e = cudaGraphInstantiate(&p->gexec, g, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(g);
                p->gexec = nullptr;
                return cuda_fail(e, "cudaGraphInstantiate");
            }
        }
        cudaGraphDestroy(g);
        p->gkey.swap(key);
    }
    cudaError_t e = cudaGraphLaunch(p->gexec, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    p->launches += p->graph_kernels;
    return OSOG_OK;
}

size_t osog_backward_workspace_size(const osog_plan_t *p, int32_t n_max, int32_t K) {
    if (!p || n_max < 0 || K < 1 || K > 3) return 0;
    return make_bwd_layout(p->geo, n_max, (n_max + kChunk - 1) / kChunk + 1, K, p->ppp).total;
}

int osog_render_backward(osog_plan_t *p, const float *soa, int64_t ld, int32_t n,
                         const osog_optics_t *optics, const float *grad_image, float *grad_soa,
                         float *grad_optics, void *ws, size_t ws_bytes, osog_stream_t stream) {
    BwdState b;
    int rc = bwd_setup(p, soa, ld, n, optics, ws, ws_bytes, b);
    if (rc) return rc;
    rc = bwd_check_grads(grad_image, grad_soa, grad_optics, n);
    if (rc) return rc;
    forget_kept(p, ws);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    rc = bwd_forward(p, soa, ld, b, nullptr, st);  // recompute up to the filtered columns
    if (rc) return rc;
    return bwd_adjoint(p, b, grad_image, grad_soa, ld, grad_optics, st);
}

int osog_render_keep(osog_plan_t *p, const float *soa, int64_t ld, int32_t n,
                     const osog_optics_t *optics, float *image, void *ws, size_t ws_bytes,
                     osog_stream_t stream) {
    BwdState b;
    int rc = bwd_setup(p, soa, ld, n, optics, ws, ws_bytes, b);
    if (rc) return rc;
    if (!image) return fail(OSOG_ERR_INVALID_ARG, "image is NULL");
    forget_kept(p, ws);
    rc = bwd_forward(p, soa, ld, b, image, reinterpret_cast<cudaStream_t>(stream));
    if (rc) return rc;
    osog_plan::Kept k{};
    k.ws = ws;
    k.ws_bytes = ws_bytes;
    k.soa = soa;
    k.ld = ld;
    k.n = n;
    k.optics = *optics;
    std::lock_guard<std::mutex> guard(p->kept_lock);
    if (p->kept.size() >= kMaxKept) p->kept.erase(p->kept.begin());  // the oldest goes
    p->kept.push_back(k);
    return OSOG_OK;
}

int osog_render_backward_kept(osog_plan_t *p, const float *soa, int64_t ld, int32_t n,
                              const osog_optics_t *optics, const float *grad_image,
                              float *grad_soa, float *grad_optics, void *ws, size_t ws_bytes,
                              osog_stream_t stream) {
    BwdState b;
    int rc = bwd_setup(p, soa, ld, n, optics, ws, ws_bytes, b);
    if (rc) return rc;
    rc = bwd_check_grads(grad_image, grad_soa, grad_optics, n);
    if (rc) return rc;
    bool found = false;
    {
        std::lock_guard<std::mutex> guard(p->kept_lock);
        for (const osog_plan::Kept &k : p->kept)
            found = found || (k.ws == ws && k.ws_bytes == ws_bytes && k.soa == soa &&
                              k.ld == ld && k.n == n && same_optics(k.optics, *optics));
    }
    if (!found)
        return fail(OSOG_ERR_INVALID_ARG, "no forward state kept in this workspace for these "
                                          "arguments (osog_render_keep)");
    forget_kept(p, ws);  // the adjoint overwrites the kept spectra
    return bwd_adjoint(p, b, grad_image, grad_soa, ld, grad_optics,
                       reinterpret_cast<cudaStream_t>(stream));
}

int osog_autotune(osog_plan_t *p, const float *soa_all, int64_t ld, const int32_t *offsets,
                  int32_t S, const osog_optics_t *optics, float *images, void *ws,
                  size_t ws_bytes, osog_stream_t stream, osog_tuning_t *out) {
    // Validate once through the direct path (it also warms the kernels up).
    osog_tuning_t base{};
    base.use_graph = -1;
    base.persistent = -1;
    int rc = osog_batch_submit(p, soa_all, ld, offsets, S, optics, images, &base, ws, ws_bytes, stream);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int K = popcount3(optics[0].modes);
    const int64_t n_total = (int64_t)offsets[S] - offsets[0];
    std::vector<int> bands;
    for (int bh = p->geo.BH; bh <= p->H && bands.size() < 4; bh *= 2) bands.push_back(bh);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(OSOG_ERR_CUDA, "cudaEventCreate");
    float best = 1e30f;
    GroupOpts chosen;
    for (int bh : bands) {
        GroupOpts o;
        o.band_rows = bh;
        int need = 1;
        rc = batch_enqueue(p, soa_all, ld, offsets, S, optics, images, K, o, ws, ws_bytes, st,
                           kBinOnly, &need);
        if (rc) break;
        o.ppp = need;
        if (ws_need(p, n_total, K, S, o.ppp) > ws_bytes) continue;
        for (int mode = 0; mode < (p->H == p->W ? 3 : 2); ++mode) {
            o.persistent = mode == 2;       // one persistent launch
            o.raster_tiles = mode == 1;     // the raster in a kernel of its own
            float t[5];
            for (int r = 0; r < 5 && rc == OSOG_OK; ++r) {
                cudaEventRecord(e0, st);
                rc = batch_enqueue(p, soa_all, ld, offsets, S, optics, images, K, o, ws, ws_bytes, st);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t[r], e0, e1) != cudaSuccess)
                    rc = fail(OSOG_ERR_CUDA, "autotune timing");
            }
            if (rc) break;
            std::sort(t, t + 5);
            const float med = t[2];
            if (med < best) {
                best = med;
                chosen = o;
            }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // The dry runs may have latched a bin overflow for candidates they then
    // sized exactly: clear the status word.
    cudaMemsetAsync(p->status, 0, sizeof(int32_t), st);
    cudaStreamSynchronize(st);
    if (rc) return rc;
    bool found = false;
    for (auto &t : p->tuned)
        if (t.S == S && t.n == n_total && t.K == K) {
            t = {S, n_total, K, chosen.ppp, chosen.persistent ? 1 : -1, chosen.band_rows,
                 chosen.raster_tiles ? 1 : -1};
            found = true;
        }
    if (!found)
        p->tuned.push_back({S, n_total, K, chosen.ppp, chosen.persistent ? 1 : -1, chosen.band_rows,
                            chosen.raster_tiles ? 1 : -1});
    if (out) {
        *out = osog_tuning_t{};
        out->pairs_per_particle = chosen.ppp;
        out->use_graph = 1;
        out->persistent = chosen.persistent ? 1 : -1;
        out->band_rows = chosen.band_rows;
        out->raster = chosen.raster_tiles ? 1 : -1;
    }
    return OSOG_OK;
}

// ------------------------------------------------------------ image losses
// The target table: K complex spectra [K][W/B][H][B] (column-blocked like
// Q), then the K largest amplitudes.
static size_t loss_table_spectra(const osog_plan *p, int K) {
    return align256((size_t)K * p->H * p->W * sizeof(float2));
}

size_t osog_loss_table_size(const osog_plan_t *p, int32_t K) {
    if (!p || K < 1 || K > kMaxScenes) return 0;
    return loss_table_spectra(p, K) + align256((size_t)K * sizeof(float));
}

// Workspace of the loss passes: G and Q of K single-modality images, the
// column ranges, then the per-block partial sums.
static size_t loss_ws_part(const osog_plan *p, int K) {
    return make_layout(p->geo, 0, 0, K, 1, 0).total;
}

size_t osog_loss_workspace_size(const osog_plan_t *p, int32_t K) {
    if (!p || K < 1 || K > kMaxScenes) return 0;
    return loss_ws_part(p, K) + align256((size_t)K * p->geo.nblocks * 2 * sizeof(float));
}

// The spectra of K real images through the strip and column passes, with
// modality md (kOpSpectrum or kOpLoss) per image; the column ranges are
// set by the scan kernel (every column for these operations).
static int loss_passes(osog_plan *p, const float *images, int K, ModeDev md, float2 *tab,
                       const LossDev *loss, float *grad, void *ws, cudaStream_t st) {
    const Geometry &geo = p->geo;
    const Layout l = make_layout(geo, 0, 0, K, 1, 0);
    const Work w = carve(ws, l, p->status);
    GroupDev gd{};
    gd.S = K;
    gd.K = 1;
    StripArgs sa{};
    sa.geo = geo;
    sa.w = w;
    sa.tw = p->tw_w;
    sa.opd_att = reinterpret_cast<const float2 *>(images);
    sa.S = K;
    ColumnArgs ca{};
    ca.geo = geo;
    ca.w = w;
    ca.tw = p->tw_h;
    ca.S = K;
    ca.K = 1;
    if (loss) ca.loss = *loss;
    for (int s = 0; s < K; ++s) {
        md.tab = tab + (size_t)s * geo.H * geo.W;
        gd.md[s][0] = md;
        ca.md[s][0] = md;
    }
    int rc = run_kernel(p, OSOG_KERNEL_BIN_SCAN, st, [&] { return launch_bin_scan(gd, geo, w, st); });
    if (rc) return rc;
    rc = run_kernel(p, OSOG_KERNEL_STRIP_FORWARD, st,
                    [&] { return launch_strip_forward(sa, kStripFromReal, st); });
    if (rc) return rc;
    rc = run_kernel(p, OSOG_KERNEL_COLUMN, st, [&] { return launch_column(ca, st); });
    if (rc || !grad) return rc;
    InverseArgs ia{};
    ia.geo = geo;
    ia.w = w;
    ia.tw = p->tw_w;
    ia.images = grad;
    ia.S = K;
    ia.K = 1;
    ia.real_out = 1;
    return run_kernel(p, OSOG_KERNEL_STRIP_INVERSE, st, [&] { return launch_strip_inverse(ia, st); });
}

int osog_loss_target(osog_plan_t *p, const float *target, int32_t K, void *table,
                     size_t table_bytes, void *ws, size_t ws_bytes, osog_stream_t stream) {
    if (!p) return fail(OSOG_ERR_INVALID_ARG, "plan is NULL");
    if (K < 1 || K > kMaxScenes || !target || !table)
        return fail(OSOG_ERR_INVALID_ARG, "need 1 <= K <= 32 and non-NULL target, table");
    if (reinterpret_cast<uintptr_t>(table) & 255 || table_bytes < osog_loss_table_size(p, K))
        return fail(OSOG_ERR_WORKSPACE, "loss table too small or not 256-byte aligned");
    int rc = check_ws(ws, osog_loss_workspace_size(p, K), ws_bytes);
    if (rc) return rc;
    forget_kept(p, ws);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ModeDev md{};
    md.op = kOpSpectrum;
    md.scale = 1.f;
    float2 *spec = static_cast<float2 *>(table);
    rc = loss_passes(p, target, K, md, spec, nullptr, nullptr, ws, st);
    if (rc) return rc;
    float *maxamp = reinterpret_cast<float *>(static_cast<char *>(table) + loss_table_spectra(p, K));
    cudaError_t e = launch_max_amplitude(spec, K, (int64_t)p->H * p->W, maxamp, st);
    return e == cudaSuccess ? OSOG_OK : cuda_fail(e, "osog_loss_target");
}

int osog_image_loss(osog_plan_t *p, const float *image, int32_t K, const void *table,
                    size_t table_bytes, const osog_loss_t *params, float *loss,
                    float *grad_image, void *ws, size_t ws_bytes, osog_stream_t stream) {
    if (!p) return fail(OSOG_ERR_INVALID_ARG, "plan is NULL");
    if (K < 1 || K > kMaxScenes || !image || !table || !params || !loss)
        return fail(OSOG_ERR_INVALID_ARG, "need 1 <= K <= 32 and non-NULL image, table, params, loss");
    if (reinterpret_cast<uintptr_t>(table) & 255 || table_bytes < osog_loss_table_size(p, K))
        return fail(OSOG_ERR_WORKSPACE, "loss table too small or not 256-byte aligned");
    if (!finite_all({params->dx_um, params->misfit_scale, params->spectral_weight, params->eps_rel}) ||
        !(params->dx_um > 0) || !(params->eps_rel > 0))
        return fail(OSOG_ERR_INVALID_ARG, "loss parameters need finite values, dx_um > 0, eps_rel > 0");
    if ((params->misfit_scale != 0.0 && !params->cutoff) ||
        (reinterpret_cast<uintptr_t>(params->cutoff) & 3))
        return fail(OSOG_ERR_INVALID_ARG, "the misfit needs a 4-byte aligned device cutoff");
    int rc = check_ws(ws, osog_loss_workspace_size(p, K), ws_bytes);
    if (rc) return rc;
    forget_kept(p, ws);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    LossDev L{};
    L.cutoff = params->misfit_scale != 0.0 ? params->cutoff : nullptr;
    L.misfit_scale = (float)params->misfit_scale;
    L.spectral_weight = (float)params->spectral_weight;
    L.eps_rel = (float)params->eps_rel;
    L.inv_ntot = (float)(1.0 / ((double)K * p->H * p->W));
    L.fx_scale = (float)(1.0 / ((double)p->W * params->dx_um));
    L.fy_scale = (float)(1.0 / ((double)p->H * params->dx_um));
    L.maxamp = reinterpret_cast<const float *>(static_cast<const char *>(table) +
                                               loss_table_spectra(p, K));
    L.part = reinterpret_cast<float *>(static_cast<char *>(ws) + loss_ws_part(p, K));
    ModeDev md{};
    md.op = kOpLoss;
    rc = loss_passes(p, image, K, md, const_cast<float2 *>(static_cast<const float2 *>(table)),
                     &L, grad_image, ws, st);
    if (rc) return rc;
    cudaError_t e = launch_loss_reduce(L.part, (int64_t)K * p->geo.nblocks, loss, st);
    return e == cudaSuccess ? OSOG_OK : cuda_fail(e, "osog_image_loss");
}

int osog_plan_set_pairs_per_particle(osog_plan_t *p, int32_t pairs_per_particle) {
    if (!p) return fail(OSOG_ERR_INVALID_ARG, "plan is NULL");
    if (pairs_per_particle < 1 || pairs_per_particle > kMaxBands)
        return fail(OSOG_ERR_INVALID_ARG, "pairs_per_particle must be in 1..64");
    forget_all_kept(p);  // a kept state's layout depends on the reservation
    p->ppp = pairs_per_particle;
    return OSOG_OK;
}

int32_t osog_pairs_for_extent(const osog_plan_t *p, double max_half_extent_px) {
    if (!p || !(max_half_extent_px >= 0.0) || !isfinite(max_half_extent_px)) return 0;
    // a bounding rectangle spans at most 2 h + 4 rows (widened for rounding),
    // which meet at most floor((2 h + 3) / BH) + 2 bands of BH rows
    const double bands = floor((2.0 * max_half_extent_px + 3.0) / p->geo.BH) + 2.0;
    return (int32_t)(bands < p->geo.nbands ? bands : p->geo.nbands);
}

int osog_plan_bind_optics_params(osog_plan_t *p, const float *params_dev) {
    if (!p) return fail(OSOG_ERR_INVALID_ARG, "plan is NULL");
    if (reinterpret_cast<uintptr_t>(params_dev) & 3)
        return fail(OSOG_ERR_INVALID_ARG, "optics parameters not 4-byte aligned");
    p->optics_dyn = params_dev;
    return OSOG_OK;
}

int osog_sync_status(osog_plan_t *p, osog_stream_t stream) {
    if (!p) return fail(OSOG_ERR_INVALID_ARG, "plan is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(p->status_host, p->status, sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "osog_sync_status");
    return *p->status_host;
}

int64_t osog_plan_launch_count(const osog_plan_t *p) { return p ? p->launches : 0; }

int osog_profile_begin(osog_plan_t *p) {
    if (!p) return fail(OSOG_ERR_INVALID_ARG, "plan is NULL");
    p->prof = true;
    p->ev_used = 0;
    memset(p->prof_launches, 0, sizeof p->prof_launches);
    return OSOG_OK;
}

int osog_profile_end(osog_plan_t *p, osog_stream_t stream, float *ms, int32_t *launches) {
    if (!p) return fail(OSOG_ERR_INVALID_ARG, "plan is NULL");
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "osog_profile_end");
    float acc[OSOG_KERNEL_CLASS_COUNT] = {};
    for (int i = 0; i < p->ev_used; ++i) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, p->ev[2 * i], p->ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        acc[p->ev_cls[i]] += t;
    }
    for (int c = 0; c < OSOG_KERNEL_CLASS_COUNT; ++c) {
        if (ms) ms[c] = acc[c];
        if (launches) launches[c] = p->prof_launches[c];
    }
    p->prof = false;
    p->ev_used = 0;
    return OSOG_OK;
}

}  // extern "C"
