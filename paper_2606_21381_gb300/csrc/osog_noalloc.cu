// osog_render_noalloc: the forward render with its scratch memory in a
// fixed static device array instead of a caller-provided workspace.
//
// Some callers cannot allocate device memory at all: code running under an
// allocator that forbids cudaMalloc outside start-up, plugins that must not
// grow a host application's memory footprint, or real-time loops that may
// not block on an allocation.  They cannot create a plan (plan creation
// allocates twiddle tables and a status word) nor own a workspace.  This
// entry point serves them: the twiddle tables, the status word and all
// intermediate buffers (particle records, band bins, row spectra, filtered
// columns) live in file-scope static __device__ arrays that every GPU which
// loads the library holds until the process exits.  The caller still passes
// the particle tensor and the output image.
#include <math.h>
#include <mutex>

#include "osog_fft.cuh"
#include "osog_kernels.h"

using namespace osog;

namespace {

constexpr size_t kScratchBytes = (size_t)8 << 20;  // 8 MiB of intermediate buffers
constexpr int kTwiddleCount = 32 + 64 + 128 + 256 + 512 + 1024 + 2048;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) float2 g_twiddles[kTwiddleCount];  // tables of sizes 32..2048
static __device__ __align__(256) int32_t g_status;

struct DeviceState {
    bool ready = false;
    unsigned char *scratch = nullptr;  // device address of g_scratch
    float2 *twiddles = nullptr;        // device address of g_twiddles
    int32_t *status = nullptr;         // device address of g_status
};

std::mutex g_setup_lock;
DeviceState g_state[kMaxDevices];

int twiddle_offset(int n) {  // start of the n-point table inside g_twiddles
    int off = 0;
    for (int m = 32; m < n; m <<= 1) off += m;
    return off;
}

// Once per device, with that device current: resolve the device addresses
// of the static arrays (their names are only host-side stand-ins in host
// code), upload the FP64-built twiddle tables and opt the kernels in to
// their shared-memory sizes.  No device memory is allocated.
int setup_device(int dev, DeviceState **out) {
    std::lock_guard<std::mutex> guard(g_setup_lock);
    DeviceState &st = g_state[dev];
    if (!st.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return OSOG_ERR_CUDA;
        st.scratch = static_cast<unsigned char *>(p);
        if (cudaGetSymbolAddress(&p, g_twiddles) != cudaSuccess) return OSOG_ERR_CUDA;
        st.twiddles = static_cast<float2 *>(p);
        if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return OSOG_ERR_CUDA;
        st.status = static_cast<int32_t *>(p);
        static float2 host_tw[kTwiddleCount];
        for (int n = 32; n <= 2048; n <<= 1) fill_twiddles(n, host_tw + twiddle_offset(n));
        if (cudaMemcpyToSymbol(g_twiddles, host_tw, sizeof host_tw) != cudaSuccess)
            return OSOG_ERR_CUDA;
        for (int n = 32; n <= 2048; n <<= 1)
            if (prepare_kernels(n, n) != cudaSuccess) return OSOG_ERR_CUDA;
        st.ready = true;
    }
    *out = &st;
    return OSOG_OK;
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

bool pow2_ok(int v) { return v >= 32 && v <= 2048 && (v & (v - 1)) == 0; }

}  // namespace

extern "C" int osog_render_noalloc(const float *soa, int64_t ld, int32_t n,
                                   const osog_optics_t *o, float *image,
                                   osog_stream_t stream) {
    if (!o || !image || n < 0 || (int64_t)n > ld || (n > 0 && !soa)) return OSOG_ERR_INVALID_ARG;
    if (!pow2_ok(o->H) || !pow2_ok(o->W)) return OSOG_ERR_UNSUPPORTED_SIZE;
    const double v[] = {o->dx_um, o->lambda_um, o->NA, o->n_medium, o->defocus_um,
                        o->oblique_frac, o->oblique_angle, o->shear_px, o->shear_angle,
                        o->bias_phase, o->bevel_slope};
    for (double x : v)
        if (!isfinite(x)) return OSOG_ERR_INVALID_ARG;
    if (!(o->dx_um > 0) || !(o->lambda_um > 0) || !(o->NA > 0) || !(o->n_medium >= o->NA) ||
        !(o->bevel_slope > 0) || o->modes == 0 || (o->modes & ~7u))
        return OSOG_ERR_INVALID_ARG;
    const int K = (int)(o->modes & 1u) + (int)((o->modes >> 1) & 1u) + (int)((o->modes >> 2) & 1u);
    const Geometry geo = make_geometry(o->H, o->W);

    // Scratch layout (the regions of an osog_render workspace).  The band
    // lists come last and take whatever the other regions leave, up to the
    // most a scene can need (every particle in every band).
    const int64_t chunks = ((int64_t)n + kChunk - 1) / kChunk;
    size_t off = 0;
    const size_t o_rec = off;
    off = up256(off + (size_t)n * sizeof(PRec));
    const size_t o_rrec = off;
    off = up256(off + (size_t)n * sizeof(RRec));
    const size_t o_rect = off;
    off = up256(off + (size_t)n * sizeof(Rect));
    const size_t o_cnt = off;
    off = up256(off + (size_t)chunks * geo.nbands * sizeof(int32_t));
    const size_t o_band = off;
    off = up256(off + (size_t)(geo.nbands + 1) * sizeof(int32_t));
    const size_t o_G = off;
    off = up256(off + (size_t)geo.H * geo.W * sizeof(float2));
    const size_t o_Q = off;
    off = up256(off + (size_t)K * geo.H * geo.W * sizeof(float2));
    const size_t o_colrange = off;
    off = up256(off + sizeof(int2));
    const size_t o_pairs = off;
    if (off > kScratchBytes || (n > 0 && kScratchBytes - off < (size_t)n * sizeof(int32_t)))
        return OSOG_ERR_WORKSPACE;  // beyond the 8 MiB static scratch
    const int64_t pair_room = (int64_t)((kScratchBytes - off) / sizeof(int32_t));
    const int64_t pair_most = (int64_t)n * geo.nbands;
    const int64_t pairs = pair_room < pair_most ? pair_room : pair_most;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return OSOG_ERR_CUDA;
    DeviceState *st = nullptr;
    int rc = setup_device(dev, &st);
    if (rc) return rc;

    Work w;
    w.rec = reinterpret_cast<PRec *>(st->scratch + o_rec);
    w.rrec = reinterpret_cast<RRec *>(st->scratch + o_rrec);
    w.rect = reinterpret_cast<Rect *>(st->scratch + o_rect);
    w.cnt = reinterpret_cast<int32_t *>(st->scratch + o_cnt);
    w.band_off = reinterpret_cast<int32_t *>(st->scratch + o_band);
    w.pairs = reinterpret_cast<int32_t *>(st->scratch + o_pairs);
    w.G = reinterpret_cast<float2 *>(st->scratch + o_G);
    w.Q = reinterpret_cast<float2 *>(st->scratch + o_Q);
    w.colrange = reinterpret_cast<int2 *>(st->scratch + o_colrange);
    w.slotmap = nullptr;
    w.slotmap_ppp = 0;
    w.status = st->status;

    // Scene and transfer-function constants (double precision on the host).
    GroupDev gd{};
    gd.S = 1;
    gd.K = K;
    gd.nchunks = (int32_t)chunks;
    SceneDev &sc = gd.sc[0];
    sc = scene_dev(*o);
    sc.p0 = 0;
    sc.n = n;
    sc.chunk0 = 0;
    sc.pair0 = 0;
    sc.pair_cap = (int32_t)pairs;
    for (int bit = 0, k = 0; bit < 3; ++bit)
        if (o->modes & (1u << bit)) gd.md[0][k++] = mode_dev(*o, 1u << bit, nullptr);

    // Every scratch region is written in full before it is read; the status
    // word keeps what earlier calls latched until osog_noalloc_sync_status.
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float2 *tw_w = st->twiddles + twiddle_offset(o->W);
    const float2 *tw_h = st->twiddles + twiddle_offset(o->H);
    if (launch_bin_count(soa, ld, gd, geo, w, s) != cudaSuccess) return OSOG_ERR_CUDA;
    if (launch_bin_scan(gd, geo, w, s) != cudaSuccess) return OSOG_ERR_CUDA;
    if (launch_bin_fill(gd, geo, w, s) != cudaSuccess) return OSOG_ERR_CUDA;
    StripArgs sa{};
    sa.geo = geo;
    sa.w = w;
    sa.tw = tw_w;
    sa.S = 1;
    sa.sc[0] = sc;
    if (launch_strip_forward(sa, kStripRender, s) != cudaSuccess) return OSOG_ERR_CUDA;
    ColumnArgs ca{};
    ca.geo = geo;
    ca.w = w;
    ca.tw = tw_h;
    ca.S = 1;
    ca.K = K;
    for (int m = 0; m < K; ++m) ca.md[0][m] = gd.md[0][m];
    if (launch_column(ca, s) != cudaSuccess) return OSOG_ERR_CUDA;
    InverseArgs ia{};
    ia.geo = geo;
    ia.w = w;
    ia.tw = tw_w;
    ia.images = image;
    ia.S = 1;
    ia.K = K;
    if (launch_strip_inverse(ia, s) != cudaSuccess) return OSOG_ERR_CUDA;
    return OSOG_OK;
}

extern "C" int osog_noalloc_sync_status(osog_stream_t stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return OSOG_ERR_CUDA;
    DeviceState *st = nullptr;
    int rc = setup_device(dev, &st);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int32_t code = 0;  // pageable: the copy below completes before it returns
    if (cudaStreamSynchronize(s) != cudaSuccess) return OSOG_ERR_CUDA;
    if (cudaMemcpy(&code, st->status, sizeof code, cudaMemcpyDeviceToHost) != cudaSuccess)
        return OSOG_ERR_CUDA;
    if (cudaMemset(st->status, 0, sizeof(int32_t)) != cudaSuccess) return OSOG_ERR_CUDA;
    return code;
}
