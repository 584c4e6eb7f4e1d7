// Internal definitions shared by the libosog translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "osog.h"
#include "osog_ff.h"

namespace osog {

// ---------------------------------------------------------------- layout
// Every FFT-bearing kernel works on a set of complex samples held in shared
// memory: a strip of R = set_elems(W) / W full rows, or a block of
// B = set_elems(H) / H full columns (fewer when the canvas is smaller).  A
// set of an n-point transform holds 8192 samples for n >= 1024 (8 lines at
// 1024, 4 at 2048) and kSetLines lines below that (at least kThreads
// samples), so that a single small canvas still spreads over many CTAs.
constexpr int kMaxSetElems = 8192;
constexpr int kSetLines = 4;
constexpr int kThreads = 512;          // threads of every FFT-bearing CTA
__host__ __device__ constexpr int set_elems(int n) {
    return n >= 1024 ? kMaxSetElems : kSetLines * n < kThreads ? kThreads : kSetLines * n;
}
constexpr int kChunk = 256;            // particles per binning CTA
constexpr int kMaxBands = 64;          // bands (binning rows) per canvas
constexpr int kMinBandRows = 16;       // rows of the thinnest band
constexpr int kMaxScenes = 32;         // scenes per launch group
constexpr int kMaxModes = 3;
constexpr int kMaxPlanes = 32;         // half-spaces per general polyhedron

// Shared-memory index of element i of an FFT line: one float2 of padding
// after every 16 keeps the strided Stockham accesses free of bank conflicts.
__host__ __device__ constexpr int pad16(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int line_stride(int n) { return n + (n >> 4) + 4; }

struct Geometry {
    int H, W;
    int R;        // rows per strip
    int nstrips;  // H / R
    int B;        // columns per column block
    int nblocks;  // W / B
    int BH;       // rows per binning band (multiple of R)
    int nbands;   // H / BH
};

__host__ inline Geometry make_geometry(int H, int W) {
    Geometry g;
    g.H = H;
    g.W = W;
    g.R = set_elems(W) / W < H ? set_elems(W) / W : H;
    g.nstrips = H / g.R;
    g.B = set_elems(H) / H < W ? set_elems(H) / H : W;
    g.nblocks = W / g.B;
    // At least kMinBandRows rows per band, so that a particle's bounding box
    // spans few bands (and pair lists stay short) however thin the strips.
    int bh = H / kMaxBands;
    if (bh < kMinBandRows) bh = kMinBandRows < H ? kMinBandRows : H;
    g.BH = bh > g.R ? bh : g.R;
    g.nbands = H / g.BH;
    return g;
}

// Per-particle record written by the setup pass (64 bytes).  Angles and
// inverse semi-axes are stored as float-float pairs (hi + lo), computed in
// float-float arithmetic (cos, sin to 2^-47, reciprocals to 2^-47) so that
// the ellipsoid rim can be evaluated with ~2^-44 relative error (see
// ellipse_delta_ff()).
struct __align__(16) PRec {
    float cx, cy;
    float ch, cl, sh, sl;     // cos(theta), sin(theta) hi/lo
    float p0h, p0l, p1h, p1l; // ellipsoid: 1/a, 1/b hi/lo; prism: hx, hy, -, -
    float T, dn, mu;
    float g;                  // 0 for an ellipsoid, 2 s_b dx for a prism
};
static_assert(sizeof(PRec) == 64, "PRec is 64 bytes");

// Per-particle constants of the row-span raster (48 bytes), written by the
// setup pass beside PRec.  For an ellipsoid the chord through pixel centre
// (X, Y) is t = T sqrt(1 - rho^2), and along the row Y
//   1 - rho^2 = alpha ((x0 + w - X)(X - (x0 - w))),  x0 = cx + m ey,
//   w^2 = 1/alpha - kappa ey^2,  ey = Y - cy,
// with alpha = c^2/a^2 + s^2/b^2, m = -c s (1/a^2 - 1/b^2) / alpha and
// kappa = 1 / (a^2 b^2 alpha^2) (the quadric of (u/a)^2 + (v/b)^2 in ex for
// fixed ey).  The setup pass computes them as float-float pairs, to about
// 2^-44 relative (ellipse_quadric(), in the cancellation-free form
// m = -c s (b^2 - a^2) / D, D = b^2 c^2 + a^2 s^2), so that the row's chord
// ends x0 -+ w are known to ~1e-11 px at a 100 px semi-axis, which the square
// root near the rim needs.
struct __align__(16) RRec {
    float cx, cy;
    float p[6];   // ellipsoid: m, 1/alpha, kappa (hi, lo each)
                  // prism: cos, sin, hx, hy (px), g = 2 s_b dx, T
                  // polyhedron: plane offset, plane count (int bits)
    float tsa;    // ellipsoid: T sqrt(alpha)
    float dn, mu;
    int32_t kind;
};
static_assert(sizeof(RRec) == 48, "RRec is 48 bytes");

// Bounding rectangle of the pixels a particle may touch (inclusive), or an
// empty rectangle (x0 > x1) for a skipped particle.
struct __align__(8) Rect {
    int16_t x0, x1, y0, y1;
};

// Per-scene constants of a launch group (kernel parameters, by value).
struct SceneDev {
    int32_t p0;        // first record of the scene (soa column - group base)
    int32_t n;         // particles
    int32_t chunk0;    // first binning chunk
    int32_t pair0;     // first slot of the scene's pair region
    int32_t pair_cap;  // slots reserved for the scene
    float two_over_lambda;
    float prism_g;     // 2 s_b dx
    float dx_um;       // pixel pitch (um)
};

// Transfer-function constants of one (scene, modality).
struct ModeDev {
    double r2;            // (NA / lambda)^2, cycles^2 / um^2
    double ox, oy;        // pupil centre shift (cycles / um)
    double fx_scale;      // 1 / (W dx)
    double fy_span;       // H dx (um): signed row index per cycle/um
    float kstep_x, kstep_y;  // 2 pi / (W dx), 2 pi / (H dx)
    float qoff_x, qoff_y;    // 2 pi (ox, oy)
    float k0, dz;
    float dsx, dsy, bias;
    float scale;          // 1 / (H W)
    int32_t dic;          // 1 for the DIC factor
    float dsx1, dsy1;     // d(dsx, dsy) / d(shear_px): dx (cos, sin)(shear_angle) / 2
    int32_t op;           // kOpPupil, kOpAllPass, kOpTable or kOpSpectrum
    float2 *tab;          // kOpTable: multiplier table; kOpSpectrum: output
                          // (both column-blocked [W/B][H][B] like Q)
    const float *dyn;     // bound optics scalars (defocus_um, shear_px, shear_angle,
                          // bias_phase) read when the kernel runs; null: dz .. bias above
    float half_dx;        // dx / 2 (um): dsx, dsy of the bound shear
    int32_t fixed_dz;     // 1: dz stays as set here whatever is bound (an operation
                          // that applies no defocus)
};

// The modality with the plan's bound optics scalars applied (see
// osog_plan_bind_optics_params): defocus, DIC shear and bias are read from
// device memory when the kernel runs, so a replayed CUDA graph sees values
// updated on the device between replays.
__device__ __forceinline__ ModeDev live_mode(const ModeDev &m) {
    ModeDev r = m;
    if (m.dyn) {
        const float sp = m.dyn[1];
        float sa, ca;
        sincosf(m.dyn[2], &sa, &ca);
        if (!m.fixed_dz) r.dz = m.dyn[0];
        r.dsx = m.half_dx * sp * ca;
        r.dsy = m.half_dx * sp * sa;
        r.dsx1 = m.half_dx * ca;
        r.dsy1 = m.half_dx * sa;
        r.bias = m.dyn[3];
    }
    return r;
}

// What the column pass does with one (scene, modality):
//   kOpPupil     multiply by the transfer function inside the pupil chord
//   kOpAllPass   the same transfer function (without the pupil circle) on
//                every frequency
//   kOpTable     multiply every frequency by tab / tab[0] (real DC term)
//   kOpSpectrum  write the forward column spectrum times scale to tab (no
//                inverse transform, Q untouched)
//   kOpLoss      the image losses of inverse rendering (see LossDev): per
//                frequency their terms, summed per column block, and the
//                complex gradient of their weighted sum, inverse-transformed
//                to Q (tab holds the target's spectrum)
enum { kOpPupil = 0, kOpAllPass = 1, kOpTable = 2, kOpSpectrum = 3, kOpLoss = 4 };

// Parameters of kOpLoss, the same for every image of a launch.  With A the
// image's unnormalised spectrum and B the target's:
//   misfit    scale / (H W) sum_{|f| <= cutoff} |A - B|^2 (the low-pass
//             image misfit by Parseval), gradient term 2 scale / (H W) (A - B);
//   spectral  1 / ntot sum_f (log(|A| + e) - log(|B| + e))^2 (Eq. 8), e =
//             eps_rel max|B| of that image, gradient term weight 2 d A /
//             (ntot |A| (|A| + e)).
struct LossDev {
    const float *cutoff;    // device scalar: low-pass radius (cycles / um); null: misfit off
    float misfit_scale;
    float spectral_weight;  // 0: spectral loss off
    float eps_rel;
    float inv_ntot;         // 1 / (K H W)
    float fx_scale, fy_scale;  // 1 / (W dx), 1 / (H dx): cycles / um per index
    const float *maxamp;    // [images] largest target amplitude
    float *part;            // [images][blocks][2] per-block sums (misfit, spectral)
};

struct GroupDev {
    int32_t S;
    int32_t K;
    int32_t nchunks;               // total binning chunks
    int32_t pad_;
    SceneDev sc[kMaxScenes];
    ModeDev md[kMaxScenes][kMaxModes];
};

// Pointers into the workspace for one launch group.
struct Work {
    PRec *rec;
    RRec *rrec;         // row-span raster constants, one per record
    Rect *rect;
    int32_t *cnt;       // [nchunks][nbands]: counts, then exclusive prefix
    int32_t *band_off;  // [S][nbands + 1]
    int32_t *pairs;     // record indices, per band, ascending
    Rect *pair_rect = nullptr;  // per pair slot: the record's rectangle, its kind in bits
                        // 12-13 of x1 (null: readers gather rect[] and rrec[])
    float2 *G;          // [S][W/B][H][B] row spectra
    float2 *Q;          // [S][K][W/B][H][B] filtered columns
    int2 *colrange;     // [S] signed column frequencies [lo, hi] outside which no
                        // pupil passes anything (a hull, possibly wider)
    int32_t *slotmap;   // [n][pairs per particle] band-list slot of each (particle,
                        // band); written by the fill pass when not null (adjoint)
    int32_t slotmap_ppp;
    int32_t *status;    // plan status word
    // General polyhedra (kind 2): the caller's planes (a_x, a_y, a_z, b),
    // per-particle row offsets [n + 1], and their per-particle pixel-affine
    // bounds written by the setup pass (see setup_particle()).
    const float4 *planes = nullptr;
    const int32_t *plane_off = nullptr;
    int32_t n_planes = 0;
    float4 *plane_coef = nullptr;
};

// ---------------------------------------------------------------- pupil
// Interval [lo, hi] of signed row frequencies fy inside the (shifted) pupil
// circle for column frequency fx, decided in double precision:
// (fx / (W dx) + ox)^2 + (fy / (H dx) + oy)^2 <= (NA / lambda)^2.
// An empty column returns lo > hi.
__device__ __forceinline__ int2 pupil_chord(const ModeDev &md, int fx) {
    const double ax = (double)fx * md.fx_scale + md.ox;
    const double rem = md.r2 - ax * ax;
    if (rem < 0.0) return make_int2(1, 0);
    const double root = sqrt(rem);
    const double lo = (-root - md.oy) * md.fy_span;
    const double hi = (root - md.oy) * md.fy_span;
    return make_int2((int)ceil(lo), (int)floor(hi));
}

// Rows [lo, hi] of column fx (signed) that a modality's column operation
// touches on an H-row canvas: the pupil chord, or the whole column for the
// operations without a pupil circle.
__device__ __forceinline__ int2 mode_chord(const ModeDev &md, int fx, int H) {
    return md.op == kOpPupil ? pupil_chord(md, fx) : make_int2(-H / 2, H / 2 - 1);
}

// ---------------------------------------------------------------- launches
// Programmatic dependent launch.  Every kernel of the render and adjoint
// chains starts with pdl_enter(): it first lets the next kernel of the
// stream be dispatched (once all CTAs of this grid have done the same), then
// waits until the kernels before it in the stream have completed and their
// writes are visible.  Nothing is read from global memory before the wait,
// so the overlap covers launch and CTA dispatch only.  Launched without the
// attribute (launch_chain), or after other stream work, the wait returns at
// once.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launch of a chain kernel, with programmatic stream serialization allowed
// for grids of at most kPdlMaxCtas CTAs: it shortens chains of small,
// latency-bound launches (one scene), while for grids of many waves (the
// batched path) the early dispatch measured slower.
constexpr long kPdlMaxCtas = 1024;
template <typename... KArgs, typename... Args>
inline cudaError_t launch_chain(void (*kernel)(KArgs...), dim3 grid, int block, size_t smem,
                                cudaStream_t st, Args &&...args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = (long)grid.x * grid.y * grid.z <= kPdlMaxCtas ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
    if (e != cudaSuccess) (void)cudaGetLastError();  // reported once, by the return value
    return e;
}

// ---------------------------------------------------------------- status
__device__ __forceinline__ void latch(int32_t *status, int code) {
    atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// The products are written as one rounded product and one fused
// multiply-add, so that every kernel that inlines them rounds alike
// (the compiler cannot contract them differently in different kernels).
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -__fmul_rn(a.y, b.y)), fmaf(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(fmaf(a.x, b.x, __fmul_rn(a.y, b.y)), fmaf(a.y, b.x, -__fmul_rn(a.x, b.y)));
}

// ---------------------------------------------------------------- float-float
// struct ff and its error-free transformations: osog_ff.h.

// ---------------------------------------------------------------- geometry
// 1 - rho^2 of an ellipsoid at pixel centre (x, y) in float-float, from the
// float-float record: u = c ex + s ey, v = -s ex + c ey, rho^2 = (u/a)^2 +
// (v/b)^2 with ex = x - cx taken exactly (TwoSum).  Used where the float32
// value of 1 - rho^2 is small: there the float32 rounding of rho^2 (~2e-7)
// would put an error of order T sqrt(2e-7) on the thickness T sqrt(1 - rho^2).
__device__ __forceinline__ float ellipse_delta_ff(const PRec &r, float x, float y) {
    ff exf = two_sum(x, -r.cx);
    ff eyf = two_sum(y, -r.cy);
    ff c = {r.ch, r.cl}, s = {r.sh, r.sl};
    ff uf = ff_add(ff_mul(c, exf), ff_mul(s, eyf));
    ff vf = ff_add(ff_mul(c, eyf), ff_neg(ff_mul(s, exf)));
    ff uaf = ff_mul(uf, ff{r.p0h, r.p0l});
    ff vbf = ff_mul(vf, ff{r.p1h, r.p1l});
    ff rho2 = ff_add(ff_mul(uaf, uaf), ff_mul(vbf, vbf));
    ff d = ff_add(ff{1.f, 0.f}, ff_neg(rho2));
    return d.h + d.l;
}

// Band of 1 - rho^2 (float32) inside which the ellipsoid is re-evaluated in
// float-float.  Outside it the float32 error of the thickness is below
// T * 5e-7 / (2 sqrt(4e-3)) ~ 4e-6 T.
constexpr float kRimBand = 4e-3f;

}  // namespace osog
