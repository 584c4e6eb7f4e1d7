// Host-side launchers of the libosog kernels (one definition per .cu file).
#pragma once

#include <math.h>

#include "osog_common.cuh"

namespace osog {

// Stage selector of the forward strip kernel.
// kStripFromReal: the strip's field is a real image [H][W] (float, read
// from opd_att), used as (value, 0) without an exit-wave step.
// kStripFromPhase: the strip's exit wave from the fixed-point phase and
// absorption words that the tile raster wrote (StripArgs.phase).
enum StripMode { kStripRender = 0, kStripOpdOnly = 1, kStripFromMap = 2, kStripFromReal = 3,
                 kStripFromPhase = 4 };

struct StripArgs {
    Geometry geo;
    Work w;
    const float2 *tw;        // W-point twiddles
    const float2 *opd_att;   // kStripFromMap input [H][W] (opd, att)
    float2 *opd_out;         // kStripOpdOnly output [H][W]
    const uint2 *phase;      // kStripFromPhase input [S][H][W]
    int32_t S;
    SceneDev sc[kMaxScenes];
};

// The tile raster: one CTA per tile of BH rows (one binning band) by TW
// columns of one scene; writes the tile's fixed-point phase and absorption
// words (see raster_region) to P [S][H][W].
struct RasterArgs {
    Geometry geo;
    Work w;
    uint2 *P;
    int32_t S;
    int32_t TW;
    SceneDev sc[kMaxScenes];
};

struct ColumnArgs {
    Geometry geo;
    Work w;
    const float2 *tw;        // H-point twiddles
    int32_t S, K;
    int32_t unit_input;      // 1: the column spectrum is 1 everywhere (no G read, no DFT)
    int32_t wait_polls;      // bulk-copy wait: polls before it gives up (0: the default)
    int32_t wait_extra;      // failure-detection test: the bulk-copy barrier expects 16
                             // bytes more than arrive, so its wait runs out
    LossDev loss;            // kOpLoss parameters
    ModeDev md[kMaxScenes][kMaxModes];
};

struct InverseArgs {
    Geometry geo;
    Work w;
    const float2 *tw;        // W-point twiddles
    float *images;           // [S][K][H][W]
    int32_t S, K;
    int32_t real_out;        // 1: write Re(E) instead of |E|^2
};

// The three render stages of a launch group in one persistent launch
// (square canvases).  ctr[0] hands out work items; ctr[1 + s] counts the
// finished strips of scene s, ctr[1 + S + s] its finished column blocks;
// ctr[1 + 2 S] is raised when a wait of the launch gives up.
struct PersistArgs {
    StripArgs sa;
    ColumnArgs ca;
    InverseArgs ia;
    int32_t *ctr;      // [2 + 2 S], zero at launch
    int32_t total;     // work items
    int32_t wait_polls;   // polls before a wait gives up (latching OSOG_ERR_TIMEOUT)
    int32_t wait_extra;   // failure-detection test: added to the column items' target
};

// Adjoint passes (osog_render_backward).
struct BwdRowsArgs {  // dL/dQ_m = DFT_rows(2 gI_m E_m), written over Q_m
    Geometry geo;
    Work w;
    const float2 *tw;          // W-point tables
    const float *grad_image;   // [S][K][H][W]
    int32_t S, K;
};

struct BwdColumnArgs {  // dL/dG = IDFT_cols(sum_m conj(H_m) DFT_cols(dL/dQ_m)), over G
    Geometry geo;
    Work w;
    const float2 *tw;          // H-point tables
    float *opart;              // [S][W/B][4] per-block optics partials
    int32_t S, K;
    ModeDev md[kMaxScenes][kMaxModes];
};

struct BwdStripArgs {  // per-(band slot, strip) particle partials
    Geometry geo;
    Work w;
    const float2 *tw;          // W-point tables
    float *part;               // [pair slots][strips per band][8]
    int32_t S;
    SceneDev sc[kMaxScenes];
};

struct BwdReduceArgs {  // fixed-order sums into the particle and optics gradients
    Geometry geo;
    Work w;
    const float *part;
    const float *opart;
    float *grad_soa;           // [9][ld], columns of this group
    int64_t ld;
    float *grad_optics;        // [S][4]
    int32_t S, nchunks;
    SceneDev sc[kMaxScenes];
};

// Host: the scene constants of one optics struct (the caller fills in the
// launch fields p0, n, chunk0, pair0 and pair_cap), and the transfer-
// function constants of one modality bit, in double precision rounded
// once.  dyn is the plan's bound optics array (or null).
inline SceneDev scene_dev(const osog_optics_t &o) {
    SceneDev s{};
    s.two_over_lambda = (float)(2.0 / o.lambda_um);
    s.prism_g = (float)(2.0 * o.bevel_slope * o.dx_um);
    s.dx_um = (float)o.dx_um;
    return s;
}

inline ModeDev mode_dev(const osog_optics_t &o, uint32_t mode, const float *dyn) {
    const double two_pi = 6.283185307179586476925286766559;
    ModeDev m{};
    const double r = o.NA / o.lambda_um;
    m.r2 = r * r;
    m.ox = m.oy = 0.0;
    if (mode == OSOG_MODE_OBLIQUE) {
        m.ox = o.oblique_frac * r * cos(o.oblique_angle);
        m.oy = o.oblique_frac * r * sin(o.oblique_angle);
    }
    m.fx_scale = 1.0 / ((double)o.W * o.dx_um);
    m.fy_span = (double)o.H * o.dx_um;
    m.kstep_x = (float)(two_pi / ((double)o.W * o.dx_um));
    m.kstep_y = (float)(two_pi / ((double)o.H * o.dx_um));
    m.qoff_x = (float)(two_pi * m.ox);
    m.qoff_y = (float)(two_pi * m.oy);
    m.k0 = (float)(two_pi * o.n_medium / o.lambda_um);
    m.dz = (float)o.defocus_um;
    m.dsx = (float)(0.5 * o.shear_px * o.dx_um * cos(o.shear_angle));
    m.dsy = (float)(0.5 * o.shear_px * o.dx_um * sin(o.shear_angle));
    m.bias = (float)o.bias_phase;
    m.scale = (float)(1.0 / ((double)o.H * o.W));
    m.dic = mode == OSOG_MODE_DIC ? 1 : 0;
    m.dsx1 = (float)(0.5 * o.dx_um * cos(o.shear_angle));
    m.dsy1 = (float)(0.5 * o.dx_um * sin(o.shear_angle));
    m.dyn = dyn;
    m.half_dx = (float)(0.5 * o.dx_um);
    return m;
}

cudaError_t launch_bin_count(const float *soa, int64_t ld, const GroupDev &gd,
                             const Geometry &geo, const Work &w, cudaStream_t st);
cudaError_t launch_bin_scan(const GroupDev &gd, const Geometry &geo, const Work &w,
                            cudaStream_t st);
cudaError_t launch_bin_fill(const GroupDev &gd, const Geometry &geo, const Work &w,
                            cudaStream_t st);
// count + scan + fill in one launch for a single scene of one chunk
// (1..kChunk particles); same results as the three launches
cudaError_t launch_bin_single(const float *soa, int64_t ld, const GroupDev &gd,
                              const Geometry &geo, const Work &w, cudaStream_t st);

size_t strip_forward_smem(int W, bool opd_mode = false);  // opd_mode: kStripOpdOnly
size_t column_smem(int H, int K);
size_t strip_inverse_smem(int W);
cudaError_t prepare_kernels(int H, int W);  // opt-in shared memory sizes
cudaError_t launch_strip_forward(const StripArgs &a, StripMode mode, cudaStream_t st);
cudaError_t launch_column(const ColumnArgs &a, cudaStream_t st);
cudaError_t launch_strip_inverse(const InverseArgs &a, cudaStream_t st);
int raster_tile_cols(const Geometry &geo);  // TW of the tile raster
cudaError_t launch_raster_tiles(const RasterArgs &a, cudaStream_t st);
// largest |spectrum| of each of S column-blocked H x W spectra (one CTA each)
cudaError_t launch_max_amplitude(const float2 *spec, int S, int64_t count, float *maxamp,
                                 cudaStream_t st);
// fixed-order sums of kOpLoss's per-block partials into loss[0] (misfit)
// and loss[1] (spectral loss)
cudaError_t launch_loss_reduce(const float *part, int64_t nparts, float *loss, cudaStream_t st);

size_t persistent_smem(int N, int K);
cudaError_t launch_persistent(const PersistArgs &a, cudaStream_t st);

size_t bwd_column_smem(int H);
size_t bwd_strip_smem(int W);
cudaError_t prepare_backward(int H, int W);
cudaError_t launch_bwd_rows(const BwdRowsArgs &a, cudaStream_t st);
cudaError_t launch_bwd_column(const BwdColumnArgs &a, cudaStream_t st);
cudaError_t launch_bwd_strip(const BwdStripArgs &a, cudaStream_t st);
cudaError_t launch_bwd_reduce(const BwdReduceArgs &a, cudaStream_t st);

}  // namespace osog
