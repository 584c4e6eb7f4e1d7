// Host-side launchers of the libosog kernels (one definition per .cu file).
#pragma once

#include "osog_common.cuh"

namespace osog {

// Stage selector of the forward strip kernel.
// kStripFromReal: the strip's field is a real image [H][W] (float, read
// from opd_att), used as (value, 0) without an exit-wave step.
enum StripMode { kStripRender = 0, kStripOpdOnly = 1, kStripFromMap = 2, kStripFromReal = 3 };

struct StripArgs {
    Geometry geo;
    Work w;
    const float2 *tw;        // W-point twiddles
    const float2 *opd_att;   // kStripFromMap input [H][W] (opd, att)
    float2 *opd_out;         // kStripOpdOnly output [H][W]
    int32_t S;
    SceneDev sc[kMaxScenes];
};

struct ColumnArgs {
    Geometry geo;
    Work w;
    const float2 *tw;        // H-point twiddles
    int32_t S, K;
    int32_t unit_input;      // 1: the column spectrum is 1 everywhere (no G read, no DFT)
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
// finished strips of scene s, ctr[1 + S + s] its finished column blocks.
struct PersistArgs {
    StripArgs sa;
    ColumnArgs ca;
    InverseArgs ia;
    int32_t *ctr;      // [1 + 2 S], zero at launch
    int32_t total;     // work items
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

size_t strip_forward_smem(int W);
size_t column_smem(int H, int K);
size_t strip_inverse_smem(int W);
cudaError_t prepare_kernels(int H, int W);  // opt-in shared memory sizes
cudaError_t launch_strip_forward(const StripArgs &a, StripMode mode, cudaStream_t st);
cudaError_t launch_column(const ColumnArgs &a, cudaStream_t st);
cudaError_t launch_strip_inverse(const InverseArgs &a, cudaStream_t st);

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
