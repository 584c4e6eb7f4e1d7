// Host-side launchers of the libosog kernels (one definition per .cu file).
#pragma once

#include "osog_common.cuh"

namespace osog {

// Stage selector of the forward strip kernel.
enum StripMode { kStripRender = 0, kStripOpdOnly = 1, kStripFromMap = 2 };

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
    ModeDev md[kMaxScenes][kMaxModes];
};

struct InverseArgs {
    Geometry geo;
    Work w;
    const float2 *tw;        // W-point twiddles
    float *images;           // [S][K][H][W]
    int32_t S, K;
};

cudaError_t launch_bin_count(const float *soa, int64_t ld, const GroupDev &gd,
                             const Geometry &geo, const Work &w, cudaStream_t st);
cudaError_t launch_bin_scan(const GroupDev &gd, const Geometry &geo, const Work &w,
                            cudaStream_t st);
cudaError_t launch_bin_fill(const GroupDev &gd, const Geometry &geo, const Work &w,
                            cudaStream_t st);

size_t strip_forward_smem(int W);
size_t column_smem(int H, int K);
size_t strip_inverse_smem(int W);
cudaError_t prepare_kernels(int H, int W);  // opt-in shared memory sizes
cudaError_t launch_strip_forward(const StripArgs &a, StripMode mode, cudaStream_t st);
cudaError_t launch_column(const ColumnArgs &a, cudaStream_t st);
cudaError_t launch_strip_inverse(const InverseArgs &a, cudaStream_t st);

}  // namespace osog
