// Render kernels: raster + exit wave + row FFT, column pass with the
// optical head, inverse row FFT + intensity.
//
// Data flow for one H x W scene (complex64 intermediates in HBM):
//   strip forward  (CTA per strip of R = set_elems(W)/W rows): gathers the OPD and
//                  ATT of every particle overlapping the strip in ascending
//                  particle order (Eq. 2, Eq. 7), forms the exit wave
//                  exp(-ATT) exp(i 2 pi OPD / lambda) (Eq. 2, Eq. 4), runs
//                  the forward row DFTs and writes G in a column-blocked
//                  layout [W/B][H][B] so that the column pass reads one
//                  contiguous block.
//   column         (CTA per block of B = set_elems(H)/H columns): forward column
//                  DFTs, then for every modality the transfer function of
//                  Eq. 3 / Eq. 5 / oblique shift times 1/(HW), inverse column
//                  DFTs, written as Q[m] in the same blocked layout.
//   strip inverse  (CTA per strip and modality): inverse row DFTs and
//                  I = |E|^2 (Sec. III.B), float32 image rows.
#include <math.h>

#include "osog_strip.cuh"

namespace osog {

namespace {

// The FFT passes of the sets of 8192 samples run with one thread group per
// line (named barriers) instead of CTA-wide barriers.
constexpr bool kGroupFft = true;

// One strip (rows [strip R, strip R + R)) of scene s.
template <int N, int MODE, bool SQ = false>
__device__ __forceinline__ void strip_forward_item(const StripArgs &a, int s, int strip,
                                                   unsigned char *smem_raw) {
    constexpr int L = set_elems(N) / N;
    constexpr int LS = line_stride(N);
    constexpr int ACC = MODE == kStripOpdOnly ? kAccOpd : kAccPhase;
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    // accumulators: one uint2 per padded slot (phase mode) or two int64 (OPD mode)
    unsigned char *scratch = smem_raw + (ACC == kAccOpd ? 2 : 1) * L * LS * sizeof(float2);
    const Geometry &geo = a.geo;
    const int R = SQ ? sq_rb(N) : geo.R;
    const int y0 = strip * R;
    const int RN = R * N;  // <= set_elems(N); lines R..L-1 are never read back
    if constexpr (MODE == kStripFromReal) {
        const float *src = reinterpret_cast<const float *>(a.opd_att) + ((size_t)s * geo.H + y0) * N;
        float v[ept(N)];
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            if (e < RN) v[i] = src[e];
        }
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            if (e < RN) buf[(e / N) * LS + pad16(e % N)] = make_float2(v[i], 0.f);
        }
    } else if constexpr (MODE == kStripFromPhase) {
        const uint2 *src = a.phase + ((size_t)s * geo.H + y0) * N;
        uint2 v[ept(N)];
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            if (e < RN) v[i] = src[e];
        }
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            if (e < RN) buf[(e / N) * LS + pad16(e % N)] = exit_wave_fixed(v[i]);
        }
    } else if constexpr (MODE == kStripFromMap) {
        const float2 *src = a.opd_att + (size_t)y0 * N;
        float2 v[ept(N)];
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            if (e < RN) v[i] = src[e];
        }
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            if (e < RN) buf[(e / N) * LS + pad16(e % N)] = v[i];
        }
    } else {
        float4 *b4 = reinterpret_cast<float4 *>(buf);
        const int n4 = (ACC == kAccOpd ? 2 : 1) * R * LS / 2;
        for (int i = threadIdx.x; i < n4; i += kThreads) b4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        raster_strip<N, ACC>(a.geo, a.w, a.sc[s], s, y0, R, smem_raw, scratch);
    }
    __syncthreads();
    if constexpr (MODE == kStripRender) {
        // the exit wave of the accumulated words is formed as the first FFT
        // pass loads them, and the last pass stores G (column-blocked, only
        // the columns some pupil passes)
        constexpr bool GRP = kGroupFft && fft_grouped(N);
        fft_first_pass<N, L, false, true, GRP>(buf, [&](int l, int x) -> float2 {
            return l < R ? exit_wave_fixed(*reinterpret_cast<const uint2 *>(buf + l * LS + pad16(x)))
                         : make_float2(0.f, 0.f);
        });
        fft_pass_range<N, L, false, 1, fft_passes(N) - 1, GRP>(buf, a.tw);
        const int B = SQ ? sq_rb(N) : geo.B;
        const int lb = SQ ? clog2(sq_rb(N)) : ilog2(B);
        const int H = SQ ? N : geo.H;
        float2 *G = a.w.G + (size_t)s * H * N;
        const int2 cr = a.w.colrange[s];
        fft_last_pass<N, L, false, false, GRP>(buf, a.tw, [&](int l, int kx, float2 v) {
            const int fx = kx < N / 2 ? kx : kx - N;
            if (l < R && fx >= cr.x && fx <= cr.y)  // columns outside every pupil are never read
                G[((size_t)(kx >> lb) * H + y0 + l) * B + (kx & (B - 1))] = v;
        });
        return;
    } else if constexpr (MODE == kStripOpdOnly) {
        const longlong2 *acc = reinterpret_cast<const longlong2 *>(smem_raw);
        float2 *dst = a.opd_out + (size_t)y0 * N;
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            if (e < RN) {
                const longlong2 v = acc[(e / N) * LS + pad16(e % N)];
                dst[e] = make_float2(__ll2float_rn(v.x) * 2.3283064365386963e-10f,
                                     __ll2float_rn(v.y) * 2.3283064365386963e-10f);  // 2^-32
            }
        }
        return;
    } else {
        if constexpr (MODE == kStripFromMap) {
            const float tol = a.sc[s].two_over_lambda;
#pragma unroll
            for (int i = 0; i < ept(N); ++i) {
                const int e = threadIdx.x + i * kThreads;
                if (e < RN) {
                    float2 *v = buf + (e / N) * LS + pad16(e % N);
                    const float2 oa = *v;
                    *v = oa.x != 0.f || oa.y != 0.f ? exit_wave(oa.x, oa.y, tol)
                                                    : make_float2(1.f, 0.f);
                }
            }
        }
        __syncthreads();
        fft_lines<N, L, false>(buf, a.tw);
        const int B = SQ ? sq_rb(N) : geo.B;
        const int lb = SQ ? clog2(sq_rb(N)) : ilog2(B), lr = SQ ? clog2(sq_rb(N)) : ilog2(R);
        const int H = SQ ? N : geo.H;
        float2 *G = a.w.G + (size_t)s * H * N;
        const int2 cr = a.w.colrange[s];
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            const int c = e & (B - 1), r = (e >> lb) & (R - 1), bk = e >> (lb + lr);
            const int kx = bk * B + c, fx = kx < N / 2 ? kx : kx - N;
            if (e < RN && fx >= cr.x && fx <= cr.y)  // columns outside every pupil are never read
                G[((size_t)bk * H + y0 + r) * B + c] = buf[r * LS + pad16(kx)];
        }
    }
}

// ------------------------------------------------------------ tile raster
constexpr int kRThreads = 256;

__global__ void __launch_bounds__(kRThreads, 4) k_raster_tiles(const __grid_constant__ RasterArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_enter();
    const Geometry &geo = a.geo;
    const int s = blockIdx.z, band = blockIdx.y;
    const int TW = a.TW, TH = geo.BH;
    const int tx0 = blockIdx.x * TW, ty0 = band * TH;
    uint2 *acc = reinterpret_cast<uint2 *>(smem_raw);
    unsigned char *scratch = smem_raw + (size_t)TH * TW * sizeof(uint2);
    uint4 *a4 = reinterpret_cast<uint4 *>(acc);
    for (int i = threadIdx.x; i < TH * TW / 2; i += kRThreads) a4[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const SceneDev &sc = a.sc[s];
    const int32_t *off = a.w.band_off + (size_t)s * (geo.nbands + 1);
    const int hi = min(off[band + 1], sc.pair_cap);
    const int lo = min(off[band], hi);
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(acc);
    auto slot = [base, TW, tx0](int row, int x) -> uint32_t {
        return base + (uint32_t)(row * TW + (x - tx0)) * 8u;
    };
    raster_region<kRThreads, kAccPhase>(a.w, a.w.pairs + sc.pair0,
                                        a.w.pair_rect ? a.w.pair_rect + sc.pair0 : nullptr, lo, hi, ty0, TH, tx0,
                                        tx0 + TW - 1, 0.5f * sc.two_over_lambda, slot, scratch);
    __syncthreads();
    // the tile's rows, two pixels per 16-byte store
    const int lw = ilog2(TW / 2);
    uint4 *dst = reinterpret_cast<uint4 *>(a.P + ((size_t)s * geo.H + ty0) * geo.W + tx0);
    for (int i = threadIdx.x; i < TH * TW / 2; i += kRThreads)
        dst[(size_t)(i >> lw) * (geo.W / 2) + (i & (TW / 2 - 1))] = a4[i];
}

template <int N, int MODE, bool SQ>
__global__ void __launch_bounds__(kThreads, 2) k_strip_forward(const __grid_constant__ StripArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_enter();
    strip_forward_item<N, MODE, SQ>(a, blockIdx.y, blockIdx.x, smem_raw);
}

// The image losses of inverse rendering on one column block of image s
// (kOpLoss, see LossDev): buf0 holds the image's unnormalised spectrum A,
// md.tab the target's B.  Writes the complex gradient of the weighted loss
// to buf1 (the caller inverse-transforms it) and the block's two sums,
// reduced in a fixed order, to part[s][bk].
template <int N>
__device__ __forceinline__ void loss_columns(const ColumnArgs &a, int s, int bk, int B, int W,
                                             const float2 *buf0, float2 *buf1) {
    constexpr int LS = line_stride(N);
    __shared__ float red[2 * (kThreads / 32)];
    const LossDev &L = a.loss;
    const float2 *Tb = a.md[s][0].tab + (size_t)bk * N * B;
    const bool mis = L.cutoff != nullptr;
    const float cut = mis ? *L.cutoff : 0.f;
    const float cut2 = cut * cut;
    const float gm = 2.f * L.misfit_scale / ((float)N * (float)W);  // 2 scale / (H W)
    const bool spec = L.spectral_weight != 0.f;
    const float e = L.eps_rel * L.maxamp[s];
    const float gs = 2.f * L.spectral_weight * L.inv_ntot;
    const int half = W / 2;
    float pm = 0.f, ps = 0.f;
#pragma unroll 4
    for (int i = 0; i < ept(N); ++i) {
        const int el = threadIdx.x + i * kThreads;  // line-major: consecutive y
        const int c = el / N, y = el % N;
        if (c < B) {
            const int kx = bk * B + c;
            const float fx = (float)(kx < half ? kx : kx - W) * L.fx_scale;
            const float fy = (float)(y < N / 2 ? y : y - N) * L.fy_scale;
            const float2 A = buf0[c * LS + pad16(y)];
            const float2 T = Tb[y * B + c];
            float2 g = make_float2(0.f, 0.f);
            if (mis && fmaf(fx, fx, fy * fy) <= cut2) {
                const float2 D = csub(A, T);
                pm = fmaf(D.x, D.x, fmaf(D.y, D.y, pm));
                g = make_float2(gm * D.x, gm * D.y);
            }
            if (spec) {
                const float ma = sqrtf(fmaf(A.x, A.x, A.y * A.y));
                const float mb = sqrtf(fmaf(T.x, T.x, T.y * T.y));
                const float d = __logf(ma + e) - __logf(mb + e);
                ps = fmaf(d, d, ps);
                if (ma > 0.f) {
                    const float q = __fdividef(gs * d, ma * (ma + e));
                    g = make_float2(fmaf(q, A.x, g.x), fmaf(q, A.y, g.y));
                }
            }
            buf1[c * LS + pad16(y)] = g;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        pm += __shfl_xor_sync(0xffffffffu, pm, d);
        ps += __shfl_xor_sync(0xffffffffu, ps, d);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[2 * warp] = pm;
        red[2 * warp + 1] = ps;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        float v = 0.f;
        for (int w = 0; w < kThreads / 32; ++w) v += red[2 * w + threadIdx.x];
        const float k = threadIdx.x == 0 ? L.misfit_scale / ((float)N * (float)W) : L.inv_ntot;
        L.part[((size_t)s * (W / B) + bk) * 2 + threadIdx.x] = v * k;
    }
}

// ------------------------------------------------------------ bulk copies
// A contiguous global -> shared copy made by the TMA unit (cp.async.bulk),
// completing on an mbarrier of the CTA: both addresses 16-byte aligned, the
// size a multiple of 16.  The CTA's threads wait on the barrier with a
// bounded number of polls; a wait that runs out latches OSOG_ERR_TIMEOUT,
// waits once more (again bounded) for the copy in flight and lets the item
// go on with whatever has arrived, so the launch always ends.
__device__ __forceinline__ uint32_t shared_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// `missing` bytes more than the copy delivers are expected on the barrier
// (a failure-detection test: the wait then runs out; 0 in normal use).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar, uint32_t missing = 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(shared_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                 ::"r"(shared_addr(bar)), "r"(bytes + missing) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(shared_addr(dst)), "l"(src), "r"(bytes), "r"(shared_addr(bar)) : "memory");
}

constexpr int kBulkPolls = 1 << 20;

__device__ __forceinline__ bool bulk_try(uint64_t *bar, int polls) {
    const uint32_t b = shared_addr(bar);
    for (int it = 0; it < polls; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(b) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_wait(uint64_t *bar, int32_t *status, int polls) {
    if (polls <= 0) polls = kBulkPolls;
    if (!bulk_try(bar, polls)) {
        latch(status, OSOG_ERR_TIMEOUT);
        (void)bulk_try(bar, polls);
    }
}

// The first Stockham pass (radix P0, stride 1) of the L columns of a column
// block whose samples are still in the block's global layout, (y, c) at
// raw[y L + c], where the bulk copy put them (raw aliases buf).  A warp's
// lanes take (c = lane mod L, consecutive j), so its loads cover 32
// consecutive samples and its stores spread over the banks like those of
// the regular pass; columns whose bit in `live` is clear read as zero.
template <int N, bool INV>
__device__ __forceinline__ void first_pass_from_block(float2 *buf, unsigned live) {
    constexpr int L = set_elems(N) / N;
    constexpr int P = fft_radix(N, 0);
    constexpr int NB = N / P;
    constexpr int LS = line_stride(N);
    static_assert(L * NB == kThreads && 32 % L == 0, "one butterfly per thread");
    const int lane = threadIdx.x & 31;
    const int c = lane % L, j = (threadIdx.x >> 5) * (32 / L) + lane / L;
    const bool on = (live >> c) & 1u;
    float2 v[P];
#pragma unroll
    for (int r = 0; r < P; ++r) v[r] = on ? buf[(j + r * NB) * L + c] : make_float2(0.f, 0.f);
    __syncthreads();
    dft<P, INV>(v);
    float2 *dst = buf + c * LS + pad16(j * P);
#pragma unroll
    for (int r = 0; r < P; ++r) dst[r] = v[r];
    __syncthreads();
}

// One column block bk of scene s.
// BULK: a square canvas of N >= 1024 (L = B full columns per block) whose
// G block arrives by one bulk copy.
template <int N, bool MULTI, bool SQ = false, bool BULK = false>
__device__ __forceinline__ void column_item(const ColumnArgs &a, int s, int bk,
                                            unsigned char *smem_raw) {
    constexpr int L = set_elems(N) / N;
    constexpr int LS = line_stride(N);
    float2 *buf0 = reinterpret_cast<float2 *>(smem_raw);
    float2 *buf1 = MULTI ? buf0 + L * LS : buf0;
    int2 *chords = reinterpret_cast<int2 *>(buf1 + L * LS);
    const Geometry &geo = a.geo;
    const int B = SQ ? sq_rb(N) : geo.B, lb = SQ ? clog2(sq_rb(N)) : ilog2(B), K = a.K;
    const int W = SQ ? N : geo.W;
    const int2 cr = a.w.colrange[s];
    // A block whose columns all lie outside every pupil has nothing to filter:
    // its Q block is never read.  The block's unsigned columns [u0, u1] map to
    // signed frequencies [u0, min(u1, W/2 - 1)] and [max(u0, W/2), u1] - W.
    const int u0 = bk * B, u1 = u0 + B - 1, half = W / 2;
    const bool lo_part = u0 < half && u0 <= cr.y && min(u1, half - 1) >= cr.x;
    const bool hi_part = u1 >= half && max(u0, half) - W <= cr.y && u1 - W >= cr.x;
    if (!lo_part && !hi_part) return;
    const float2 *G = a.w.G + ((size_t)s * geo.nblocks + bk) * N * B;
    const int NB_ = N * B;  // <= set_elems(N); lines B..L-1 are never read back
    static_assert(!BULK || (SQ && N >= 1024), "bulk staging needs full column blocks");
    __shared__ uint64_t bar;  // completes the bulk copy (BULK)
    const bool bulk = BULK && !a.unit_input;
    constexpr bool GRP = kGroupFft && fft_grouped(N);
    if (bulk) {
        if constexpr (BULK)
            if (threadIdx.x == 0)
                bulk_load(buf0, G, (uint32_t)(N * L * sizeof(float2)), &bar, a.wait_extra ? 16u : 0u);
    } else if (a.unit_input) {  // the spectrum of a unit impulse: 1 at every frequency
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            if (e < NB_) buf0[(e & (B - 1)) * LS + pad16(e >> lb)] = make_float2(1.f, 0.f);
        }
    } else {
        float2 v[ept(N)];
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            const int kx = u0 + (e & (B - 1)), fx = kx < half ? kx : kx - W;
            v[i] = e < NB_ && fx >= cr.x && fx <= cr.y ? G[e] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            if (e < NB_) buf0[(e & (B - 1)) * LS + pad16(e >> lb)] = v[i];
        }
    }
    for (int j = threadIdx.x; j < K * B; j += kThreads) {  // this block's chords
        const int m = j >> lb, c = j & (B - 1), kx = u0 + c;
        chords[m * L + c] = mode_chord(a.md[s][m], kx < half ? kx : kx - W, N);
    }
    __syncthreads();  // (bulk) the barrier's initialisation precedes every wait
    if constexpr (BULK) {
        if (bulk) {
            unsigned live = 0;  // columns inside the pupils' hull; the others read as zero
#pragma unroll
            for (int c = 0; c < L; ++c) {
                const int kx = u0 + c, fx = kx < half ? kx : kx - W;
                live |= (fx >= cr.x && fx <= cr.y ? 1u : 0u) << c;
            }
            bulk_wait(&bar, a.w.status, a.wait_polls);
            first_pass_from_block<N, false>(buf0, live);
            fft_pass_range<N, L, false, 1, fft_passes(N), GRP>(buf0, a.tw);
            if constexpr (GRP) __syncthreads();  // every line done before any thread reads another's
        }
    } else if (!a.unit_input) {
        fft_lines<N, L, false>(buf0, a.tw);
    }
    for (int m = 0; m < K; ++m) {
        const ModeDev md = live_mode(a.md[s][m]);
        if (md.op == kOpSpectrum) {  // the forward spectrum itself, to md.tab
            float2 *T = md.tab + (size_t)bk * N * B;
#pragma unroll
            for (int i = 0; i < ept(N); ++i) {
                const int e = threadIdx.x + i * kThreads;
                if (e < NB_) {
                    const float2 v = buf0[(e & (B - 1)) * LS + pad16(e >> lb)];
                    T[e] = make_float2(v.x * md.scale, v.y * md.scale);
                }
            }
            continue;  // buf0 is only read: the next modality may still use it
        }
        float2 *Qm = a.w.Q + (((size_t)s * K + m) * geo.nblocks + bk) * N * B;
        if (md.op == kOpPupil || md.op == kOpAllPass) {
            // the transfer function is applied as the first inverse pass
            // loads the spectrum (in place when buf1 is buf0)
            auto ld = [&](int c, int y) -> float2 {
                if (c < B) {
                    const int2 ch = chords[m * L + c];
                    const int fy = y < N / 2 ? y : y - N;
                    if (fy >= ch.x && fy <= ch.y) {
                        const int kx = bk * B + c;
                        return cmul(buf0[c * LS + pad16(y)], transfer(md, kx < half ? kx : kx - W, fy));
                    }
                }
                return make_float2(0.f, 0.f);
            };
            fft_first_pass<N, L, true, !MULTI, GRP>(buf1, ld);
        } else {
            if (md.op == kOpLoss) {
                loss_columns<N>(a, s, bk, B, W, buf0, buf1);
            } else {  // kOpTable
                const float2 *T = md.tab + (size_t)bk * N * B;
                const float tnorm = md.scale / md.tab[0].x;
#pragma unroll 4
                for (int i = 0; i < ept(N); ++i) {
                    const int e = threadIdx.x + i * kThreads;  // line-major: consecutive y
                    const int c = e / N, y = e % N;
                    if (c < B) {
                        const float2 t = T[y * B + c];
                        buf1[c * LS + pad16(y)] =
                            cmul(buf0[c * LS + pad16(y)], make_float2(t.x * tnorm, t.y * tnorm));
                    }
                }
            }
            __syncthreads();
            fft_pass_range<N, L, true, 0, 1>(buf1, a.tw);
        }
        fft_pass_range<N, L, true, 1, fft_passes(N) - 1, GRP>(buf1, a.tw);
        if constexpr (GRP) __syncthreads();
        // the last pass stores Q; consecutive threads take the block's
        // columns, so a warp writes whole rows of the block
        fft_last_pass<N, L, true, true, false>(buf1, a.tw, [&](int c, int y, float2 v) {
            if (c < B) Qm[(size_t)y * B + c] = v;
        });
        __syncthreads();
    }
}

template <int N, bool MULTI, bool SQ>
__global__ void __launch_bounds__(kThreads, 2) k_column(const __grid_constant__ ColumnArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_enter();
    column_item<N, MULTI, SQ, SQ && N >= 1024>(a, blockIdx.y, blockIdx.x, smem_raw);
}

// One strip of the image sm = s K + m.
template <int N, bool SQ = false>
__device__ __forceinline__ void inverse_item(const InverseArgs &a, int sm, int strip,
                                             unsigned char *smem_raw) {
    constexpr int L = set_elems(N) / N;
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    const Geometry &geo = a.geo;
    const int K = a.K;
    const int R = SQ ? sq_rb(N) : geo.R, B = SQ ? sq_rb(N) : geo.B;
    const int lb = SQ ? clog2(sq_rb(N)) : ilog2(B);
    const int H = SQ ? N : geo.H;
    const int y0 = strip * R;
    const float2 *Qm = a.w.Q + (size_t)sm * geo.nblocks * H * B;
    const int2 cr = a.w.colrange[sm / K];
    // the first pass reads the strip's rows of Q straight from global memory
    // (columns that no pupil passes, and lines past the strip, read as zero);
    // the last pass writes the intensity rows
    constexpr bool GRP = kGroupFft && fft_grouped(N);
    fft_first_pass<N, L, true, false, GRP>(buf, [&](int l, int kx) -> float2 {
        const int fx = kx < N / 2 ? kx : kx - N;
        return l < R && fx >= cr.x && fx <= cr.y
                   ? Qm[((size_t)(kx >> lb) * H + y0 + l) * B + (kx & (B - 1))]
                   : make_float2(0.f, 0.f);
    });
    fft_pass_range<N, L, true, 1, fft_passes(N) - 1, GRP>(buf, a.tw);
    float *img = a.images + ((size_t)sm * H + y0) * N;
    const int real_out = a.real_out;
    fft_last_pass<N, L, true, false, GRP>(buf, a.tw, [&](int l, int x, float2 v) {
        if (l < R) img[(size_t)l * N + x] = real_out ? v.x : fmaf(v.x, v.x, __fmul_rn(v.y, v.y));
    });
}

template <int N, bool SQ>
__global__ void __launch_bounds__(kThreads, 2) k_strip_inverse(const __grid_constant__ InverseArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_enter();
    inverse_item<N, SQ>(a, blockIdx.y, blockIdx.x, smem_raw);
}

// ------------------------------------------------------------ persistent
// Bounded wait on a completion counter: thread 0 polls until it reaches
// target or `polls` polls run out; then it raises the launch's gave-up flag,
// latches OSOG_ERR_TIMEOUT in the status word and the item proceeds on
// whatever is there, so the launch always ends.  Once the flag is up, later
// waits of the launch return at once.  The fence orders the producer's
// writes before this CTA's reads.

__device__ __forceinline__ void wait_count(const int32_t *cnt, int target, int32_t *gave_up,
                                           int32_t *status, int polls) {
    if (threadIdx.x == 0) {
        const volatile int32_t *flag = gave_up;
        int spins = 0;
        while (*reinterpret_cast<const volatile int32_t *>(cnt) < target && !*flag) {
            __nanosleep(100);
            if (++spins >= polls) {
                atomicExch(gave_up, 1);
                latch(status, OSOG_ERR_TIMEOUT);
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Work items in dispatch order: wave t holds the strips of scene t, the
// column blocks of scene t - 1 and the inverse strips of scene t - 2, so a
// column (inverse) item of scene s is handed out only after every strip
// (column block) item of s, to CTAs that are already running.
__device__ __forceinline__ void decode_item(int it, int S, int na, int nb, int nc, int &stage,
                                            int &s, int &idx) {
    for (int t = 0; t < S + 2; ++t) {
        const int sa = t < S ? na : 0;
        const int sb = t >= 1 && t - 1 < S ? nb : 0;
        const int sc = t >= 2 && t - 2 < S ? nc : 0;
        if (it < sa) { stage = 0; s = t; idx = it; return; }
        it -= sa;
        if (it < sb) { stage = 1; s = t - 1; idx = it; return; }
        it -= sb;
        if (it < sc) { stage = 2; s = t - 2; idx = it; return; }
        it -= sc;
    }
    stage = 3;
}

// Two CTAs per SM when one modality keeps the largest stage (the strip
// kernel) within half of the shared memory, as the separate kernels run.
template <int N, bool MULTI>
__global__ void __launch_bounds__(kThreads, MULTI ? 1 : 2) k_persistent(const __grid_constant__ PersistArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int item[3];
    const Geometry &geo = a.sa.geo;
    const int S = a.sa.S, K = a.ca.K;
    const int na = geo.nstrips, nb = geo.nblocks, nc = K * geo.nstrips;
    int32_t *doneA = a.ctr + 1, *doneB = a.ctr + 1 + S, *gave_up = a.ctr + 1 + 2 * S;
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = atomicAdd(a.ctr, 1);
            int stage = 3, s = 0, idx = 0;
            if (it < a.total) decode_item(it, S, na, nb, nc, stage, s, idx);
            item[0] = stage;
            item[1] = s;
            item[2] = idx;
        }
        __syncthreads();
        const int stage = item[0], s = item[1], idx = item[2];
        __syncthreads();
        if (stage == 3) break;
        if (stage == 0) {
            strip_forward_item<N, kStripRender, true>(a.sa, s, idx, smem_raw);
        } else if (stage == 1) {
            wait_count(doneA + s, na + a.wait_extra, gave_up, a.sa.w.status, a.wait_polls);
            column_item<N, MULTI, true>(a.ca, s, idx, smem_raw);
        } else {
            wait_count(doneB + s, nb, gave_up, a.sa.w.status, a.wait_polls);
            inverse_item<N, true>(a.ia, s * K + idx / na, idx % na, smem_raw);
        }
        __syncthreads();
        if (threadIdx.x == 0 && stage < 2) {
            __threadfence();
            atomicAdd(stage == 0 ? doneA + s : doneB + s, 1);
        }
    }
}

template <int N>
struct PersistLaunch {
    static cudaError_t run(const PersistArgs &a, cudaStream_t st) {
        const size_t smem = persistent_smem(N, a.ca.K);
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        if (a.ca.K > 1)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent<N, true>, kThreads, smem);
        else
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent<N, false>, kThreads, smem);
        if (e != cudaSuccess) return e;
        const int grid = max(1, min(a.total, max(per, 1) * sms));
        if (a.ca.K > 1)
            k_persistent<N, true><<<grid, kThreads, smem, st>>>(a);
        else
            k_persistent<N, false><<<grid, kThreads, smem, st>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t prepare() {
        cudaError_t e = cudaFuncSetAttribute(k_persistent<N, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)persistent_smem(N, 1));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_persistent<N, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)persistent_smem(N, 3));
        return e;
    }
};

template <int N>
struct StripFwdLaunch {
    static cudaError_t run(const StripArgs &a, StripMode mode, cudaStream_t st) {
        dim3 grid(a.geo.nstrips, a.S);
        const size_t smem = strip_forward_smem(N), smem_opd = strip_forward_smem(N, true);
        const size_t smem_fft = strip_inverse_smem(N);  // the set alone: no raster
        if (mode == kStripRender && a.geo.H == a.geo.W)
            return launch_chain(k_strip_forward<N, kStripRender, true>, grid, kThreads, smem, st, a);
        else if (mode == kStripRender)
            return launch_chain(k_strip_forward<N, kStripRender, false>, grid, kThreads, smem, st, a);
        else if (mode == kStripOpdOnly)
            return launch_chain(k_strip_forward<N, kStripOpdOnly, false>, grid, kThreads, smem_opd, st, a);
        else if (mode == kStripFromReal)
            return launch_chain(k_strip_forward<N, kStripFromReal, false>, grid, kThreads, smem, st, a);
        else if (mode == kStripFromPhase && a.geo.H == a.geo.W)
            return launch_chain(k_strip_forward<N, kStripFromPhase, true>, grid, kThreads, smem_fft, st, a);
        else if (mode == kStripFromPhase)
            return launch_chain(k_strip_forward<N, kStripFromPhase, false>, grid, kThreads, smem_fft, st, a);
        else
            return launch_chain(k_strip_forward<N, kStripFromMap, false>, grid, kThreads, smem, st, a);
    }
    static cudaError_t prepare() {
        const int smem = (int)strip_forward_smem(N), smem_opd = (int)strip_forward_smem(N, true);
        cudaError_t e = cudaFuncSetAttribute(k_strip_forward<N, kStripRender, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_strip_forward<N, kStripRender, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_strip_forward<N, kStripOpdOnly, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem_opd);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_strip_forward<N, kStripFromMap, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_strip_forward<N, kStripFromReal, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        for (int sq = 0; sq < 2 && e == cudaSuccess; ++sq)
            e = cudaFuncSetAttribute(sq ? k_strip_forward<N, kStripFromPhase, true>
                                        : k_strip_forward<N, kStripFromPhase, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)strip_inverse_smem(N));
        return e;
    }
};

template <int N>
struct ColumnLaunch {
    static cudaError_t run(const ColumnArgs &a, cudaStream_t st, size_t smem) {
        dim3 grid(a.geo.nblocks, a.S);
        const bool sq = a.geo.H == a.geo.W;
        if (a.K > 1 && sq)
            return launch_chain(k_column<N, true, true>, grid, kThreads, smem, st, a);
        else if (a.K > 1)
            return launch_chain(k_column<N, true, false>, grid, kThreads, smem, st, a);
        else if (sq)
            return launch_chain(k_column<N, false, true>, grid, kThreads, smem, st, a);
        else
            return launch_chain(k_column<N, false, false>, grid, kThreads, smem, st, a);
    }
    static cudaError_t prepare(size_t smem1, size_t smem2) {
        cudaError_t e = cudaSuccess;
        for (int sq = 0; sq < 2 && e == cudaSuccess; ++sq) {
            e = cudaFuncSetAttribute(sq ? k_column<N, false, true> : k_column<N, false, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(sq ? k_column<N, true, true> : k_column<N, true, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
        }
        return e;
    }
};

template <int N>
struct InverseLaunch {
    static cudaError_t run(const InverseArgs &a, cudaStream_t st, size_t smem) {
        dim3 grid(a.geo.nstrips, a.S * a.K);
        if (a.geo.H == a.geo.W)
            return launch_chain(k_strip_inverse<N, true>, grid, kThreads, smem, st, a);
        else
            return launch_chain(k_strip_inverse<N, false>, grid, kThreads, smem, st, a);
    }
    static cudaError_t prepare(size_t smem) {
        cudaError_t e = cudaFuncSetAttribute(k_strip_inverse<N, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_strip_inverse<N, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return e;
    }
};

template <int N>
struct Prepare {
    static cudaError_t run(int which, int other) {
        (void)other;
        if (which == 0) return StripFwdLaunch<N>::prepare();
        if (which == 1) return ColumnLaunch<N>::prepare(column_smem(N, 1), column_smem(N, 3));
        if (which == 3) return PersistLaunch<N>::prepare();
        return InverseLaunch<N>::prepare(strip_inverse_smem(N));
    }
};

// Largest |z| of spectrum blockIdx.y (count samples), as the maximum of
// |z|^2 over grid-strided CTAs merged by an integer atomicMax on the
// float's bits (non-negative floats order like their bits; the maximum does
// not depend on the order).  out must start at zero; the square root is
// taken by the reader.
__global__ void __launch_bounds__(256) k_max_amplitude(const float2 *spec, int64_t count,
                                                       float *out) {
    __shared__ float red[8];
    const float2 *p = spec + (size_t)blockIdx.y * count;
    float m = 0.f;
    for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < count; i += (int64_t)gridDim.x * 256) {
        const float2 v = p[i];
        m = fmaxf(m, fmaf(v.x, v.x, v.y * v.y));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
        atomicMax(reinterpret_cast<int *>(out) + blockIdx.y, __float_as_int(m));
    }
}

__global__ void k_sqrt_inplace(float *v, int n) {
    if ((int)threadIdx.x < n) v[threadIdx.x] = sqrtf(v[threadIdx.x]);
}

// loss[c] = sum over i of part[2 i + c] (c = 0, 1): lanes stride over the
// partials in double, then a fixed butterfly and the warps in order.
__global__ void __launch_bounds__(256) k_loss_reduce(const float *part, int64_t nparts,
                                                     float *loss) {
    __shared__ double red[2][8];
    double v0 = 0.0, v1 = 0.0;
    for (int64_t i = threadIdx.x; i < nparts; i += 256) {
        v0 += (double)part[2 * i];
        v1 += (double)part[2 * i + 1];
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, d);
        v1 += __shfl_xor_sync(0xffffffffu, v1, d);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = v0;
        red[1][threadIdx.x >> 5] = v1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[threadIdx.x][w];
        loss[threadIdx.x] = (float)t;
    }
}

}  // namespace

cudaError_t launch_max_amplitude(const float2 *spec, int S, int64_t count, float *maxamp,
                                 cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(maxamp, 0, sizeof(float) * S, st);
    if (e != cudaSuccess) return e;
    k_max_amplitude<<<dim3(256, S), 256, 0, st>>>(spec, count, maxamp);
    k_sqrt_inplace<<<1, 32, 0, st>>>(maxamp, S);
    return cudaGetLastError();
}

cudaError_t launch_loss_reduce(const float *part, int64_t nparts, float *loss, cudaStream_t st) {
    k_loss_reduce<<<1, 256, 0, st>>>(part, nparts, loss);
    return cudaGetLastError();
}

size_t strip_forward_smem(int W, bool opd_mode) {
    const int L = set_elems(W) / W;
    return (size_t)(opd_mode ? 2 : 1) * L * line_stride(W) * sizeof(float2) + raster_smem<kThreads>();
}

size_t column_smem(int H, int K) {
    const int L = set_elems(H) / H;
    return (size_t)(K > 1 ? 2 : 1) * L * line_stride(H) * sizeof(float2) +
           (size_t)kMaxModes * L * sizeof(int2);
}

size_t strip_inverse_smem(int W) {
    const int L = set_elems(W) / W;
    return (size_t)L * line_stride(W) * sizeof(float2);
}

size_t persistent_smem(int N, int K) {
    const size_t a = strip_forward_smem(N), b = column_smem(N, K), c = strip_inverse_smem(N);
    return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

int raster_tile_cols(const Geometry &geo) {
    int tw = 4096 / geo.BH;
    if (tw < 32) tw = 32;
    return tw > geo.W ? geo.W : tw;
}

static size_t raster_tiles_smem(int BH, int TW) {
    return (size_t)BH * TW * sizeof(uint2) + raster_smem<kRThreads>();
}

cudaError_t launch_raster_tiles(const RasterArgs &a, cudaStream_t st) {
    const dim3 grid(a.geo.W / a.TW, a.geo.nbands, a.S);
    const size_t smem = raster_tiles_smem(a.geo.BH, a.TW);
    if (smem > 48 * 1024) {  // tall bands: opt in to the size (host-side, cached by the driver)
        const cudaError_t e = cudaFuncSetAttribute(k_raster_tiles,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_chain(k_raster_tiles, grid, kRThreads, smem, st, a);
}

cudaError_t prepare_kernels(int H, int W) {
    cudaError_t e = dispatch_n<Prepare>(W, 0, 0);
    if (e == cudaSuccess) e = dispatch_n<Prepare>(H, 1, 0);
    if (e == cudaSuccess) e = dispatch_n<Prepare>(W, 2, 0);
    if (e == cudaSuccess && H == W) e = dispatch_n<Prepare>(W, 3, 0);
    return e;
}

cudaError_t launch_persistent(const PersistArgs &a, cudaStream_t st) {
    if (a.sa.geo.H != a.sa.geo.W) return cudaErrorInvalidValue;
    return dispatch_n<PersistLaunch>(a.sa.geo.W, a, st);
}

cudaError_t launch_strip_forward(const StripArgs &a, StripMode mode, cudaStream_t st) {
    return dispatch_n<StripFwdLaunch>(a.geo.W, a, mode, st);
}

cudaError_t launch_column(const ColumnArgs &a, cudaStream_t st) {
    return dispatch_n<ColumnLaunch>(a.geo.H, a, st, column_smem(a.geo.H, a.K));
}

cudaError_t launch_strip_inverse(const InverseArgs &a, cudaStream_t st) {
    return dispatch_n<InverseLaunch>(a.geo.W, a, st, strip_inverse_smem(a.geo.W));
}

}  // namespace osog
