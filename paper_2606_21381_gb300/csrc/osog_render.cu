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

// One strip (rows [strip R, strip R + R)) of scene s.
template <int N, int MODE, bool SQ = false>
__device__ __forceinline__ void strip_forward_item(const StripArgs &a, int s, int strip,
                                                   unsigned char *smem_raw) {
    constexpr int L = set_elems(N) / N;
    constexpr int LS = line_stride(N);
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    PRec *srec = reinterpret_cast<PRec *>(buf + L * LS);
    Rect *srect = reinterpret_cast<Rect *>(srec + kThreads);
    int *wsum = reinterpret_cast<int *>(srect + kThreads);
    const Geometry &geo = a.geo;
    const int R = SQ ? sq_rb(N) : geo.R;
    const int y0 = strip * R;
    const int RN = R * N;  // <= set_elems(N); lines R..L-1 are never read back
    if constexpr (MODE == kStripFromReal) {
        const float *src = reinterpret_cast<const float *>(a.opd_att) + (size_t)y0 * N;
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
        for (int i = threadIdx.x; i < R * LS / 2; i += kThreads) b4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        raster_strip<N>(a.geo, a.w, a.sc[s], s, y0, buf, srec, srect, wsum);
    }
    __syncthreads();
    if constexpr (MODE == kStripOpdOnly) {
        float2 *dst = a.opd_out + (size_t)y0 * N;
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            if (e < RN) dst[e] = buf[(e / N) * LS + pad16(e % N)];
        }
        return;
    } else {
        const float tol = a.sc[s].two_over_lambda;
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            if (MODE != kStripFromReal && e < RN) {
                float2 *v = buf + (e / N) * LS + pad16(e % N);
                const float2 oa = *v;
                if (oa.x != 0.f || oa.y != 0.f) {  // empty pixels keep E = 1
                    *v = exit_wave(oa.x, oa.y, tol);
                } else {
                    *v = make_float2(1.f, 0.f);
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

template <int N, int MODE, bool SQ>
__global__ void __launch_bounds__(kThreads, 2) k_strip_forward(const __grid_constant__ StripArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_enter();
    strip_forward_item<N, MODE, SQ>(a, blockIdx.y, blockIdx.x, smem_raw);
}

// One column block bk of scene s.
template <int N, bool MULTI, bool SQ = false>
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
    if (a.unit_input) {  // the spectrum of a unit impulse: 1 at every frequency
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
    __syncthreads();
    if (!a.unit_input) fft_lines<N, L, false>(buf0, a.tw);
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
        const float2 *T = md.op == kOpTable ? md.tab + (size_t)bk * N * B : nullptr;
        const float tnorm = md.op == kOpTable ? md.scale / md.tab[0].x : 0.f;
#pragma unroll 4
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;  // line-major: consecutive y
            const int c = e / N, y = e % N;
            if (c < B) {
                const int kx = bk * B + c;
                const int fx = kx < half ? kx : kx - W;
                const int fy = y < N / 2 ? y : y - N;
                const int2 ch = chords[m * L + c];
                float2 v = make_float2(0.f, 0.f);
                if (T) {
                    const float2 t = T[y * B + c];
                    v = cmul(buf0[c * LS + pad16(y)], make_float2(t.x * tnorm, t.y * tnorm));
                } else if (fy >= ch.x && fy <= ch.y) {
                    v = cmul(buf0[c * LS + pad16(y)], transfer(md, fx, fy));
                }
                buf1[c * LS + pad16(y)] = v;
            }
        }
        __syncthreads();
        fft_lines<N, L, true>(buf1, a.tw);
        float2 *Qm = a.w.Q + (((size_t)s * K + m) * geo.nblocks + bk) * N * B;
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            if (e < NB_) Qm[e] = buf1[(e & (B - 1)) * LS + pad16(e >> lb)];
        }
        __syncthreads();
    }
}

template <int N, bool MULTI, bool SQ>
__global__ void __launch_bounds__(kThreads, 2) k_column(const __grid_constant__ ColumnArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_enter();
    column_item<N, MULTI, SQ>(a, blockIdx.y, blockIdx.x, smem_raw);
}

// One strip of the image sm = s K + m.
template <int N, bool SQ = false>
__device__ __forceinline__ void inverse_item(const InverseArgs &a, int sm, int strip,
                                             unsigned char *smem_raw) {
    constexpr int L = set_elems(N) / N;
    constexpr int LS = line_stride(N);
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    const Geometry &geo = a.geo;
    const int K = a.K;
    const int R = SQ ? sq_rb(N) : geo.R, B = SQ ? sq_rb(N) : geo.B;
    const int lb = SQ ? clog2(sq_rb(N)) : ilog2(B), lr = SQ ? clog2(sq_rb(N)) : ilog2(R);
    const int H = SQ ? N : geo.H;
    const int y0 = strip * R;
    const float2 *Qm = a.w.Q + (size_t)sm * geo.nblocks * H * B;
    const int2 cr = a.w.colrange[sm / K];
    const int RN = R * N;  // <= set_elems(N); lines R..L-1 are never read back
    {
        float2 v[ept(N)];
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            const int c = e & (B - 1), r = (e >> lb) & (R - 1), bk = e >> (lb + lr);
            const int kx = bk * B + c, fx = kx < N / 2 ? kx : kx - N;
            v[i] = e < RN && fx >= cr.x && fx <= cr.y ? Qm[((size_t)bk * H + y0 + r) * B + c]
                                                      : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;
            const int c = e & (B - 1), r = (e >> lb) & (R - 1), bk = e >> (lb + lr);
            if (e < RN) buf[r * LS + pad16(bk * B + c)] = v[i];
        }
    }
    __syncthreads();
    fft_lines<N, L, true>(buf, a.tw);
    float *img = a.images + ((size_t)sm * H + y0) * N;
#pragma unroll
    for (int i = 0; i < ept(N); ++i) {
        const int e = threadIdx.x + i * kThreads;
        if (e < RN) {
            const float2 v = buf[(e / N) * LS + pad16(e % N)];
            img[e] = a.real_out ? v.x : fmaf(v.x, v.x, __fmul_rn(v.y, v.y));
        }
    }
}

template <int N, bool SQ>
__global__ void __launch_bounds__(kThreads, 2) k_strip_inverse(const __grid_constant__ InverseArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_enter();
    inverse_item<N, SQ>(a, blockIdx.y, blockIdx.x, smem_raw);
}

// ------------------------------------------------------------ persistent
// Bounded wait on a completion counter: thread 0 polls until it reaches
// target or the iteration limit runs out (then the status word records a
// timeout and the item proceeds on whatever is there, so the launch always
// ends); the fence orders the producer's writes before this CTA's reads.
constexpr int kSpinLimit = 1 << 24;

__device__ __forceinline__ void wait_count(const int32_t *cnt, int target, int32_t *status) {
    if (threadIdx.x == 0) {
        int spins = 0;
        while (*reinterpret_cast<const volatile int32_t *>(cnt) < target) {
            __nanosleep(100);
            if (++spins >= kSpinLimit) {
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
    int32_t *doneA = a.ctr + 1, *doneB = a.ctr + 1 + S;
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
            wait_count(doneA + s, na, a.sa.w.status);
            column_item<N, MULTI, true>(a.ca, s, idx, smem_raw);
        } else {
            wait_count(doneB + s, nb, a.sa.w.status);
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
    static cudaError_t run(const StripArgs &a, StripMode mode, cudaStream_t st, size_t smem) {
        dim3 grid(a.geo.nstrips, a.S);
        if (mode == kStripRender && a.geo.H == a.geo.W)
            return launch_chain(k_strip_forward<N, kStripRender, true>, grid, kThreads, smem, st, a);
        else if (mode == kStripRender)
            return launch_chain(k_strip_forward<N, kStripRender, false>, grid, kThreads, smem, st, a);
        else if (mode == kStripOpdOnly)
            return launch_chain(k_strip_forward<N, kStripOpdOnly, false>, grid, kThreads, smem, st, a);
        else if (mode == kStripFromReal)
            return launch_chain(k_strip_forward<N, kStripFromReal, false>, grid, kThreads, smem, st, a);
        else
            return launch_chain(k_strip_forward<N, kStripFromMap, false>, grid, kThreads, smem, st, a);
    }
    static cudaError_t prepare(size_t smem) {
        cudaError_t e = cudaFuncSetAttribute(k_strip_forward<N, kStripRender, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_strip_forward<N, kStripRender, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_strip_forward<N, kStripOpdOnly, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_strip_forward<N, kStripFromMap, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_strip_forward<N, kStripFromReal, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
        if (which == 0) return StripFwdLaunch<N>::prepare(strip_forward_smem(N));
        if (which == 1) return ColumnLaunch<N>::prepare(column_smem(N, 1), column_smem(N, 3));
        if (which == 3) return PersistLaunch<N>::prepare();
        return InverseLaunch<N>::prepare(strip_inverse_smem(N));
    }
};

}  // namespace

size_t strip_forward_smem(int W) {
    const int L = set_elems(W) / W;
    return (size_t)L * line_stride(W) * sizeof(float2) + kThreads * (sizeof(PRec) + sizeof(Rect)) +
           64;
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
    return dispatch_n<StripFwdLaunch>(a.geo.W, a, mode, st, strip_forward_smem(a.geo.W));
}

cudaError_t launch_column(const ColumnArgs &a, cudaStream_t st) {
    return dispatch_n<ColumnLaunch>(a.geo.H, a, st, column_smem(a.geo.H, a.K));
}

cudaError_t launch_strip_inverse(const InverseArgs &a, cudaStream_t st) {
    return dispatch_n<InverseLaunch>(a.geo.W, a, st, strip_inverse_smem(a.geo.W));
}

}  // namespace osog
