// Adjoint of the render (osog_render_backward): gradients of a loss of the
// images with respect to every particle field and to the optics scalars
// (defocus, shear length, shear angle, DIC bias).
//
// With E the exit wave, G its row DFT, E^ = DFT_cols(G), Q_m =
// IDFT_cols(E^ H_m) and E_m = IDFT_rows(Q_m), I_m = |E_m|^2, and complex
// gradients g = dL/dRe + i dL/dIm, the chain runs backwards as
//   rows    dL/dQ_m = DFT_rows(2 gI_m E_m)               (E_m recomputed)
//   column  dL/dZ_m = DFT_cols(dL/dQ_m),  dL/dE^ = sum_m conj(H_m) dL/dZ_m,
//           dL/dG = IDFT_cols(dL/dE^);  dL/d(optics) = sum Re(conj(dL/dZ_m)
//           E^ dH_m/d(optics))                             (E^ recomputed)
//   strip   dL/dE = IDFT_rows(dL/dG); OPD and ATT re-rasterised, E recomputed;
//           dL/dOPD = (2 pi / lambda) Re(conj(dL/dE) i E),
//           dL/dATT = -Re(conj(dL/dE) E); each particle's pixels are then
//           gathered by one warp into a partial per (band slot, strip)
//   reduce  fixed-order sums of the partials per particle and of the
//           per-block optics partials.
// The intermediates G and Q_m of the recomputed forward pass are overwritten
// in place by dL/dG and dL/dQ_m.  Every sum runs in a fixed order, so the
// gradients are bitwise reproducible.
#include "osog_strip.cuh"

namespace osog {

namespace {

// Deterministic warp sum (fixed butterfly pattern).
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

template <int N>
__global__ void __launch_bounds__(kThreads, 1) k_bwd_rows(const __grid_constant__ BwdRowsArgs a) {
    pdl_enter();
    constexpr int L = set_elems(N) / N;
    constexpr int LS = line_stride(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    const Geometry &geo = a.geo;
    const int sm = blockIdx.y, K = a.K;
    const int y0 = blockIdx.x * geo.R;
    const int RN = geo.R * N;
    float2 *Qm = a.w.Q + (size_t)sm * geo.nblocks * geo.H * geo.B;
    const int2 cr = a.w.colrange[sm / K];
    load_strip_blocked<N>(buf, Qm, geo, y0, cr);
    __syncthreads();
    fft_lines<N, L, true>(buf, a.tw);  // E_m rows
    const float *gI = a.grad_image + ((size_t)sm * geo.H + y0) * N;
#pragma unroll
    for (int i = 0; i < ept(N); ++i) {
        const int e = threadIdx.x + i * kThreads;
        if (e < RN) {
            float2 *v = buf + (e / N) * LS + pad16(e % N);
            const float g2 = 2.f * gI[e];
            *v = make_float2(g2 * v->x, g2 * v->y);
        }
    }
    __syncthreads();
    fft_lines<N, L, false>(buf, a.tw);  // adjoint of the inverse row DFT
    store_strip_blocked<N>(buf, Qm, geo, y0, cr);
}

template <int N>
__global__ void __launch_bounds__(kThreads, 1) k_bwd_column(const __grid_constant__ BwdColumnArgs a) {
    pdl_enter();
    constexpr int L = set_elems(N) / N;
    constexpr int LS = line_stride(N);
    constexpr int NW = kThreads / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *bufE = reinterpret_cast<float2 *>(smem_raw);
    float2 *bufZ = bufE + L * LS;
    int2 *chords = reinterpret_cast<int2 *>(bufZ + L * LS);
    float *red = reinterpret_cast<float *>(chords + kMaxModes * L);
    const Geometry &geo = a.geo;
    const int s = blockIdx.y, bk = blockIdx.x, K = a.K;
    const int B = geo.B, lb = ilog2(B), half = geo.W / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *opart = a.opart + ((size_t)s * geo.nblocks + bk) * 4;
    const int2 cr = a.w.colrange[s];
    if (!block_active(geo, bk, cr)) {  // no pupil passes these columns: no gradient
        if (threadIdx.x < 4) opart[threadIdx.x] = 0.f;
        return;
    }
    float2 *Gb = a.w.G + ((size_t)s * geo.nblocks + bk) * N * B;
    load_block<N>(bufE, Gb, geo, bk, cr);
    for (int j = threadIdx.x; j < K * B; j += kThreads) {  // this block's chords
        const int m = j >> lb, c = j & (B - 1), kx = bk * B + c;
        chords[m * L + c] = mode_chord(a.md[s][m], kx < half ? kx : kx - geo.W, N);
    }
    __syncthreads();
    fft_lines<N, L, false>(bufE, a.tw);  // E^ of the block's columns
    float2 acc[ept(N)];
#pragma unroll
    for (int i = 0; i < ept(N); ++i) acc[i] = make_float2(0.f, 0.f);
    float po[4] = {0.f, 0.f, 0.f, 0.f};
    for (int m = 0; m < K; ++m) {
        const ModeDev md = live_mode(a.md[s][m]);
        const float2 *Qb = a.w.Q + (((size_t)s * K + m) * geo.nblocks + bk) * N * B;
        load_block<N>(bufZ, Qb, geo, bk, cr);
        __syncthreads();
        fft_lines<N, L, false>(bufZ, a.tw);  // dL/dZ_m (adjoint of the inverse column DFT)
#pragma unroll 4
        for (int i = 0; i < ept(N); ++i) {
            const int e = threadIdx.x + i * kThreads;  // line-major: consecutive rows
            const int c = e / N, y = e % N;
            if (c < B) {
                const int kx = bk * B + c;
                const int fx = kx < half ? kx : kx - geo.W;
                const int fy = y < N / 2 ? y : y - N;
                const int2 ch = chords[m * L + c];
                if (fy >= ch.x && fy <= ch.y) {
                    float2 h, dh[4];
                    transfer_grad(md, fx, fy, h, dh);
                    const float2 gz = bufZ[c * LS + pad16(y)];
                    const float2 eh = bufE[c * LS + pad16(y)];
                    acc[i] = cadd(acc[i], cmulc(gz, h));  // conj(H) dL/dZ
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float2 w = cmul(eh, dh[k]);
                        po[k] = fmaf(gz.x, w.x, fmaf(gz.y, w.y, po[k]));
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < ept(N); ++i) {
        const int e = threadIdx.x + i * kThreads;
        const int c = e / N, y = e % N;
        if (c < B) bufZ[c * LS + pad16(y)] = acc[i];
    }
    __syncthreads();
    fft_lines<N, L, true>(bufZ, a.tw);  // dL/dG (adjoint of the forward column DFT)
    store_block<N>(bufZ, Gb, geo);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float v = warp_sum(po[k]);
        if (lane == 0) red[warp * 4 + k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        float v = 0.f;
        for (int w = 0; w < NW; ++w) v += red[w * 4 + threadIdx.x];
        opart[threadIdx.x] = v;
    }
}

template <int N>
__global__ void __launch_bounds__(kThreads, 1) k_bwd_strip(const __grid_constant__ BwdStripArgs a) {
    pdl_enter();
    constexpr int L = set_elems(N) / N;
    constexpr int LS = line_stride(N);
    constexpr int NW = kThreads / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *bufG = reinterpret_cast<float2 *>(smem_raw);
    float2 *bufO = bufG + L * LS;
    PRec *srec = reinterpret_cast<PRec *>(bufO + L * LS);
    Rect *srect = reinterpret_cast<Rect *>(srec + kThreads);
    int *sslot = reinterpret_cast<int *>(srect + kThreads);
    int *wsum = sslot + kThreads;
    const Geometry &geo = a.geo;
    const int s = blockIdx.y;
    const int y0 = blockIdx.x * geo.R, ylast = y0 + geo.R - 1;
    const int RN = geo.R * N;
    const SceneDev &sc = a.sc[s];
    const int2 cr = a.w.colrange[s];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    load_strip_blocked<N>(bufG, a.w.G + (size_t)s * geo.H * N, geo, y0, cr);
    float4 *o4 = reinterpret_cast<float4 *>(bufO);
    for (int i = threadIdx.x; i < geo.R * LS / 2; i += kThreads) o4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    fft_lines<N, L, true>(bufG, a.tw);                                    // dL/dE
    // OPD and ATT as fixed-point accumulators in bufO (its staging shares
    // the gather's staging area below, used only after the raster)
    raster_strip<N, kAccPhase>(geo, a.w, sc, s, y0, geo.R, bufO,
                               reinterpret_cast<unsigned char *>(srec));
    __syncthreads();
    const float k2pi = 3.14159265358979323846f * sc.two_over_lambda;   // 2 pi / lambda
#pragma unroll
    for (int i = 0; i < ept(N); ++i) {
        const int e = threadIdx.x + i * kThreads;
        if (e < RN) {
            const int idx = (e / N) * LS + pad16(e % N);
            const float2 g = bufG[idx];
            const float2 E = exit_wave_fixed(reinterpret_cast<const uint2 *>(bufO)[idx]);
            const float ex = E.x, ey = E.y;
            bufO[idx] = make_float2(k2pi * fmaf(g.y, ex, -g.x * ey), -fmaf(g.x, ex, g.y * ey));
        }
    }
    __syncthreads();
    // Gather: one warp per staged particle, partial per (band slot, strip).
    const int band = y0 / geo.BH;
    const int spb = geo.BH / geo.R, kstrip = (y0 - band * geo.BH) / geo.R;
    const int32_t *off = a.w.band_off + (size_t)s * (geo.nbands + 1);
    const int hi = min(off[band + 1], sc.pair_cap);
    const int lo = min(off[band], hi);
    const int32_t *ids = a.w.pairs + sc.pair0;
    const unsigned lt = lanemask_lt();
    for (int base = lo; base < hi; base += kThreads) {
        const int i = base + threadIdx.x;
        int id = 0;
        Rect q = {1, 0, 1, 0};
        if (i < hi) {
            id = ids[i];
            q = a.w.rect[id];
        }
        const bool keep = i < hi && q.y0 <= ylast && q.y1 >= y0;
        const unsigned m = __ballot_sync(kFull, keep);
        if (lane == 0) wsum[warp] = __popc(m);
        __syncthreads();
        int before = 0, nl = 0;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int c = wsum[k];
            before += k < warp ? c : 0;
            nl += c;
        }
        if (keep) {
            const int slot = before + __popc(m & lt);
            srect[slot] = q;
            srec[slot] = a.w.rec[id];
            sslot[slot] = i;
        }
        __syncthreads();
        for (int k = warp; k < nl; k += NW) {
            const PRec r = srec[k];
            const Rect rq = srect[k];
            const int xa = rq.x0, xb = rq.x1;
            const int ya = max((int)rq.y0, y0), yb = min((int)rq.y1, ylast);
            const int bh = yb - ya + 1;
            const int lyn = bh >= 32 ? 32 : (bh <= 1 ? 1 : 1 << (32 - __clz(bh - 1)));
            const int lxn = 32 / lyn, shx = ilog2(lxn);
            const int lx = lane & (lxn - 1), ly = lane >> shx;
            float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int yy = ya + ly; yy <= yb; yy += lyn) {
                const float2 *row = bufO + (yy - y0) * LS;
                for (int xx = xa + lx; xx <= xb; xx += lxn) {
                    const float2 g = row[pad16(xx)];
                    thickness_grad(r, (float)xx + 0.5f, (float)yy + 0.5f, g.x, g.y, acc);
                }
            }
            float *dst = a.part + ((size_t)(sc.pair0 + sslot[k]) * spb + kstrip) * 8;
#pragma unroll
            for (int f = 0; f < 8; ++f) {
                const float v = warp_sum(acc[f]);
                if (lane == f) dst[f] = v;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kChunk) k_bwd_reduce(const __grid_constant__ BwdReduceArgs a) {
    pdl_enter();
    const Geometry &geo = a.geo;
    if ((int)blockIdx.x >= a.nchunks) {  // optics: sum the per-block partials
        // Warp f sums component f: lane l adds blocks l, l + 32, ... in
        // double, then a fixed butterfly combines the lanes (same order on
        // every run).
        const int s = blockIdx.x - a.nchunks;
        const int f = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (f < 4) {
            double v = 0.0;
            for (int bk = lane; bk < geo.nblocks; bk += 32)
                v += (double)a.opart[((size_t)s * geo.nblocks + bk) * 4 + f];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
            if (lane == 0) a.grad_optics[s * 4 + f] = (float)v;
        }
        return;
    }
    int s = 0;
    for (int t = 1; t < a.S; ++t)
        if (a.sc[t].chunk0 <= (int)blockIdx.x) s = t;
    const SceneDev &sc = a.sc[s];
    const int local = ((int)blockIdx.x - sc.chunk0) * kChunk + threadIdx.x;
    if (local >= sc.n) return;
    const int p = sc.p0 + local;
    const Rect q = a.w.rect[p];
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (q.x0 <= q.x1 && q.y0 <= q.y1) {
        // The particle's band slots, 8 at a time: all slot loads first, then
        // the partials of every (slot, strip) in band and strip order.
        const int spb = geo.BH / geo.R;
        const int b0 = q.y0 / geo.BH;
        const int nb = min(q.y1 / geo.BH - b0 + 1, a.w.slotmap_ppp);
        const int32_t *sm = a.w.slotmap + (size_t)p * a.w.slotmap_ppp;
        for (int j0 = 0; j0 < nb; j0 += 8) {
            int slot[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) slot[j] = j0 + j < nb ? sm[j0 + j] : -1;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (slot[j] < 0) continue;
                const int b = b0 + j0 + j;
                const float4 *src =
                    reinterpret_cast<const float4 *>(a.part + (size_t)(sc.pair0 + slot[j]) * spb * 8);
                for (int k = 0; k < spb; ++k) {
                    const int r0 = b * geo.BH + k * geo.R;
                    if (r0 > q.y1 || r0 + geo.R - 1 < q.y0) continue;
                    const float4 u = src[2 * k], v = src[2 * k + 1];
                    acc[0] += u.x;
                    acc[1] += u.y;
                    acc[2] += u.z;
                    acc[3] += u.w;
                    acc[4] += v.x;
                    acc[5] += v.y;
                    acc[6] += v.z;
                    acc[7] += v.w;
                }
            }
        }
    }
#pragma unroll
    for (int f = 0; f < 8; ++f) a.grad_soa[(int64_t)f * a.ld + p] = acc[f];
    a.grad_soa[(int64_t)8 * a.ld + p] = 0.f;
}

template <int N>
struct BwdLaunch {
    static cudaError_t rows(const BwdRowsArgs &a, cudaStream_t st) {
        return launch_chain(k_bwd_rows<N>, dim3(a.geo.nstrips, a.S * a.K), kThreads,
                            strip_inverse_smem(N), st, a);
    }
    static cudaError_t column(const BwdColumnArgs &a, cudaStream_t st) {
        return launch_chain(k_bwd_column<N>, dim3(a.geo.nblocks, a.S), kThreads, bwd_column_smem(N),
                            st, a);
    }
    static cudaError_t strip(const BwdStripArgs &a, cudaStream_t st) {
        return launch_chain(k_bwd_strip<N>, dim3(a.geo.nstrips, a.S), kThreads, bwd_strip_smem(N), st,
                            a);
    }
    static cudaError_t prepare(int which) {
        if (which == 0)
            return cudaFuncSetAttribute(k_bwd_rows<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)strip_inverse_smem(N));
        if (which == 1)
            return cudaFuncSetAttribute(k_bwd_column<N>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)bwd_column_smem(N));
        return cudaFuncSetAttribute(k_bwd_strip<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)bwd_strip_smem(N));
    }
};

template <int N>
struct BwdRows {
    static cudaError_t run(const BwdRowsArgs &a, cudaStream_t st) { return BwdLaunch<N>::rows(a, st); }
};
template <int N>
struct BwdColumn {
    static cudaError_t run(const BwdColumnArgs &a, cudaStream_t st) { return BwdLaunch<N>::column(a, st); }
};
template <int N>
struct BwdStrip {
    static cudaError_t run(const BwdStripArgs &a, cudaStream_t st) { return BwdLaunch<N>::strip(a, st); }
};
template <int N>
struct BwdPrepare {
    static cudaError_t run(int which) { return BwdLaunch<N>::prepare(which); }
};

}  // namespace

size_t bwd_column_smem(int H) {
    const int L = set_elems(H) / H;
    return (size_t)2 * L * line_stride(H) * sizeof(float2) + (size_t)kMaxModes * L * sizeof(int2) +
           (kThreads / 32) * 4 * sizeof(float);
}

size_t bwd_strip_smem(int W) {
    const int L = set_elems(W) / W;
    const size_t gather = kThreads * (sizeof(PRec) + sizeof(Rect) + sizeof(int)) + 64;
    return (size_t)2 * L * line_stride(W) * sizeof(float2) +
           (gather > raster_smem<kThreads>() ? gather : raster_smem<kThreads>());
}

cudaError_t prepare_backward(int H, int W) {
    cudaError_t e = dispatch_n<BwdPrepare>(W, 0);
    if (e == cudaSuccess) e = dispatch_n<BwdPrepare>(H, 1);
    if (e == cudaSuccess) e = dispatch_n<BwdPrepare>(W, 2);
    return e;
}

cudaError_t launch_bwd_rows(const BwdRowsArgs &a, cudaStream_t st) {
    return dispatch_n<BwdRows>(a.geo.W, a, st);
}
cudaError_t launch_bwd_column(const BwdColumnArgs &a, cudaStream_t st) {
    return dispatch_n<BwdColumn>(a.geo.H, a, st);
}
cudaError_t launch_bwd_strip(const BwdStripArgs &a, cudaStream_t st) {
    return dispatch_n<BwdStrip>(a.geo.W, a, st);
}
cudaError_t launch_bwd_reduce(const BwdReduceArgs &a, cudaStream_t st) {
    return launch_chain(k_bwd_reduce, dim3(a.nchunks + a.S), kChunk, 0, st, a);
}

}  // namespace osog
