// Particle setup and deterministic particle-to-band binning.
//
// The composition step of the paper (Sec. III.C, Eq. 7) scatters every
// particle's patch into the canvas with an atomic accumulate.  Here the
// canvas is instead gathered per pixel in a fixed particle order, so the
// sum is deterministic and needs no floating-point atomics.  To find the
// particles that can touch a strip of rows, particles are binned to bands
// of BH rows:
//
//   count  (one CTA per chunk of 256 particles): per-particle setup (record,
//          bounding rectangle, band range), then per band a warp ballot of
//          the particles that overlap it; per-warp counts are summed into
//          cnt[chunk][band].
//   scan   (one CTA per scene): exclusive prefix of cnt over the scene's
//          chunks for every band, then over bands, giving each band's list
//          start in the scene's pair region.
//          The same kernel bounds, per scene, the columns that any pupil
//          passes (the column kernels compute the exact chords).
//   fill   (one CTA per chunk): the ballots again; a particle's slot is the
//          band start + chunk prefix + earlier warps of the chunk + the
//          popcount of lower lanes.  Each band list is therefore in
//          ascending particle order.
#include <math.h>

#include "osog_kernels.h"

namespace osog {

namespace {

__device__ __forceinline__ int scene_of_chunk(const GroupDev &gd, int chunk) {
    int s = 0;
    for (int t = 1; t < gd.S; ++t)
        if (gd.sc[t].chunk0 <= chunk) s = t;
    return s;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Band range [b0, b1] of a particle from its rectangle (b0 > b1: none).
__device__ __forceinline__ void band_range(const Rect &r, int BH, int &b0, int &b1) {
    if (r.x0 > r.x1 || r.y0 > r.y1) {
        b0 = 1;
        b1 = 0;
    } else {
        b0 = r.y0 / BH;
        b1 = r.y1 / BH;
    }
}

// Kind-2 setup: every plane a . (u, v, z) <= b of the particle, with the
// local frame u = dx (c ex + s ey), v = dx (-s ex + c ey) of the pixel
// offset (ex, ey) from the centre, becomes a bound affine in (ex, ey):
//   a . (u, v) = kx ex + ky ey,  kx = dx (a_x c - a_y s),  ky = dx (a_x s + a_y c),
//   a_z > 0:  z <= (b - kx ex - ky ey) / a_z      (w = +1)
//   a_z < 0:  z >= (b - kx ex - ky ey) / a_z      (w = -1)
//   a_z = 0:  inside iff b - kx ex - ky ey >= 0   (w =  0)
// stored as (c0, cx, cy, w) with the bound c0 - cx ex - cy ey, in double
// precision rounded once.  False if a plane is not finite.
__device__ bool setup_planes(const Work &w, int off, int m, double c, double s, double dx) {
    for (int i = 0; i < m; ++i) {
        const float4 pl = __ldg(w.planes + off + i);
        if (!isfinite(pl.x) || !isfinite(pl.y) || !isfinite(pl.z) || !isfinite(pl.w)) return false;
        const double kx = dx * ((double)pl.x * c - (double)pl.y * s);
        const double ky = dx * ((double)pl.x * s + (double)pl.y * c);
        const double az = pl.z;
        const double d = az != 0.0 ? az : 1.0;
        w.plane_coef[off + i] = make_float4((float)((double)pl.w / d), (float)(kx / d),
                                            (float)(ky / d), az > 0.0 ? 1.f : (az < 0.0 ? -1.f : 0.f));
    }
    return true;
}

// Setup of one particle: validation, float-float record, bounding rect.
__device__ Rect setup_particle(const float *soa, int64_t ld, int p, const SceneDev &sc,
                               const Geometry &geo, const Work &w) {
    PRec *rec = w.rec;
    int32_t *status = w.status;
    float f[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) f[k] = __ldg(soa + (int64_t)k * ld + p);
    const Rect empty = {1, 0, 1, 0};
    bool finite = true;
#pragma unroll
    for (int k = 0; k < 9; ++k) finite = finite && isfinite(f[k]);
    if (!finite) {
        latch(status, OSOG_ERR_NONFINITE_INPUT);
        return empty;
    }
    const float cx = f[0], cy = f[1], th = f[2], a = f[3], b = f[4], T = f[5];
    const float kind = f[8];
    if (!(a > 0.f) || !(b > 0.f) || !(T >= 0.f) || !(kind == 0.f || kind == 1.f || kind == 2.f)) {
        latch(status, OSOG_ERR_INVALID_PARTICLE);
        return empty;
    }
    int poff = 0, pcnt = 0;
    if (kind == 2.f) {  // planes given, 1..kMaxPlanes of them, inside the list
        if (!w.planes || !w.plane_off || !w.plane_coef) {
            latch(status, OSOG_ERR_INVALID_PARTICLE);
            return empty;
        }
        poff = __ldg(w.plane_off + p);
        pcnt = __ldg(w.plane_off + p + 1) - poff;
        if (poff < 0 || pcnt < 1 || pcnt > kMaxPlanes || poff + pcnt > w.n_planes) {
            latch(status, OSOG_ERR_INVALID_PARTICLE);
            return empty;
        }
    }
    // cos and sin of the angle in float-float on the FP32 pipes (angles
    // beyond 2^20 rad, a case of no physical use, in double)
    ff cf, sf;
    if (fabsf(th) <= kMaxReducedAngle) {
        ff_sincos(th, &cf, &sf);
    } else {
        double sd, cd;
        sincos((double)th, &sd, &cd);
        cf.h = (float)cd;
        cf.l = (float)(cd - (double)cf.h);
        sf.h = (float)sd;
        sf.l = (float)(sd - (double)sf.h);
    }
    PRec r;
    r.cx = cx;
    r.cy = cy;
    r.ch = cf.h;
    r.cl = cf.l;
    r.sh = sf.h;
    r.sl = sf.l;
    r.T = T;
    r.dn = f[6];
    r.mu = f[7];
    float ex, ey;
    const float c = fabsf(r.ch), s = fabsf(r.sh);
    RRec rr;
    rr.cx = cx;
    rr.cy = cy;
    rr.tsa = 0.f;
    rr.dn = f[6];
    rr.mu = f[7];
    if (kind == 2.f) {
        const double cd = (double)cf.h + (double)cf.l, sd = (double)sf.h + (double)sf.l;
        if (!setup_planes(w, poff, pcnt, cd, sd, (double)sc.dx_um)) {
            latch(status, OSOG_ERR_NONFINITE_INPUT);
            return empty;
        }
        r.p0h = __int_as_float(poff);
        r.p0l = 0.f;
        r.p1h = __int_as_float(pcnt);
        r.p1l = 0.f;
        r.g = -1.f;  // marks a general polyhedron
        ex = ey = a;  // circumscribed radius of the footprint (px)
        rr.p[0] = __int_as_float(poff);
        rr.p[1] = __int_as_float(pcnt);
        rr.p[2] = rr.p[3] = rr.p[4] = rr.p[5] = 0.f;
        rr.kind = 2;
    } else if (kind == 1.f) {
        r.p0h = a;
        r.p0l = 0.f;
        r.p1h = b;
        r.p1l = 0.f;
        r.g = sc.prism_g;
        ex = a * c + b * s;
        ey = a * s + b * c;
        rr.p[0] = r.ch;
        rr.p[1] = r.sh;
        rr.p[2] = a;
        rr.p[3] = b;
        rr.p[4] = sc.prism_g;
        rr.p[5] = T;
        rr.kind = 1;
    } else {
        const ff ia = ff_recip(a), ib = ff_recip(b);
        r.p0h = ia.h;
        r.p0l = ia.l;
        r.p1h = ib.h;
        r.p1l = ib.l;
        r.g = 0.f;
        ex = sqrtf(a * a * c * c + b * b * s * s);
        ey = sqrtf(a * a * s * s + b * b * c * c);
        // the row quadric of (u/a)^2 + (v/b)^2 (see RRec), in float-float
        const Quadric q = ellipse_quadric(a, b, cf, sf);
        rr.p[0] = q.m.h;
        rr.p[1] = q.m.l;
        rr.p[2] = q.inv_alpha.h;
        rr.p[3] = q.inv_alpha.l;
        rr.p[4] = q.kappa.h;
        rr.p[5] = q.kappa.l;
        rr.tsa = f_fma(T, q.sqrt_alpha.l, f_mul(T, q.sqrt_alpha.h));
        rr.kind = 0;
    }
    rec[p] = r;
    w.rrec[p] = rr;
    // Pixel centres j + 0.5 inside [cx - ex, cx + ex], widened by one pixel
    // on each side; the thickness is exactly zero on the extra pixels.
    const float xl = floorf(cx - ex - 1.5f), xh = ceilf(cx + ex + 0.5f);
    const float yl = floorf(cy - ey - 1.5f), yh = ceilf(cy + ey + 0.5f);
    if (xh < 0.f || yh < 0.f || xl > (float)(geo.W - 1) || yl > (float)(geo.H - 1))
        return empty;
    Rect q;
    q.x0 = (int16_t)fmaxf(xl, 0.f);
    q.x1 = (int16_t)fminf(xh, (float)(geo.W - 1));
    q.y0 = (int16_t)fmaxf(yl, 0.f);
    q.y1 = (int16_t)fminf(yh, (float)(geo.H - 1));
    return q;
}

// Hull [lo, hi] of the signed column frequencies that any modality of scene
// s may pass: for a pupil, the columns with (fx / (W dx) + ox)^2 <= r2,
// widened by one column on each side (rounding); every column for the other
// operations.  Columns outside the hull are never read or written; the
// column kernels decide the rest from the exact chords.
__device__ int2 column_hull(const GroupDev &gd, int s, const Geometry &geo) {
    const double wlo = -(double)(geo.W / 2), whi = (double)(geo.W / 2 - 1);
    int lo = INT32_MAX, hi = INT32_MIN;
    for (int m = 0; m < gd.K; ++m) {
        const ModeDev &md = gd.md[s][m];
        double a = wlo, b = whi;
        if (md.op == kOpPupil) {
            const double r = sqrt(md.r2);
            a = fmin(fmax(floor((-r - md.ox) / md.fx_scale) - 1.0, wlo), whi + 1.0);
            b = fmax(fmin(ceil((r - md.ox) / md.fx_scale) + 1.0, whi), wlo - 1.0);
        }
        if (a <= b) {
            lo = min(lo, (int)a);
            hi = max(hi, (int)b);
        }
    }
    return make_int2(lo, hi);
}

__global__ void __launch_bounds__(kChunk)
k_bin_count(const float *__restrict__ soa, int64_t ld, const __grid_constant__ GroupDev gd,
            Geometry geo, Work w) {
    __shared__ int wcnt[kChunk / 32][kMaxBands];
    pdl_enter();
    const int chunk = blockIdx.x;
    const int s = scene_of_chunk(gd, chunk);
    const SceneDev &sc = gd.sc[s];
    const int local = (chunk - sc.chunk0) * kChunk + threadIdx.x;
    const bool mine = local < sc.n;
    const int p = sc.p0 + local;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < (kChunk / 32) * kMaxBands; i += kChunk) (&wcnt[0][0])[i] = 0;
    int b0 = 1, b1 = 0;
    if (mine) {
        Rect r = setup_particle(soa, ld, p, sc, geo, w);
        w.rect[p] = r;
        band_range(r, geo.BH, b0, b1);
    }
    __syncthreads();
    const bool any = b0 <= b1;
    const int lo = __reduce_min_sync(0xffffffffu, any ? b0 : kMaxBands);
    const int hi = __reduce_max_sync(0xffffffffu, any ? b1 : -1);
    for (int b = lo; b <= hi; ++b) {
        const unsigned m = __ballot_sync(0xffffffffu, any && b0 <= b && b <= b1);
        if (lane == 0) wcnt[warp][b] = __popc(m);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < geo.nbands; b += kChunk) {
        int t = 0;
#pragma unroll
        for (int k = 0; k < kChunk / 32; ++k) t += wcnt[k][b];
        w.cnt[(int64_t)chunk * geo.nbands + b] = t;
    }
}

// Scan of one scene's band counts (CTA s): for every band the exclusive
// prefix over the scene's chunks, in place; then the bands' starts and the
// scene's column hull.  The counts are laid out [chunk][band], so a band's
// column is strided: the CTA moves tiles of kScanTile chunks x all bands
// between global memory and shared memory with coalesced accesses (one
// 128-byte line per 32 counts instead of one line per count) and scans the
// columns in shared memory, two bands per warp, one or two chunks per lane,
// carrying each band's running total from tile to tile.
constexpr int kScanTile = 64;

__global__ void __launch_bounds__(1024)
k_bin_scan(const __grid_constant__ GroupDev gd, Geometry geo, Work w) {
    __shared__ int tile[kScanTile][kMaxBands + 1];  // one pad word: conflict-free columns
    __shared__ int run[kMaxBands];
    pdl_enter();
    const int s = blockIdx.x;
    const SceneDev &sc = gd.sc[s];
    const int nch = (s + 1 < gd.S ? gd.sc[s + 1].chunk0 : gd.nchunks) - sc.chunk0;
    const int nb = geo.nbands;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 992)  // lane 0 of the last warp
        w.colrange[s] = column_hull(gd, s, geo);
    if ((int)threadIdx.x < nb) run[threadIdx.x] = 0;
    int32_t *cnt = w.cnt + (int64_t)sc.chunk0 * nb;  // [nch][nb]
    for (int t0 = 0; t0 < nch; t0 += kScanTile) {
        const int nt = min(kScanTile, nch - t0);
        for (int e = threadIdx.x; e < nt * nb; e += 1024)
            tile[e / nb][e % nb] = cnt[(int64_t)t0 * nb + e];
        __syncthreads();
        for (int b = warp; b < nb; b += 32) {
            const int v0 = lane < nt ? tile[lane][b] : 0;
            const int v1 = lane + 32 < nt ? tile[lane + 32][b] : 0;
            int i0 = v0, i1 = v1;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, i0, d);
                const int u = __shfl_up_sync(0xffffffffu, i1, d);
                if (lane >= d) {
                    i0 += t;
                    i1 += u;
                }
            }
            const int tot0 = __shfl_sync(0xffffffffu, i0, 31);
            const int tot1 = __shfl_sync(0xffffffffu, i1, 31);
            const int base = run[b];
            if (lane < nt) tile[lane][b] = base + i0 - v0;
            if (lane + 32 < nt) tile[lane + 32][b] = base + tot0 + i1 - v1;
            __syncwarp();
            if (lane == 0) run[b] = base + tot0 + tot1;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nt * nb; e += 1024)
            cnt[(int64_t)t0 * nb + e] = tile[e / nb][e % nb];
        __syncthreads();  // the tile is written back before the next one is loaded
    }
    __syncthreads();  // (a scene without chunks: run[] initialised)
    if (warp == 0) {  // the bands' starts: exclusive over the bands, two per lane (nbands <= 64)
        const int ba = 2 * lane, bb = ba + 1;
        const int ta = ba < nb ? run[ba] : 0, tb = bb < nb ? run[bb] : 0;
        int inc = ta + tb;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += t;
        }
        int32_t *off = w.band_off + (int64_t)s * (nb + 1);
        if (ba < nb) off[ba] = inc - ta - tb;
        if (bb < nb) off[bb] = inc - tb;
        const int all = __shfl_sync(0xffffffffu, inc, 31);
        if (lane == 0) {
            off[nb] = all;
            if (all > sc.pair_cap) latch(w.status, OSOG_ERR_BIN_OVERFLOW);
        }
    }
}

__global__ void __launch_bounds__(kChunk)
k_bin_fill(const __grid_constant__ GroupDev gd, Geometry geo, Work w) {
    __shared__ int wpre[kChunk / 32][kMaxBands];
    __shared__ int start[kMaxBands];  // band list start + this chunk's prefix
    pdl_enter();
    const int chunk = blockIdx.x;
    const int s = scene_of_chunk(gd, chunk);
    const SceneDev &sc = gd.sc[s];
    const int local = (chunk - sc.chunk0) * kChunk + threadIdx.x;
    const bool mine = local < sc.n;
    const int p = sc.p0 + local;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t *off = w.band_off + (int64_t)s * (geo.nbands + 1);
    const int32_t *pre = w.cnt + (int64_t)chunk * geo.nbands;
    for (int i = threadIdx.x; i < (kChunk / 32) * kMaxBands; i += kChunk) (&wpre[0][0])[i] = 0;
    for (int b = threadIdx.x; b < geo.nbands; b += kChunk) start[b] = off[b] + pre[b];
    int b0 = 1, b1 = 0;
    Rect pr{};
    if (mine) {
        pr = w.rect[p];
        band_range(pr, geo.BH, b0, b1);
        if (b0 <= b1) pr.x1 = (int16_t)(pr.x1 | (w.rrec[p].kind << 12));
    }
    __syncthreads();
    const bool any = b0 <= b1;
    const int lo = __reduce_min_sync(0xffffffffu, any ? b0 : kMaxBands);
    const int hi = __reduce_max_sync(0xffffffffu, any ? b1 : -1);
    for (int b = lo; b <= hi; ++b) {
        const unsigned m = __ballot_sync(0xffffffffu, any && b0 <= b && b <= b1);
        if (lane == 0) wpre[warp][b] = __popc(m);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < geo.nbands; b += kChunk) {  // exclusive over warps
        int acc = 0;
#pragma unroll
        for (int k = 0; k < kChunk / 32; ++k) {
            const int t = wpre[k][b];
            wpre[k][b] = acc;
            acc += t;
        }
    }
    __syncthreads();
    const unsigned lt = lanemask_lt();
    for (int b = lo; b <= hi; ++b) {
        const bool in = any && b0 <= b && b <= b1;
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) {
            const int slot = start[b] + wpre[warp][b] + __popc(m & lt);
            if (slot < sc.pair_cap) {
                w.pairs[sc.pair0 + slot] = p;
                if (w.pair_rect) w.pair_rect[sc.pair0 + slot] = pr;
            }
            if (w.slotmap && b - b0 < w.slotmap_ppp)
                w.slotmap[(size_t)p * w.slotmap_ppp + (b - b0)] = slot < sc.pair_cap ? slot : -1;
        }
    }
}

// One scene of at most kChunk particles: count, scan and fill in one CTA.
// The slots are those of the three kernels (band start, then the earlier
// warps, then the lower lanes: ascending particle order in every band list),
// and the scene's column hull is bounded as in the scan.
__global__ void __launch_bounds__(kChunk)
k_bin_single(const float *__restrict__ soa, int64_t ld, const __grid_constant__ GroupDev gd,
             Geometry geo, Work w) {
    __shared__ int wpre[kChunk / 32][kMaxBands];
    __shared__ int start[kMaxBands];
    pdl_enter();
    const SceneDev &sc = gd.sc[0];
    const int local = threadIdx.x;
    const bool mine = local < sc.n;
    const int p = sc.p0 + local;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < (kChunk / 32) * kMaxBands; i += kChunk) (&wpre[0][0])[i] = 0;
    int b0 = 1, b1 = 0;
    Rect pr{};
    if (mine) {
        const Rect r = setup_particle(soa, ld, p, sc, geo, w);
        w.rect[p] = r;
        band_range(r, geo.BH, b0, b1);
        pr = r;
        if (b0 <= b1) pr.x1 = (int16_t)(pr.x1 | (w.rrec[p].kind << 12));
    }
    __syncthreads();
    const bool any = b0 <= b1;
    const int lo = __reduce_min_sync(0xffffffffu, any ? b0 : kMaxBands);
    const int hi = __reduce_max_sync(0xffffffffu, any ? b1 : -1);
    for (int b = lo; b <= hi; ++b) {
        const unsigned m = __ballot_sync(0xffffffffu, any && b0 <= b && b <= b1);
        if (lane == 0) wpre[warp][b] = __popc(m);
    }
    __syncthreads();
    int total = 0;
    if (threadIdx.x < geo.nbands) {  // exclusive over the warps, in place
        const int b = threadIdx.x;
#pragma unroll
        for (int k = 0; k < kChunk / 32; ++k) {
            const int t = wpre[k][b];
            wpre[k][b] = total;
            total += t;
        }
        start[b] = total;
    }
    __syncthreads();
    if (warp == 0) {  // exclusive over the bands, two per lane (nbands <= 64)
        const int ba = 2 * lane, bb = ba + 1;
        const int ta = ba < geo.nbands ? start[ba] : 0, tb = bb < geo.nbands ? start[bb] : 0;
        int inc = ta + tb;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += t;
        }
        const int all = __shfl_sync(0xffffffffu, inc, 31);
        __syncwarp();
        int32_t *off = w.band_off;  // scene 0
        if (ba < geo.nbands) {
            start[ba] = inc - ta - tb;
            off[ba] = inc - ta - tb;
        }
        if (bb < geo.nbands) {
            start[bb] = inc - tb;
            off[bb] = inc - tb;
        }
        if (lane == 0) {
            off[geo.nbands] = all;
            if (all > sc.pair_cap) latch(w.status, OSOG_ERR_BIN_OVERFLOW);
            w.colrange[0] = column_hull(gd, 0, geo);
        }
    }
    __syncthreads();
    const unsigned lt = lanemask_lt();
    for (int b = lo; b <= hi; ++b) {
        const bool in = any && b0 <= b && b <= b1;
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) {
            const int slot = start[b] + wpre[warp][b] + __popc(m & lt);
            if (slot < sc.pair_cap) {
                w.pairs[sc.pair0 + slot] = p;
                if (w.pair_rect) w.pair_rect[sc.pair0 + slot] = pr;
            }
            if (w.slotmap && b - b0 < w.slotmap_ppp)
                w.slotmap[(size_t)p * w.slotmap_ppp + (b - b0)] = slot < sc.pair_cap ? slot : -1;
        }
    }
}

}  // namespace

cudaError_t launch_bin_count(const float *soa, int64_t ld, const GroupDev &gd,
                             const Geometry &geo, const Work &w, cudaStream_t st) {
    if (gd.nchunks == 0) return cudaSuccess;
    return launch_chain(k_bin_count, dim3(gd.nchunks), kChunk, 0, st, soa, ld, gd, geo, w);
}

cudaError_t launch_bin_scan(const GroupDev &gd, const Geometry &geo, const Work &w,
                            cudaStream_t st) {
    return launch_chain(k_bin_scan, dim3(gd.S), 1024, 0, st, gd, geo, w);
}

cudaError_t launch_bin_single(const float *soa, int64_t ld, const GroupDev &gd,
                              const Geometry &geo, const Work &w, cudaStream_t st) {
    return launch_chain(k_bin_single, dim3(1), kChunk, 0, st, soa, ld, gd, geo, w);
}

cudaError_t launch_bin_fill(const GroupDev &gd, const Geometry &geo, const Work &w,
                            cudaStream_t st) {
    if (gd.nchunks == 0) return cudaSuccess;
    return launch_chain(k_bin_fill, dim3(gd.nchunks), kChunk, 0, st, gd, geo, w);
}

}  // namespace osog
