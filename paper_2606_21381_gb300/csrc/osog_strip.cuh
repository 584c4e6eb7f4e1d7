// Device pieces shared by the forward and adjoint render kernels: the
// fixed-point strip raster, the transfer functions of the optical head, and
// a dispatcher over the power-of-two transform sizes.
#pragma once

#include "osog_fft.cuh"
#include "osog_kernels.h"

namespace osog {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }
__host__ __device__ constexpr int clog2(int v) { return v <= 1 ? 0 : 1 + clog2(v >> 1); }

// Rows per strip and columns per column block of a square N x N canvas
// (both min(set_elems(N) / N, N)); kernels specialised for square canvases use
// these compile-time values instead of the geometry's.
__host__ __device__ constexpr int sq_rb(int n) { return set_elems(n) / n < n ? set_elems(n) / n : n; }

// ------------------------------------------------------------ raster
// Composition of a strip's OPD and ATT (Eq. 2's integral over z, Eq. 7's
// accumulate) by integer addition in shared memory.  Every (particle, pixel)
// contribution is rounded once to a fixed-point integer and added with a
// shared-memory atomic; integer sums do not depend on their order, so the
// strip is bitwise the same whichever lane, warp or strip adds what (the
// batched and per-scene paths and every band height agree bit for bit).
//   kAccPhase (render, adjoint): per pixel a uint32 phase in units of 2^-23
//     cycles of dn t / lambda, summed modulo 2^32 (only the phase modulo one
//     cycle enters exp(i 2 pi OPD / lambda)), and an int32 absorption
//     exponent in units of 2^-20 with each particle's mu t clamped to
//     [-16, 16] (past e^-16 of amplitude a particle is opaque; the sum stays
//     in range while fewer than 128 such particles overlap a pixel).
//   kAccOpd (osog_render_opd): int64 OPD and ATT in units of 2^-32 um.
// Work proceeds per (particle, row) item: the row's span of pixel centres
// inside the footprint is found analytically (the ellipse's chord ends, the
// rotated rectangle's slab crossings), and the CTA's lanes are packed over
// the items' pixels, up to four per lane.
enum { kAccPhase = 0, kAccOpd = 1 };

struct __align__(16) RowItem {
    uint32_t hdr;   // first column j0 (bits 0-11), pixel count (12-23), kind (24-25)
    float f[8];     // ellipsoid: left and right chord ends (hi, lo each), T sqrt(alpha)
                    // prism: cx, g s ey, g c ey, g cos, g sin, g hx, g hy, T
                    // polyhedron: cx, ey, plane offset, plane count (int bits)
    int32_t row;    // row in the rasterised region
    float dn;       // kAccPhase: dn / lambda (cycles per um); kAccOpd: dn
    float mu;       // kAccPhase: mu in units of 2^-20 per um; kAccOpd: mu
};
static_assert(sizeof(RowItem) == 48, "RowItem is 48 bytes");

// Square root of a float-float a (a.h > 0): a float estimate s, then one
// correction step (a - s^2) / (2 s) with the residual taken exactly by a
// fused multiply-add, which also absorbs the estimate's own rounding.
__device__ __forceinline__ ff ff_sqrt(ff a) {
    const float r = rsqrtf(a.h);
    const float s = a.h * r;
    const float e = __fadd_rn(__fmaf_rn(-s, s, a.h), a.l);
    return fast_two_sum(s, e * (0.5f * r));
}

// The item of particle r on canvas row y (region row `row`), its columns
// clipped to [c0, c1] (inside the particle's bounding rectangle and the
// canvas): false when no pixel centre of the footprint is left.
template <int ACC>
__device__ __forceinline__ bool make_row_item(const RRec &r, int c0, int c1, int y, int row,
                                              float inv_lambda, RowItem &it) {
    const float yc = (float)y + 0.5f;
    float lo, hi;  // span of pixel-centre x, widened below
    float c = 0.f, sn = 0.f, s_ey = 0.f, c_ey = 0.f;
    if (r.kind == 0) {
        const ff ey = two_sum(yc, -r.cy);
        const ff x0 = ff_add(ff{r.cx, 0.f}, ff_mul(ff{r.p[0], r.p[1]}, ey));
        const ff w2 = ff_add(ff{r.p[2], r.p[3]}, ff_neg(ff_mul(ff{r.p[4], r.p[5]}, ff_mul(ey, ey))));
        if (!(w2.h > 0.f)) return false;
        const ff w = ff_sqrt(w2);
        const ff xl = ff_add(x0, ff_neg(w)), xr = ff_add(x0, w);
        it.f[0] = xl.h;
        it.f[1] = xl.l;
        it.f[2] = xr.h;
        it.f[3] = xr.l;
        it.f[4] = r.tsa;
        lo = xl.h;
        hi = xr.h;
    } else if (r.kind == 1) {
        // |c ex + s ey| < hx and |-s ex + c ey| < hy, ex = X - cx
        c = r.p[0];
        sn = r.p[1];
        const float hx = r.p[2], hy = r.p[3];
        const float ey = yc - r.cy;
        s_ey = sn * ey;
        c_ey = c * ey;
        lo = -3.0e38f;
        hi = 3.0e38f;
        if (fabsf(c) > 1e-6f) {
            const float a0 = __fdividef(-hx - s_ey, c), a1 = __fdividef(hx - s_ey, c);
            lo = fmaxf(lo, fminf(a0, a1));
            hi = fminf(hi, fmaxf(a0, a1));
        } else if (!(fabsf(s_ey) < hx + 1.f)) {
            return false;
        }
        if (fabsf(sn) > 1e-6f) {
            const float a0 = __fdividef(c_ey - hy, sn), a1 = __fdividef(c_ey + hy, sn);
            lo = fmaxf(lo, fminf(a0, a1));
            hi = fminf(hi, fmaxf(a0, a1));
        } else if (!(fabsf(c_ey) < hy + 1.f)) {
            return false;
        }
        if (!(lo <= hi)) return false;
        lo += r.cx;
        hi += r.cx;
    } else {
        it.f[0] = r.cx;
        it.f[1] = yc - r.cy;
        it.f[2] = r.p[0];
        it.f[3] = r.p[1];
        lo = (float)c0;
        hi = (float)c1 + 1.f;
    }
    // pixel centres j + 0.5 in [lo, hi], one more column on each side for
    // the rounding of the ends (their thickness evaluates to zero)
    const int j0 = max(c0, (int)floorf(fmaxf(lo - 0.5f, -2.f)) - 1);
    const int j1 = min(c1, (int)ceilf(fminf(hi - 0.5f, 4096.f)) + 1);
    if (j1 < j0) return false;
    if (r.kind == 1) {  // everything in um: g u = g c ex + g s ey, g = 2 s_b dx
        const float g = r.p[4];
        it.f[0] = r.cx;
        it.f[1] = g * s_ey;
        it.f[2] = g * c_ey;
        it.f[3] = g * c;
        it.f[4] = g * sn;
        it.f[5] = g * r.p[2];
        it.f[6] = g * r.p[3];
        it.f[7] = r.p[5];
    }
    it.hdr = (uint32_t)j0 | ((uint32_t)(j1 - j0 + 1) << 12) | ((uint32_t)r.kind << 24);
    it.row = row;
    if constexpr (ACC == kAccPhase) {
        it.dn = r.dn * inv_lambda;
        it.mu = r.mu * 1048576.f;  // the exponent's unit folded in (exact: a power of two)
    } else {
        it.dn = r.dn;
        it.mu = r.mu;
    }
    return true;
}

// Chord t (um) of an item's particle at the pixel centre X of its row, a
// function of the pixel alone (not of where the item's span starts, which
// depends on the tiling); t <= 0 outside the footprint.
//   ellipsoid: t = T sqrt(alpha) sqrt((xr - X)(X - xl)); both factors are
//              taken from the float-float chord ends, so each has a relative
//              error of one rounding even at the rim;
//   prism:     t = clamp(g min(hx - |u|, hy - |v|), 0, T), g = 2 s_b dx,
//              taken as min(g hx - |g u|, g hy - |g v|) capped at T;
//   polyhedron: t = z_hi - z_lo over the pixel-affine plane bounds, 0
//              outside a wall (Eq. 1).
__device__ __forceinline__ float item_chord(const RowItem &it, int kind, float X,
                                            const float4 *__restrict__ coef) {
    if (kind == 0) {
        const float ep = __fadd_rn(__fsub_rn(it.f[2], X), it.f[3]);
        const float en = __fsub_rn(__fsub_rn(X, it.f[0]), it.f[1]);
        const float qq = __fmul_rn(ep, en);
        return qq > 1e-30f ? it.f[4] * qq * rsqrtf(qq) : -1.f;
    }
    const float ex = X - it.f[0];
    if (kind == 1) {
        const float gu = fmaf(it.f[3], ex, it.f[1]);
        const float gv = fmaf(-it.f[4], ex, it.f[2]);
        return fminf(fminf(it.f[5] - fabsf(gu), it.f[6] - fabsf(gv)), it.f[7]);
    }
    const float4 *pc = coef + __float_as_int(it.f[2]);
    const int m = __float_as_int(it.f[3]);
    const float ey = it.f[1];
    float zlo = -INFINITY, zhi = INFINITY;
    bool inside = true;
    for (int i = 0; i < m; ++i) {
        const float4 pl = __ldg(pc + i);
        const float z = fmaf(-pl.y, ex, fmaf(-pl.z, ey, pl.x));
        if (pl.w > 0.f)
            zhi = fminf(zhi, z);
        else if (pl.w < 0.f)
            zlo = fmaxf(zlo, z);
        else
            inside = inside && z >= 0.f;
    }
    return inside && zhi > zlo ? zhi - zlo : -1.f;
}

// Adds one particle's contribution at chord t > 0 to the pixel's accumulators
// at shared-memory address acc (phase mode: a uint2 slot, x the phase in
// 2^-23 cycles, y the absorption exponent in 2^-20; OPD mode: two int64 in
// 2^-32 um).  dn and mu are the item's (phase mode: dn / lambda in cycles
// per um, mu already in 2^-20 per um).  The additions are shared-space reductions issued on the slot's
// shared address (no generic addressing, no returned value).
template <int ACC>
__device__ __forceinline__ void deposit(uint32_t acc, float t, float dn, float mu) {
    if constexpr (ACC == kAccPhase) {
        const float c = t * dn;                   // cycles
        const float r = c - rintf(c);             // in [-1/2, 1/2]
        // round(r 2^23) from the mantissa of r 2^23 + 1.5 2^23
        const int q = __float_as_int(fmaf(r, 8388608.f, 12582912.f)) - 0x4B400000;
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(acc), "r"(q) : "memory");
        if (mu != 0.f) {
            const float x = fminf(fmaxf(t * mu, -16777216.f), 16777216.f);  // |mu t| <= 16
            asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(acc + 4u), "r"(__float2int_rn(x))
                         : "memory");
        }
    } else {
        asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(acc),
                     "l"((unsigned long long)__float2ll_rn(t * dn * 4294967296.f)) : "memory");
        if (mu != 0.f)
            asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(acc + 8u),
                         "l"((unsigned long long)__float2ll_rn(t * mu * 4294967296.f)) : "memory");
    }
}

// Exit wave of a pixel's phase-mode accumulators (Eq. 2 with the
// Beer-Lambert amplitude of Eq. 4): the phase, taken modulo one cycle into
// [-1/2, 1/2) cycles, feeds the hardware sin / cos directly.  An empty
// pixel (both words zero) takes the same path: sin 0, cos 0 and 2^0 are
// exact, so it gives (1, 0) without a branch that would split the warp.
__device__ __forceinline__ float2 exit_wave_fixed(uint2 acc) {
    const int p = (int)(acc.x << 9) >> 9;  // units of 2^-23 cycles
    float s, c;
    __sincosf((float)p * 7.4901405658471572e-07f, &s, &c);              // 2 pi 2^-23
    const float a = __expf((float)(int)acc.y * -9.5367431640625e-07f);  // -2^-20
    return make_float2(a * c, a * s);
}

// Inclusive prefix sum over the lanes of a warp.
__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

// The lane whose range of a warp prefix holds key: the number of lanes whose
// inclusive prefix (field (inc >> sh) & mask, non-decreasing over the lanes)
// is at most key.  Every lane of the warp takes part; the result is at most
// 31, and it is the owning lane whenever key is below lane 31's prefix.
__device__ __forceinline__ int warp_owner(int inc, int key, int sh, int mask) {
    int e = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const int t = (__shfl_sync(kFull, inc, e + s - 1) >> sh) & mask;
        if (t <= key) e += s;
    }
    return e;
}

// Pixels of one chunk of a row item.
constexpr int kChunkPx = 4;

// Shared memory of raster_region beyond the accumulators: one wave of 32
// row items per warp and the CTA's work counter.
template <int NT>
__host__ __device__ constexpr size_t raster_smem() {
    return (size_t)NT * sizeof(RowItem) + 16;
}

// OPD and ATT of the region rows [ty0, ty0 + nrows) x columns [tx0, tx1]
// of scene s from the band list entries [lo, hi) (ids of the scene's
// records; prect, when not null, the entries' rectangles with their kinds,
// else they are gathered by id), added into the accumulators that slot(row, x) addresses (zeroed
// by the caller; kAccPhase: uint2, kAccOpd: two int64).  Each warp works on
// its own groups of 32 list entries (fewer when the list is short, so that
// every warp gets a group; the first NT / 32 groups in warp order, the rest
// handed out by a shared counter as warps finish), with no CTA barrier
// until the end:
//   1. the entries whose rectangle meets the region, compacted with the
//      ellipsoids first, the region rows each covers, and a warp prefix sum
//      of those row counts;
//   2. waves of 32 (particle, row) items, one per lane (the owning entry
//      found by a search over the prefix), built from the particle's
//      row-span constants into the warp's item slots;
//   3. the wave's pixels cut into chunks of up to kChunkPx, ellipsoid items'
//      chunks first so that most passes run one chord formula; lane l of a
//      pass takes chunk l and evaluates its pixels as independent unrolled
//      chains, adding each covered pixel with integer shared-memory
//      reductions (a step past the chunk or outside the footprint adds zero,
//      so the pass has no branch around them).
// Every thread of the CTA must call it; it ends with a CTA barrier.
template <int NT, int ACC, typename Slot>
__device__ void raster_region(const Work &w, const int32_t *ids, const Rect *prect, int lo,
                              int hi, int ty0, int nrows, int tx0, int tx1, float inv_lambda,
                              Slot slot, unsigned char *scratch) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    RowItem *items = reinterpret_cast<RowItem *>(scratch) + warp * 32;
    int *next = reinterpret_cast<int *>(reinterpret_cast<RowItem *>(scratch) + NT);
    const int tyl = ty0 + nrows - 1;
    // group size: 32 entries, or fewer for a short list so that every warp
    // gets some (a small scene's band holds a few dozen entries)
    constexpr int NW = NT / 32;
    const int gsz = min(32, max(1, (hi - lo + NW - 1) / NW));
    if (threadIdx.x == 0) *next = lo + NW * gsz;
    __syncthreads();
    int base = lo + warp * gsz;
    while (base < hi) {
        int nb = 0;
        if (lane == 0) nb = atomicAdd(next, gsz);
        // 1. the group's entries that meet the region, compacted through the
        //    warp's item slots with the ellipsoids first (so that most waves
        //    below build items of one kind)
        int id = 0, nr = 0, ry0 = 0, rx0 = 0, rx1 = 0;
        {
            const int i = base + lane;
            bool ell = false;
            if (lane < gsz && i < hi) {
                id = ids[i];
                Rect q;
                int kind = 0;
                if (prect) {  // the slot's copy: one coalesced load, the kind packed in
                    q = prect[i];
                    kind = (q.x1 >> 12) & 3;
                    q.x1 = (int16_t)(q.x1 & 0xFFF);
                } else {
                    q = w.rect[id];
                }
                ry0 = max((int)q.y0, ty0);
                rx0 = max((int)q.x0, tx0);
                rx1 = min((int)q.x1, tx1);
                nr = rx0 <= rx1 ? max(min((int)q.y1, tyl) - ry0 + 1, 0) : 0;
                if (nr > 0 && !prect) kind = w.rrec[id].kind;
                ell = nr > 0 && kind == 0;
            }
            const unsigned lt = lanemask_lt();
            const unsigned me = __ballot_sync(kFull, ell), mo = __ballot_sync(kFull, nr > 0 && !ell);
            const int ne = __popc(me);
            int4 *tmp = reinterpret_cast<int4 *>(items);
            int *tnr = reinterpret_cast<int *>(tmp + 32);
            if (nr > 0) {
                const int pos = ell ? __popc(me & lt) : ne + __popc(mo & lt);
                tmp[pos] = make_int4(id, ry0, rx0, rx1);
                tnr[pos] = nr;
            }
            __syncwarp();
            const int kept = ne + __popc(mo);
            nr = 0;
            if (lane < kept) {
                const int4 e = tmp[lane];
                id = e.x;
                ry0 = e.y;
                rx0 = e.z;
                rx1 = e.w;
                nr = tnr[lane];
            }
            __syncwarp();  // the slots are read before the first wave writes them
        }
        const int inc = warp_incl_scan(nr);
        const int ex = inc - nr;
        const int total = __shfl_sync(kFull, inc, 31);
        // 2. waves of 32 (particle, row) items
        for (int jb = 0; jb < total; jb += 32) {
            const int j = jb + lane;
            const int e = warp_owner(inc, j, 0, -1);
            const int ide = __shfl_sync(kFull, id, e);
            const int ye = __shfl_sync(kFull, ry0, e) + j - __shfl_sync(kFull, ex, e);
            const int c0 = __shfl_sync(kFull, rx0, e), c1 = __shfl_sync(kFull, rx1, e);
            RowItem it;
            bool valid = false;
            if (j < total)
                valid = make_row_item<ACC>(w.rrec[ide], c0, c1, ye, ye - ty0, inv_lambda, it);
            // 3. chunks: ellipsoid items' count in the low half-word, the
            //    other kinds' in the high one
            const int nch = valid ? (int)((((it.hdr >> 12) & 0xFFFu) + kChunkPx - 1) / kChunkPx) : 0;
            const int mine = valid && ((it.hdr >> 24) & 3u) == 0 ? nch : nch << 16;
            const int cinc = warp_incl_scan(mine);
            const int cex = cinc - mine;
            const int ctot = __shfl_sync(kFull, cinc, 31);
            const int TE = ctot & 0xFFFF, TC = TE + (ctot >> 16);
            if (valid) items[lane] = it;
            __syncwarp();
            for (int cb = 0; cb < TC; cb += 32) {
                const int c = cb + lane;
                const int sh = c < TE ? 0 : 16;
                const int key = c < TE ? c : c - TE;
                const int k = warp_owner(cinc, key, sh, 0xFFFF);
                const int kex = (__shfl_sync(kFull, cex, k) >> sh) & 0xFFFF;
                if (c < TC) {
                    const RowItem rit = items[k];  // registers: the reductions below may not alias it
                    const uint32_t h = rit.hdr;
                    const int j0 = (int)(h & 0xFFFu), cnt = (int)((h >> 12) & 0xFFFu);
                    const int kind = (int)((h >> 24) & 3u);
                    const int k0 = (key - kex) * kChunkPx;
                    const int len = min(kChunkPx, cnt - k0);
                    const int x0 = j0 + k0;
                    float t[kChunkPx];
                    if (kind == 0) {
#pragma unroll
                        for (int u = 0; u < kChunkPx; ++u)
                            t[u] = item_chord(rit, 0, (float)(x0 + u) + 0.5f, nullptr);
                    } else if (kind == 1) {
#pragma unroll
                        for (int u = 0; u < kChunkPx; ++u)
                            t[u] = item_chord(rit, 1, (float)(x0 + u) + 0.5f, nullptr);
                    } else {
#pragma unroll
                        for (int u = 0; u < kChunkPx; ++u)
                            t[u] = u < len ? item_chord(rit, 2, (float)(x0 + u) + 0.5f, w.plane_coef)
                                           : -1.f;
                    }
                    // every step deposits (zero at the chunk's first pixel when the
                    // pixel is past the chunk or outside the footprint): no branch
#pragma unroll
                    for (int u = 0; u < kChunkPx; ++u) {
                        const bool on = u < len && t[u] > 0.f;
                        deposit<ACC>(slot(rit.row, on ? x0 + u : x0), on ? t[u] : 0.f, rit.dn, rit.mu);
                    }
                }
            }
            __syncwarp();  // the wave's items are read before the next wave writes
        }
        base = __shfl_sync(kFull, nb, 0);
    }
    __syncthreads();
}

// The strip [y0, y0 + R) of scene s rasterised into the padded FFT lines of
// an N-point set (the adjoint's re-raster; osog_render_opd in OPD mode).
template <int N, int ACC>
__device__ void raster_strip(const Geometry &geo, const Work &w, const SceneDev &sc, int s,
                             int y0, int R, void *acc, unsigned char *scratch) {
    constexpr int LS = line_stride(N);
    const int band = y0 / geo.BH;
    const int32_t *off = w.band_off + (size_t)s * (geo.nbands + 1);
    const int hi = min(off[band + 1], sc.pair_cap);
    const int lo = min(off[band], hi);
    // shared address of the (row, x) slot: uint2 (phase) or two int64 (OPD)
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(acc);
    auto slot = [base](int row, int x) -> uint32_t {
        return base + (uint32_t)(row * LS + pad16(x)) * (ACC == kAccPhase ? 8u : 16u);
    };
    raster_region<kThreads, ACC>(w, w.pairs + sc.pair0, w.pair_rect ? w.pair_rect + sc.pair0 : nullptr,
                                 lo, hi, y0, R, 0, geo.W - 1, 0.5f * sc.two_over_lambda, slot,
                                 scratch);
}

// Elements of an n-point transform's set handled by each thread in the copy
// loops; the loops are fully unrolled so that every thread has all of its
// global loads in flight at once.
__host__ __device__ constexpr int ept(int n) { return set_elems(n) / kThreads; }

// ------------------------------------------------------------ fast phases
// sin and cos of x with the hardware approximations: x is first reduced to
// [-pi, pi] (x - 2 pi rint(x / 2 pi)), where __sincosf's absolute error is a
// few 1e-7; each turn removed adds at most 1.8e-7 (2 pi rounded to float).
// The transfer-function phases stay within a few turns.
__device__ __forceinline__ void phase_sincos(float x, float *s, float *c) {
    const float r = fmaf(-6.28318530717958648f, rintf(x * 0.159154943091895336f), x);
    __sincosf(r, s, c);
}

// Exit wave (Eq. 2 with the Beer-Lambert amplitude of Eq. 4):
// exp(-att) (cos, sin)(pi opd two_over_lambda), the phase reduced exactly
// in half-turns (x - 2 rint(x / 2)) before the hardware sin / cos.
__device__ __forceinline__ float2 exit_wave(float opd, float att, float two_over_lambda) {
    const float x = opd * two_over_lambda;
    const float r = fmaf(-2.f, rintf(0.5f * x), x);
    float s, c;
    __sincosf(3.14159265358979323846f * r, &s, &c);
    const float a = __expf(-att);
    return make_float2(a * c, a * s);
}

// ------------------------------------------------------------ optical head
// Transfer function at signed frequency (fx, fy) inside the pupil chord,
// including 1/(HW):
// pupil circ * exp(i dz (sqrt(k0^2 - |q|^2) - k0)) at q = k + k_ill (Eq. 3,
// oblique shift), times 2i sin(k . ds + theta) for DIC (Eq. 5).  The defocus
// phase is evaluated as -dz |q|^2 / (sqrt(k0^2 - |q|^2) + k0), which has no
// cancellation for small |q|.
// Every product that could be contracted into a fused multiply-add is
// written out (rounded product or fmaf), so that all kernels round alike.
__device__ __forceinline__ float2 transfer(const ModeDev &md, int fx, int fy) {
    // in focus and not DIC: the pupil is the constant scale (sin 0 and
    // cos 0 are exact, so this is the value the general path gives)
    if (md.dz == 0.f && !md.dic) return make_float2(md.scale, 0.f);
    const float kx = __fmul_rn((float)fx, md.kstep_x), ky = __fmul_rn((float)fy, md.kstep_y);
    const float qx = __fadd_rn(kx, md.qoff_x), qy = __fadd_rn(ky, md.qoff_y);
    const float q2 = fmaf(qx, qx, __fmul_rn(qy, qy));
    const float chi = __fdividef(__fmul_rn(-md.dz, q2),
                                 __fadd_rn(sqrtf(fmaxf(fmaf(md.k0, md.k0, -q2), 0.f)), md.k0));
    float sn, cs;
    phase_sincos(chi, &sn, &cs);
    float2 h = make_float2(cs, sn);
    if (md.dic) {
        float sa, ca;
        phase_sincos(fmaf(kx, md.dsx, fmaf(ky, md.dsy, md.bias)), &sa, &ca);
        const float g = __fmul_rn(2.f, sa);
        h = make_float2(__fmul_rn(-sn, g), __fmul_rn(cs, g));
    }
    return make_float2(__fmul_rn(h.x, md.scale), __fmul_rn(h.y, md.scale));
}

// ---------------------------------------------------------------- layouts
// A row-strip [y0, y0 + R) of a column-blocked array [W/B][H][B] (complex)
// to and from the padded shared lines of an N = W point set.  Columns whose
// signed frequency lies outside [cr.x, cr.y] (no pupil passes them) are
// neither read (zero-filled) nor written.
template <int N, bool SQ = false>
__device__ __forceinline__ void load_strip_blocked(float2 *buf, const float2 *src,
                                                   const Geometry &geo, int y0, int2 cr) {
    constexpr int LS = line_stride(N);
    const int R = SQ ? sq_rb(N) : geo.R, B = SQ ? sq_rb(N) : geo.B;
    const int lb = SQ ? clog2(sq_rb(N)) : ilog2(B), lr = SQ ? clog2(sq_rb(N)) : ilog2(R);
    const int RN = R * N, H = SQ ? N : geo.H;
    float2 v[ept(N)];
#pragma unroll
    for (int i = 0; i < ept(N); ++i) {
        const int e = threadIdx.x + i * kThreads;
        const int c = e & (B - 1), r = (e >> lb) & (R - 1), bk = e >> (lb + lr);
        const int kx = bk * B + c, fx = kx < N / 2 ? kx : kx - N;
        v[i] = e < RN && fx >= cr.x && fx <= cr.y ? src[((size_t)bk * H + y0 + r) * B + c]
                                                  : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < ept(N); ++i) {
        const int e = threadIdx.x + i * kThreads;
        const int c = e & (B - 1), r = (e >> lb) & (R - 1), bk = e >> (lb + lr);
        if (e < RN) buf[r * LS + pad16(bk * B + c)] = v[i];
    }
}

template <int N, bool SQ = false>
__device__ __forceinline__ void store_strip_blocked(const float2 *buf, float2 *dst,
                                                    const Geometry &geo, int y0, int2 cr) {
    constexpr int LS = line_stride(N);
    const int R = SQ ? sq_rb(N) : geo.R, B = SQ ? sq_rb(N) : geo.B;
    const int lb = SQ ? clog2(sq_rb(N)) : ilog2(B), lr = SQ ? clog2(sq_rb(N)) : ilog2(R);
    const int RN = R * N, H = SQ ? N : geo.H;
#pragma unroll
    for (int i = 0; i < ept(N); ++i) {
        const int e = threadIdx.x + i * kThreads;
        const int c = e & (B - 1), r = (e >> lb) & (R - 1), bk = e >> (lb + lr);
        const int kx = bk * B + c, fx = kx < N / 2 ? kx : kx - N;
        if (e < RN && fx >= cr.x && fx <= cr.y)
            dst[((size_t)bk * H + y0 + r) * B + c] = buf[r * LS + pad16(kx)];
    }
}

// A column block (B columns, N = H rows, contiguous [H][B]) to and from the
// padded shared lines (line c = column c).  Inactive columns load as zero.
template <int N>
__device__ __forceinline__ void load_block(float2 *buf, const float2 *src, const Geometry &geo,
                                           int bk, int2 cr) {
    constexpr int LS = line_stride(N);
    const int B = geo.B, lb = ilog2(B), NB = N * B, half = geo.W / 2;
    float2 v[ept(N)];
#pragma unroll
    for (int i = 0; i < ept(N); ++i) {
        const int e = threadIdx.x + i * kThreads;
        const int kx = bk * B + (e & (B - 1)), fx = kx < half ? kx : kx - geo.W;
        v[i] = e < NB && fx >= cr.x && fx <= cr.y ? src[e] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < ept(N); ++i) {
        const int e = threadIdx.x + i * kThreads;
        if (e < NB) buf[(e & (B - 1)) * LS + pad16(e >> lb)] = v[i];
    }
}

template <int N>
__device__ __forceinline__ void store_block(const float2 *buf, float2 *dst, const Geometry &geo) {
    constexpr int LS = line_stride(N);
    const int B = geo.B, lb = ilog2(B), NB = N * B;
#pragma unroll
    for (int i = 0; i < ept(N); ++i) {
        const int e = threadIdx.x + i * kThreads;
        if (e < NB) dst[e] = buf[(e & (B - 1)) * LS + pad16(e >> lb)];
    }
}

// True if some column of block bk has a signed frequency inside cr.
__device__ __forceinline__ bool block_active(const Geometry &geo, int bk, int2 cr) {
    const int u0 = bk * geo.B, u1 = u0 + geo.B - 1, half = geo.W / 2;
    const bool lo = u0 < half && u0 <= cr.y && min(u1, half - 1) >= cr.x;
    const bool hi = u1 >= half && max(u0, half) - geo.W <= cr.y && u1 - geo.W >= cr.x;
    return lo || hi;
}

// Transfer function and its derivatives with respect to (defocus,
// shear_px, shear_angle, bias) at signed frequency (fx, fy) inside the
// pupil chord, including 1/(HW).  With kappa = sqrt(k0^2 - |q|^2) - k0 the
// pupil is P = exp(i dz kappa) and dP/ddz = i kappa P; DIC multiplies by
// i g, g = 2 sin(a), a = k.ds + theta, whose derivatives are 2 cos(a) da.
__device__ __forceinline__ void transfer_grad(const ModeDev &md, int fx, int fy, float2 &h,
                                              float2 dh[4]) {
    const float kx = (float)fx * md.kstep_x, ky = (float)fy * md.kstep_y;
    const float qx = kx + md.qoff_x, qy = ky + md.qoff_y;
    const float q2 = fmaf(qx, qx, qy * qy);
    const float kappa = __fdividef(-q2, sqrtf(fmaxf(fmaf(md.k0, md.k0, -q2), 0.f)) + md.k0);
    float sn, cs;
    phase_sincos(md.dz * kappa, &sn, &cs);
    const float sc = md.scale;
    if (!md.dic) {
        h = make_float2(cs * sc, sn * sc);
        dh[0] = make_float2(-sn * kappa * sc, cs * kappa * sc);
        dh[1] = dh[2] = dh[3] = make_float2(0.f, 0.f);
        return;
    }
    float sa, ca;
    phase_sincos(fmaf(kx, md.dsx, fmaf(ky, md.dsy, md.bias)), &sa, &ca);
    const float g = 2.f * sa, gp = 2.f * ca;
    h = make_float2(-sn * g * sc, cs * g * sc);
    dh[0] = make_float2(-cs * kappa * g * sc, -sn * kappa * g * sc);
    const float da[3] = {fmaf(kx, md.dsx1, ky * md.dsy1), fmaf(-kx, md.dsy, ky * md.dsx), 1.f};
#pragma unroll
    for (int k = 0; k < 3; ++k) dh[k + 1] = make_float2(-sn * gp * da[k] * sc, cs * gp * da[k] * sc);
}

// Adds to acc[0..7] the contribution of one pixel to dL/d(cx, cy, theta,
// a|hx, b|hy, T, dn, mu) of particle r, given go = dL/dOPD and
// ga = dL/dATT at the pixel centre (x, y): dn and mu collect t go and
// t ga; the geometry collects (dn go + mu ga) dt/d(field).
//   ellipsoid: t = T sqrt(delta), delta = 1 - u'^2 - v'^2, u' = u/a,
//     v' = v/b; d delta/d(cx, cy) = 2 (u' c/a - v' s/b, u' s/a + v' c/b),
//     d delta/d theta = 2 u' v' (a/b - b/a), d delta/d(a, b) = 2 (u'^2/a,
//     v'^2/b); delta comes from float-float inside the rim band.
//   prism: t = clamp(g d, 0, T), d = min(hx - |u|, hy - |v|): on the ramp
//     dt = g dd with dd/d(hx or hy) = 1 and the chain through |u| or |v|;
//     on the plateau dt/dT = 1.
__device__ __forceinline__ void thickness_grad(const PRec &r, float xc, float yc, float go,
                                               float ga, float acc[8]) {
    const float ex = xc - r.cx, ey = yc - r.cy;
    const float wgt = fmaf(r.dn, go, r.mu * ga);
    if (r.g > 0.f) {
        const float u = fmaf(r.ch, ex, r.sh * ey);
        const float v = fmaf(-r.sh, ex, r.ch * ey);
        const float du = r.p0h - fabsf(u), dv = r.p1h - fabsf(v);
        const float gd = r.g * fminf(du, dv);
        if (!(gd > 0.f)) return;
        const float t = fminf(gd, r.T);
        acc[6] = fmaf(go, t, acc[6]);
        acc[7] = fmaf(ga, t, acc[7]);
        if (gd >= r.T) {
            acc[5] += wgt;
            return;
        }
        const float q = wgt * r.g;
        if (du <= dv) {
            const float sq = u >= 0.f ? q : -q;
            acc[0] = fmaf(sq, r.ch, acc[0]);
            acc[1] = fmaf(sq, r.sh, acc[1]);
            acc[2] = fmaf(-sq, v, acc[2]);
            acc[3] += q;
        } else {
            const float sq = v >= 0.f ? q : -q;
            acc[0] = fmaf(-sq, r.sh, acc[0]);
            acc[1] = fmaf(sq, r.ch, acc[1]);
            acc[2] = fmaf(sq, u, acc[2]);
            acc[4] += q;
        }
        return;
    }
    const float cia = r.ch * r.p0h, sia = r.sh * r.p0h;
    const float cib = r.ch * r.p1h, sib = r.sh * r.p1h;
    const float ua = fmaf(cia, ex, sia * ey);
    const float vb = fmaf(-sib, ex, cib * ey);
    float delta = 1.f - fmaf(ua, ua, vb * vb);
    if (delta < kRimBand) {
        if (delta <= -kRimBand) return;
        delta = ellipse_delta_ff(r, xc, yc);
        if (!(delta > 0.f)) return;
    }
    const float rs = rsqrtf(delta);
    const float sq = delta * rs;
    const float t = r.T * sq;
    acc[6] = fmaf(go, t, acc[6]);
    acc[7] = fmaf(ga, t, acc[7]);
    acc[5] = fmaf(wgt, sq, acc[5]);
    const float q = wgt * r.T * rs;  // 2 * wgt * dt/ddelta
    acc[0] = fmaf(q, fmaf(ua, cia, -vb * sib), acc[0]);
    acc[1] = fmaf(q, fmaf(ua, sia, vb * cib), acc[1]);
    acc[2] = fmaf(q * ua * vb, r.p1h / r.p0h - r.p0h / r.p1h, acc[2]);
    acc[3] = fmaf(q * ua * ua, r.p0h, acc[3]);
    acc[4] = fmaf(q * vb * vb, r.p1h, acc[4]);
}

template <template <int> class F, typename... Args>
cudaError_t dispatch_n(int n, Args &&...args) {
    switch (n) {
        case 32: return F<32>::run(args...);
        case 64: return F<64>::run(args...);
        case 128: return F<128>::run(args...);
        case 256: return F<256>::run(args...);
        case 512: return F<512>::run(args...);
        case 1024: return F<1024>::run(args...);
        case 2048: return F<2048>::run(args...);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace osog
