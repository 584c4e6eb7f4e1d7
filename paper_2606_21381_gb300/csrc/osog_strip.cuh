// Device pieces shared by the forward and adjoint render kernels: the
// ordered strip raster, the transfer functions of the optical head, and a
// dispatcher over the power-of-two transform sizes.
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

// Accumulate one particle's OPD / ATT over the pixels [xa, xb] x [ya, yb]
// of the strip buffer.  The warp's lanes cover the particle's rows (the
// next power of two of their count, at most 32) times 32 / that many
// consecutive columns, stepping across the columns.
//   ellipsoid: t = T sqrt(1 - rho^2), rho^2 = u'^2 + v'^2 with
//              u' = (c ex + s ey) / a, v' = (-s ex + c ey) / b, evaluated
//              in float32 and redone in float-float inside the rim band;
//   prism:     t = clamp(g min(hx - |u|, hy - |v|), 0, T), g = 2 s_b dx;
//   polyhedron (g < 0): t = z_hi - z_lo over the particle's pixel-affine
//              plane bounds coef[off .. off + m) (Eq. 1), 0 outside a wall.
__device__ __forceinline__ void raster_particle(float2 *buf, int LS, int y0, const PRec &r,
                                                const float4 *__restrict__ coef, int xa, int xb,
                                                int ya, int yb, int lane) {
    const int bh = yb - ya + 1;
    const int lyn = bh >= 32 ? 32 : (bh <= 1 ? 1 : 1 << (32 - __clz(bh - 1)));
    const int lxn = 32 / lyn;
    const int shx = ilog2(lxn);
    const int lx = lane & (lxn - 1), ly = lane >> shx;
    // Two pixels per lane and step (x and x + lxn): both chords first, then
    // both shared-memory updates, so that the loads of the pair overlap.
    // A pixel outside the footprint is skipped (t < 0).
    if (r.g < 0.f) {
        const float4 *pc = coef + __float_as_int(r.p0h);
        const int m = __float_as_int(r.p1h);
        for (int yy = ya + ly; yy <= yb; yy += lyn) {
            const float ey = ((float)yy + 0.5f) - r.cy;
            float2 *row = buf + (yy - y0) * LS;
            for (int xx = xa + lx; xx <= xb; xx += lxn) {
                const float ex = ((float)xx + 0.5f) - r.cx;
                float zlo = -INFINITY, zhi = INFINITY;
                bool inside = true;
                for (int i = 0; i < m; ++i) {
                    const float4 q = __ldg(pc + i);  // same address in every lane
                    const float z = fmaf(-q.y, ex, fmaf(-q.z, ey, q.x));
                    if (q.w > 0.f)
                        zhi = fminf(zhi, z);
                    else if (q.w < 0.f)
                        zlo = fmaxf(zlo, z);
                    else
                        inside = inside && z >= 0.f;
                }
                if (!inside || !(zhi > zlo)) continue;
                const float t = zhi - zlo;
                float2 acc = row[pad16(xx)];
                acc.x = fmaf(r.dn, t, acc.x);
                acc.y = fmaf(r.mu, t, acc.y);
                row[pad16(xx)] = acc;
            }
        }
    } else if (r.g > 0.f) {
        for (int yy = ya + ly; yy <= yb; yy += lyn) {
            const float ey = ((float)yy + 0.5f) - r.cy;
            const float s_ey = r.sh * ey, c_ey = r.ch * ey;
            float2 *row = buf + (yy - y0) * LS;
            auto chord = [&](int xx) {
                const float ex = ((float)xx + 0.5f) - r.cx;
                const float u = fmaf(r.ch, ex, s_ey);
                const float v = fmaf(-r.sh, ex, c_ey);
                const float d = fminf(r.p0h - fabsf(u), r.p1h - fabsf(v));
                return fminf(fmaxf(r.g * d, 0.f), r.T);
            };
            for (int xx = xa + lx; xx <= xb; xx += 2 * lxn) {
                const int x2 = xx + lxn;
                const float t1 = chord(xx);
                const float t2 = x2 <= xb ? chord(x2) : -1.f;
                float2 *p1 = row + pad16(xx), *p2 = row + pad16(x2);
                float2 a1 = *p1, a2;
                if (t2 >= 0.f) a2 = *p2;
                *p1 = make_float2(fmaf(r.dn, t1, a1.x), fmaf(r.mu, t1, a1.y));
                if (t2 >= 0.f) *p2 = make_float2(fmaf(r.dn, t2, a2.x), fmaf(r.mu, t2, a2.y));
            }
        }
    } else {
        const float cia = r.ch * r.p0h, sia = r.sh * r.p0h;
        const float cib = r.ch * r.p1h, sib = r.sh * r.p1h;
        for (int yy = ya + ly; yy <= yb; yy += lyn) {
            const float yc = (float)yy + 0.5f;
            const float ey = yc - r.cy;
            const float u0 = sia * ey, v0 = cib * ey;
            float2 *row = buf + (yy - y0) * LS;
            auto chord = [&](int xx) {
                const float xc = (float)xx + 0.5f;
                const float ex = xc - r.cx;
                const float ua = fmaf(cia, ex, u0);
                const float vb = fmaf(-sib, ex, v0);
                float delta = 1.f - fmaf(ua, ua, vb * vb);
                if (delta < kRimBand) {
                    if (delta <= -kRimBand) return -1.f;
                    delta = ellipse_delta_ff(r, xc, yc);
                    if (!(delta > 0.f)) return -1.f;
                }
                return r.T * delta * rsqrtf(delta);
            };
            for (int xx = xa + lx; xx <= xb; xx += 2 * lxn) {
                const int x2 = xx + lxn;
                const float t1 = chord(xx);
                const float t2 = x2 <= xb ? chord(x2) : -1.f;
                float2 *p1 = row + pad16(xx), *p2 = row + pad16(x2);
                float2 a1, a2;
                if (t1 >= 0.f) a1 = *p1;
                if (t2 >= 0.f) a2 = *p2;
                if (t1 >= 0.f) *p1 = make_float2(fmaf(r.dn, t1, a1.x), fmaf(r.mu, t1, a1.y));
                if (t2 >= 0.f) *p2 = make_float2(fmaf(r.dn, t2, a2.x), fmaf(r.mu, t2, a2.y));
            }
        }
    }
}

// OPD/ATT of the strip [y0, y0 + R) into buf, particles in list order.
// The band list is consumed kThreads entries at a time: every thread tests
// one entry against the strip's rows and the kept entries are compacted, in
// order, into shared memory together with their records (one parallel
// global load per round instead of one dependent load per particle).  Each
// warp then rasterises, in order, the staged particles that overlap its own
// N/16 columns (16 warps of the 512-thread CTA).
template <int N>
__device__ void raster_strip(const Geometry &geo, const Work &w, const SceneDev &sc, int s,
                             int y0, float2 *buf, PRec *srec, Rect *srect, int *wsum) {
    constexpr int LS = line_stride(N);
    constexpr int NW = kThreads / 32;
    const int band = y0 / geo.BH;
    const int32_t *off = w.band_off + (size_t)s * (geo.nbands + 1);
    const int hi = min(off[band + 1], sc.pair_cap);
    const int lo = min(off[band], hi);
    const int32_t *ids = w.pairs + sc.pair0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cw = N / NW;
    const int c0 = warp * cw, c1 = c0 + cw - 1;
    const int ylast = y0 + geo.R - 1;
    const unsigned lt = lanemask_lt();
    for (int base = lo; base < hi; base += kThreads) {
        const int i = base + threadIdx.x;
        int id = 0;
        Rect q = {1, 0, 1, 0};
        if (i < hi) {
            id = ids[i];
            q = w.rect[id];
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
            srec[slot] = w.rec[id];
        }
        __syncthreads();
        for (int i0 = 0; i0 < nl; i0 += 32) {
            const int k = i0 + lane;
            Rect r = {1, 0, 1, 0};
            if (k < nl) r = srect[k];
            unsigned mm = __ballot_sync(kFull, k < nl && r.x0 <= c1 && r.x1 >= c0);
            while (mm) {
                const int src = __ffs(mm) - 1;
                mm &= mm - 1;
                const Rect rq = srect[i0 + src];
                const PRec rec = srec[i0 + src];
                raster_particle(buf, LS, y0, rec, w.plane_coef, max((int)rq.x0, c0),
                                min((int)rq.x1, c1),
                                max((int)rq.y0, y0), min((int)rq.y1, ylast), lane);
                __syncwarp();
            }
        }
        __syncthreads();
    }
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
