// Shared-memory Stockham FFT for sets of lines held by one CTA.
//
// A CTA owns L lines of N complex samples (N a power of two, 32..2048) in
// shared memory, line l at buf + l * line_stride(N), sample i at pad16(i).
// The transform runs as a few radix-P passes (P in {4, 8, 16}).  In each
// pass every thread loads whole butterflies into registers, the CTA
// synchronises, and the results are written back in Stockham (self-sorting)
// order, so no bit reversal is needed and a single buffer suffices.
//
// Stockham radix-P pass with sub-transform length Ns (product of the radices
// of the earlier passes), for butterfly j in [0, N/P), k = j mod Ns:
//     v_r = x[j + r N/P] * w^{r k},   w = exp(-+ 2 pi i / (Ns P))
//     V   = DFT_P(v)
//     x'[(j - k) P + k + r Ns] = V_r
// (the self-sorting formulation of Stockham's autosort FFT, e.g.
// Govindaraju et al., "High performance discrete Fourier transforms on
// graphics processors", SC 2008).  The twiddles w^{rk} come from per-pass
// tables laid out [r - 1][k] (so the lanes of a warp, which hold
// consecutive k, read consecutive entries) that the host builds in double
// precision and rounds to float once; the tables of all passes of an
// N-point transform fit in N entries.  Inverse transforms use the conjugate
// twiddles and are unnormalised.
#pragma once

#include <math.h>

#include "osog_common.cuh"

namespace osog {

// cos and sin of 2 pi m / 16, m = 0..15 (cos(pi/8) = sqrt(2 + sqrt 2) / 2,
// sin(pi/8) = sqrt(2 - sqrt 2) / 2, cos(pi/4) = sqrt(1/2)).
__host__ __device__ constexpr float quarter_cos16(int m) {  // m in 0..4
    return m == 0 ? 1.0f
         : m == 1 ? 0.92387953251128674f
         : m == 2 ? 0.70710678118654752f
         : m == 3 ? 0.38268343236508977f
         : 0.0f;
}
__host__ __device__ constexpr float cos16(int m) {
    m &= 15;
    return m <= 4 ? quarter_cos16(m)
         : m <= 8 ? -quarter_cos16(8 - m)
         : m <= 12 ? -quarter_cos16(m - 8)
         : quarter_cos16(16 - m);
}
__host__ __device__ constexpr float sin16(int m) { return cos16(m - 4); }

// x * exp(-+ 2 pi i K / P) with K, P compile-time (P divides 16).
template <int P, int K, bool INV>
__device__ __forceinline__ float2 twc(float2 x) {
    constexpr int m = (K * 16 / P) & 15;
    if constexpr (m == 0) {
        return x;
    } else if constexpr (m == 4) {
        return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    } else if constexpr (m == 8) {
        return make_float2(-x.x, -x.y);
    } else if constexpr (m == 12) {
        return INV ? make_float2(x.y, -x.x) : make_float2(-x.y, x.x);
    } else {
        constexpr float c = cos16(m);
        constexpr float s = INV ? sin16(m) : -sin16(m);
        return make_float2(fmaf(x.x, c, -__fmul_rn(x.y, s)), fmaf(x.x, s, __fmul_rn(x.y, c)));
    }
}

template <int P, bool INV, int K = 0>
__device__ __forceinline__ void twiddle_odds(float2 *o) {
    if constexpr (K < P / 2) {
        o[K] = twc<P, K, INV>(o[K]);
        twiddle_odds<P, INV, K + 1>(o);
    }
}

// In-register DFT of P points (radix-2 decimation in time, unrolled).
template <int P, bool INV>
__device__ __forceinline__ void dft(float2 *v) {
    if constexpr (P == 2) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else {
        float2 e[P / 2], o[P / 2];
#pragma unroll
        for (int k = 0; k < P / 2; ++k) {
            e[k] = v[2 * k];
            o[k] = v[2 * k + 1];
        }
        dft<P / 2, INV>(e);
        dft<P / 2, INV>(o);
        twiddle_odds<P, INV>(o);
#pragma unroll
        for (int k = 0; k < P / 2; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + P / 2] = csub(e[k], o[k]);
        }
    }
}

// Radix plans: 32 = 8.4, 64 = 8.8, 128 = 16.8, 256 = 16.16, 512 = 8.8.8,
// 1024 = 16.8.8, 2048 = 16.16.8.
__host__ __device__ constexpr int fft_passes(int n) { return n >= 512 ? 3 : 2; }
__host__ __device__ constexpr int fft_radix(int n, int p) {
    return n == 32 ? (p == 0 ? 8 : 4)
         : n == 64 ? 8
         : n == 128 ? (p == 0 ? 16 : 8)
         : n == 256 ? 16
         : n == 512 ? 8
         : n == 1024 ? (p == 0 ? 16 : 8)
         : (p < 2 ? 16 : 8);
}
__host__ __device__ constexpr int fft_ns(int n, int p) {  // sub-transform length before pass p
    return p == 0 ? 1 : fft_ns(n, p - 1) * fft_radix(n, p - 1);
}
__host__ __device__ constexpr int fft_twoff(int n, int p) {  // start of pass p's table
    return p == 0 ? 0
                  : fft_twoff(n, p - 1) +
                        (fft_ns(n, p - 1) > 1 ? (fft_radix(n, p - 1) - 1) * fft_ns(n, p - 1) : 0);
}

// pad16(base + r * stride) - pad16(base) for the bases the Stockham passes
// write from: with stride >= 16 (a power of two) the carry into the padding
// term is r * stride / 16; with stride 8 the base's low part k < 8 never
// carries, leaving r / 2; with stride 1 the base is a multiple of the radix
// P <= 16 and base % 16 + r < 16.  Every offset folds to a constant once the
// r loop is unrolled.
__device__ __forceinline__ constexpr int stride_off(int stride, int r) {
    return stride >= 16 ? r * (stride + stride / 16) : stride == 8 ? 8 * r + (r >> 1) : r;
}

// Synchronisation of the threads that own line l when each line of the set
// belongs to its own group of kThreads / L threads (a named barrier per
// line, or the warp when a line has one warp).
template <int L>
__device__ __forceinline__ void line_sync(int l) {
    constexpr int TPL = kThreads / L;
    if constexpr (TPL == 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + l), "r"(TPL) : "memory");
    }
}

// True when the passes of an N-point transform can run with one thread
// group per line: every pass has at least one butterfly per thread of the
// group (sets of 8192 samples, N >= 1024).
__host__ __device__ constexpr bool fft_grouped(int n) {
    return set_elems(n) == kMaxSetElems && n >= 1024;
}

// Butterfly q of this thread in a pass of NB butterflies per line over L
// lines: grouped, the threads [l TPL, (l + 1) TPL) take line l; otherwise
// consecutive threads take consecutive butterflies of the whole set.
template <int L, int NB, bool G>
__device__ __forceinline__ void butterfly_of(int q, int &l, int &j) {
    if constexpr (G) {
        constexpr int TPL = kThreads / L;
        l = threadIdx.x / TPL;
        j = threadIdx.x % TPL + q * TPL;
    } else {
        const int b = threadIdx.x + q * kThreads;
        l = b / NB;
        j = b % NB;
    }
}

// Largest radix whose twiddles are formed as products (0: all read from the
// table).  A radix-P pass needs w^{r k}, r = 1..P-1: the table entries at
// r = 1, 2, 4 (and 8) are read and the others formed as products of two of
// them, which takes those reads off the load path at the cost of a few
// fused multiply-adds and a rounding error of a few units in the last place.
constexpr int kTwiddleProducts = 16;

// v[r] *= w^{r k} (conjugated for the inverse transform), r = 1..P-1, with
// t the pass's table at entry [0][k] (entries [r - 1][k] at stride NS).
template <int P, bool INV, int NS>
__device__ __forceinline__ void apply_twiddles(float2 *v, const float2 *__restrict__ t) {
    auto mul = [](float2 a, float2 w) { return INV ? cmulc(a, w) : cmul(a, w); };
    if constexpr (P == 8 && kTwiddleProducts >= 8) {
        const float2 w1 = __ldg(t), w2 = __ldg(t + NS), w4 = __ldg(t + 3 * NS);
        const float2 w3 = cmul(w2, w1);
        v[1] = mul(v[1], w1);
        v[2] = mul(v[2], w2);
        v[3] = mul(v[3], w3);
        v[4] = mul(v[4], w4);
        v[5] = mul(v[5], cmul(w4, w1));
        v[6] = mul(v[6], cmul(w4, w2));
        v[7] = mul(v[7], cmul(w4, w3));
    } else if constexpr (P == 16 && kTwiddleProducts >= 16) {
        const float2 w1 = __ldg(t), w2 = __ldg(t + NS), w4 = __ldg(t + 3 * NS),
                     w8 = __ldg(t + 7 * NS);
        const float2 w3 = cmul(w2, w1), w5 = cmul(w4, w1), w6 = cmul(w4, w2), w7 = cmul(w4, w3);
        v[1] = mul(v[1], w1);
        v[2] = mul(v[2], w2);
        v[3] = mul(v[3], w3);
        v[4] = mul(v[4], w4);
        v[5] = mul(v[5], w5);
        v[6] = mul(v[6], w6);
        v[7] = mul(v[7], w7);
        v[8] = mul(v[8], w8);
        v[9] = mul(v[9], cmul(w8, w1));
        v[10] = mul(v[10], cmul(w8, w2));
        v[11] = mul(v[11], cmul(w8, w3));
        v[12] = mul(v[12], cmul(w8, w4));
        v[13] = mul(v[13], cmul(w8, w5));
        v[14] = mul(v[14], cmul(w8, w6));
        v[15] = mul(v[15], cmul(w8, w7));
    } else {
#pragma unroll
        for (int r = 1; r < P; ++r) v[r] = mul(v[r], __ldg(t + (r - 1) * NS));
    }
}

// One Stockham pass over L lines of N points.  G: one thread group per line
// (fft_grouped(N)); the pass then synchronises only the line's group.
template <int N, int L, int P, int NS, bool INV, bool G = false>
__device__ __forceinline__ void stockham_pass(float2 *buf, const float2 *__restrict__ tw) {
    static_assert(NS == 1 || NS == 8 || NS % 16 == 0, "unsupported Stockham stride");
    constexpr int NB = N / P;
    constexpr int TOT = L * NB;
    constexpr int PER = (TOT + kThreads - 1) / kThreads;
    constexpr int LS = line_stride(N);
    static_assert(!G || (NB % (kThreads / L) == 0 && kThreads % L == 0), "grouped pass");
    float2 v[PER][P];
    int l = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        int j;
        butterfly_of<L, NB, G>(q, l, j);
        if (G || TOT % kThreads == 0 || threadIdx.x + q * kThreads < TOT) {
            if constexpr (NB % 16 == 0) {
                const float2 *src = buf + l * LS + pad16(j);
#pragma unroll
                for (int r = 0; r < P; ++r) v[q][r] = src[r * (NB + NB / 16)];
            } else {
                const float2 *src = buf + l * LS;
#pragma unroll
                for (int r = 0; r < P; ++r) v[q][r] = src[pad16(j + r * NB)];
            }
        }
    }
    if constexpr (G) line_sync<L>(l); else __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        int j;
        butterfly_of<L, NB, G>(q, l, j);
        if (G || TOT % kThreads == 0 || threadIdx.x + q * kThreads < TOT) {
            const int k = j & (NS - 1);
            if constexpr (NS > 1) apply_twiddles<P, INV, NS>(v[q], tw + k);  // entries [r - 1][k]
            dft<P, INV>(v[q]);
            float2 *dst = buf + l * LS + pad16((j - k) * P + k);
#pragma unroll
            for (int r = 0; r < P; ++r) dst[stride_off(NS, r)] = v[q][r];
        }
    }
    if constexpr (G) line_sync<L>(l); else __syncthreads();
}

// Full FFT of the L lines (forward: exp(-2 pi i jk/N); inverse: conjugate,
// unnormalised), following the radix plan above.  tw is the N-point
// transform's table block.
template <int N, int L, bool INV, int PASS = 0>
__device__ __forceinline__ void fft_lines(float2 *buf, const float2 *__restrict__ tw) {
    if constexpr (PASS < fft_passes(N)) {
        stockham_pass<N, L, fft_radix(N, PASS), fft_ns(N, PASS), INV>(buf,
                                                                      tw + fft_twoff(N, PASS));
        fft_lines<N, L, INV, PASS + 1>(buf, tw);
    }
}

// Passes [PASS, END) of the radix plan, each an in-place Stockham pass
// (G: grouped, see stockham_pass).
template <int N, int L, bool INV, int PASS, int END, bool G = false>
__device__ __forceinline__ void fft_pass_range(float2 *buf, const float2 *__restrict__ tw) {
    if constexpr (PASS < END) {
        stockham_pass<N, L, fft_radix(N, PASS), fft_ns(N, PASS), INV, G>(buf,
                                                                         tw + fft_twoff(N, PASS));
        fft_pass_range<N, L, INV, PASS + 1, END, G>(buf, tw);
    }
}

// The first pass of the plan (stride 1, no twiddles) with its inputs taken
// from ld(l, i), sample i of line l, instead of from buf: the kernels fold
// the step that produces a line (a global load, the exit wave, a transfer
// function) into the pass.  The butterflies and the order of every
// operation are those of stockham_pass, so the results are bitwise the same.
// IN_PLACE: ld reads buf itself, and the threads synchronise between the
// loads and the writes.  G: grouped (see stockham_pass); ld(l, i) may then
// read only line l of buf.  Ends with a barrier (the line's, grouped).
template <int N, int L, bool INV, bool IN_PLACE, bool G, class Ld>
__device__ __forceinline__ void fft_first_pass(float2 *buf, Ld ld) {
    constexpr int P = fft_radix(N, 0);
    constexpr int NB = N / P;
    constexpr int TOT = L * NB;
    constexpr int PER = (TOT + kThreads - 1) / kThreads;
    constexpr int LS = line_stride(N);
    static_assert(!G || (NB % (kThreads / L) == 0 && kThreads % L == 0), "grouped pass");
    float2 v[PER][P];
    int l = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        int j;
        butterfly_of<L, NB, G>(q, l, j);
        if (G || TOT % kThreads == 0 || threadIdx.x + q * kThreads < TOT) {
#pragma unroll
            for (int r = 0; r < P; ++r) v[q][r] = ld(l, j + r * NB);
        }
    }
    if constexpr (IN_PLACE) {
        if constexpr (G) line_sync<L>(l); else __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        int j;
        butterfly_of<L, NB, G>(q, l, j);
        if (G || TOT % kThreads == 0 || threadIdx.x + q * kThreads < TOT) {
            dft<P, INV>(v[q]);
            float2 *dst = buf + l * LS + pad16(j * P);
#pragma unroll
            for (int r = 0; r < P; ++r) dst[r] = v[q][r];
        }
    }
    if constexpr (G) line_sync<L>(l); else __syncthreads();
}

// The last pass of the plan with its outputs handed to st(l, i, value),
// sample i of line l, instead of written back to buf (the kernels store
// straight to global memory).  Arithmetic as in stockham_pass.  LINE_FAST:
// consecutive threads take consecutive lines (the columns of a column
// block, interleaved in global memory; the pass before must end with a CTA
// barrier); G: grouped (see stockham_pass); else consecutive butterflies of
// the whole set.  buf is only read, so there is no barrier.
template <int N, int L, bool INV, bool LINE_FAST, bool G, class St>
__device__ __forceinline__ void fft_last_pass(const float2 *buf, const float2 *__restrict__ tw,
                                              St st) {
    constexpr int PASS = fft_passes(N) - 1;
    constexpr int P = fft_radix(N, PASS), NS = fft_ns(N, PASS);
    static_assert(NS * P == N && NS > 1, "the last pass of the plan");
    static_assert(!(LINE_FAST && G), "one thread mapping");
    constexpr int NB = N / P;
    constexpr int TOT = L * NB;
    constexpr int PER = (TOT + kThreads - 1) / kThreads;
    constexpr int LS = line_stride(N);
    const float2 *__restrict__ t = tw + fft_twoff(N, PASS);
    float2 v[PER][P];
    auto which = [](int q, int &l, int &j) {
        if constexpr (LINE_FAST) {
            const int b = threadIdx.x + q * kThreads;
            l = b % L;
            j = b / L;
        } else {
            butterfly_of<L, NB, G>(q, l, j);
        }
    };
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        int l, j;
        which(q, l, j);
        if (G || TOT % kThreads == 0 || threadIdx.x + q * kThreads < TOT) {
            if constexpr (NB % 16 == 0) {
                const float2 *src = buf + l * LS + pad16(j);
#pragma unroll
                for (int r = 0; r < P; ++r) v[q][r] = src[r * (NB + NB / 16)];
            } else {
                const float2 *src = buf + l * LS;
#pragma unroll
                for (int r = 0; r < P; ++r) v[q][r] = src[pad16(j + r * NB)];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        int l, j;
        which(q, l, j);
        if (G || TOT % kThreads == 0 || threadIdx.x + q * kThreads < TOT) {
            apply_twiddles<P, INV, NS>(v[q], t + j);
            dft<P, INV>(v[q]);
#pragma unroll
            for (int r = 0; r < P; ++r) st(l, j + r * NS, v[q][r]);
        }
    }
}

// Host: the twiddle tables of an n-point transform, n entries, in double
// precision rounded once to float: pass p's block holds
// exp(-2 pi i r k / (Ns P)) at [(r - 1) Ns + k], r = 1..P-1, k = 0..Ns-1.
__host__ inline void fill_twiddles(int n, float2 *out) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int i = 0; i < n; ++i) out[i] = make_float2(0.f, 0.f);
    for (int p = 0; p < fft_passes(n); ++p) {
        const int P = fft_radix(n, p), NS = fft_ns(n, p);
        if (NS == 1) continue;
        float2 *t = out + fft_twoff(n, p);
        for (int r = 1; r < P; ++r)
            for (int k = 0; k < NS; ++k) {
                const long m = (long)r * k % (long)(NS * P);
                const double ang = two_pi * (double)m / (double)(NS * P);
                t[(r - 1) * NS + k] = make_float2((float)cos(ang), (float)-sin(ang));
            }
    }
}

}  // namespace osog
