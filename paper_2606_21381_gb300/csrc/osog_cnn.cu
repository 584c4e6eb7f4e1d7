// Convolutions of the learned warm start as implicit GEMMs on the tensor
// cores (BF16 operands, FP32 accumulation): on tcgen05 (TMEM accumulators,
// shared-memory descriptors, mbarrier completion) where it is faster --
// forward and data gradients, and filter gradients with at least 128
// output channels -- and on the warp-level MMA (mma.sync) otherwise; the
// warp-level path stays selectable for all three.
//
//   forward  Y[m = (n,p,q)][k]   = sum_{j = (r,s,c)} X(im2col)[m][j] W[k][j]
//   data     dX[m = (n,h,w)][c]  = sum_{j = (r,s,k)} dY(gathered)[m][j] Wt[c][j]
//   filter   dW[k][j = (r,s,c)]  = sum_{m = (n,p,q)} dY[m][k] X(im2col)[m][j]
//
// A CTA computes a 64 x 64 tile of the product from 32-wide slices of the
// reduction: both operands are gathered from NHWC tensors (8 channels per
// 16-byte vector, zero outside the image or for strides that skip a tap),
// staged in shared memory as [row][reduction] and fed to mma.m16n8k16
// through ldmatrix; four warps each own a 32 x 32 sub-tile.  The filter
// gradient splits its pixel reduction across CTAs and sums the partial tiles
// in a fixed order, so every result is bitwise reproducible.
#include <cuda_bf16.h>

#include "osog_cnn.h"

namespace osog {
namespace cnn {
namespace {

constexpr int BM = 64, BN = 64, BK = 32, LDS = BK + 8;  // smem row: 40 bf16 = 80 bytes
constexpr int NT = 128;
constexpr int kSplitPixels = 2048;  // pixels per CTA in the filter-gradient reduction

// kDgrad2: the data gradient of a stride-2 convolution for the input
// pixels of one parity class (h mod 2, w mod 2), reduced over the taps that
// reach them only (the other taps of that class are zero).
enum Pass { kFwd = 0, kDgrad = 1, kWgrad = 2, kDgrad2 = 3 };

struct Geo {
    int N, H, W, C, K, R, S, stride, pad, P, Q;
};

struct Args {
    Geo g;
    const __nv_bfloat16 *x;     // fwd: X, dgrad: dY, wgrad: dY
    const __nv_bfloat16 *w;     // fwd: W [K][RSC], dgrad: Wt [C][RSK], wgrad: X
    const float *bias;
    const __nv_bfloat16 *mask;  // dgrad: activation whose ReLU derivative applies
    __nv_bfloat16 *y;
    float *y32;
    float *part;                // wgrad partial tiles [splits][M][N]
    int relu;
    int M, Ncols, Kred;         // GEMM sizes
    // kDgrad2: parity class, its pixel grid and its taps
    int ph, pw, Hc, Wc, nr, ns;
    int rtap[4], stap[4];
};

__device__ __forceinline__ uint4 zero4() { return make_uint4(0u, 0u, 0u, 0u); }

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3,
                                        const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void ldsm_x4_t(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3,
                                          const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------- gathers
// Forward A: 8 reduction entries j..j+7 (same tap, 8 channels) of output
// pixel m.
__device__ __forceinline__ const __nv_bfloat16 *fwd_a_src(const Args &a, int m, int j) {
    const Geo &g = a.g;
    if (m >= a.M || j >= a.Kred) return nullptr;
    const int q = m % g.Q, t = m / g.Q, p = t % g.P, n = t / g.P;
    const int rs = j / g.C, c = j - rs * g.C, r = rs / g.S, s = rs - r * g.S;
    const int h = p * g.stride + r - g.pad, w = q * g.stride + s - g.pad;
    if (h < 0 || h >= g.H || w < 0 || w >= g.W) return nullptr;
    return a.x + (((size_t)n * g.H + h) * g.W + w) * g.C + c;
}
__device__ __forceinline__ uint4 fwd_a(const Args &a, int m, int j) {
    const __nv_bfloat16 *p = fwd_a_src(a, m, j);
    return p ? *reinterpret_cast<const uint4 *>(p) : zero4();
}

// Data-gradient A: dY at the output pixel that tap (r, s) of input pixel m
// reads, 8 output channels; zero where the stride skips it.
__device__ __forceinline__ const __nv_bfloat16 *dgrad_a_src(const Args &a, int m, int j) {
    const Geo &g = a.g;
    if (m >= a.M || j >= a.Kred) return nullptr;
    const int w = m % g.W, t = m / g.W, h = t % g.H, n = t / g.H;
    const int rs = j / g.K, k = j - rs * g.K, r = rs / g.S, s = rs - r * g.S;
    const int hp = h + g.pad - r, wq = w + g.pad - s;
    if (hp < 0 || wq < 0 || hp % g.stride || wq % g.stride) return nullptr;
    const int p = hp / g.stride, q = wq / g.stride;
    if (p >= g.P || q >= g.Q) return nullptr;
    return a.x + (((size_t)n * g.P + p) * g.Q + q) * g.K + k;
}
__device__ __forceinline__ uint4 dgrad_a(const Args &a, int m, int j) {
    const __nv_bfloat16 *p = dgrad_a_src(a, m, j);
    return p ? *reinterpret_cast<const uint4 *>(p) : zero4();
}

// Stride-2 data gradient, parity class (ph, pw): class pixel m = (n, i, j)
// is input pixel (n, 2 i + ph, 2 j + pw); reduction entry (tap, k) with tap
// = (ri, si) reads dY at ((h + pad - r) / 2, (w + pad - s) / 2), which the
// class's taps make exact.
__device__ __forceinline__ const __nv_bfloat16 *dgrad2_a_src(const Args &a, int m, int j) {
    const Geo &g = a.g;
    if (m >= a.M || j >= a.Kred) return nullptr;
    const int wi = m % a.Wc, t = m / a.Wc, hi = t % a.Hc, n = t / a.Hc;
    const int tap = j / g.K, k = j - tap * g.K, ri = tap / a.ns, si = tap - ri * a.ns;
    const int p = (2 * hi + a.ph + g.pad - a.rtap[ri]) >> 1;
    const int q = (2 * wi + a.pw + g.pad - a.stap[si]) >> 1;
    if (p < 0 || q < 0 || p >= g.P || q >= g.Q) return nullptr;
    return a.x + (((size_t)n * g.P + p) * g.Q + q) * g.K + k;
}
__device__ __forceinline__ uint4 dgrad2_a(const Args &a, int m, int j) {
    const __nv_bfloat16 *p = dgrad2_a_src(a, m, j);
    return p ? *reinterpret_cast<const uint4 *>(p) : zero4();
}

// Filters reordered [C][R][S][K], row c, reduction entry (tap, k) of the
// class's taps.
__device__ __forceinline__ const __nv_bfloat16 *dgrad2_b_src(const Args &a, int c, int j) {
    const Geo &g = a.g;
    if (c >= a.Ncols || j >= a.Kred) return nullptr;
    const int tap = j / g.K, k = j - tap * g.K, ri = tap / a.ns, si = tap - ri * a.ns;
    const int rs = a.rtap[ri] * g.S + a.stap[si];
    return a.w + ((size_t)c * g.R * g.S + rs) * g.K + k;
}
__device__ __forceinline__ uint4 dgrad2_b(const Args &a, int c, int j) {
    const __nv_bfloat16 *p = dgrad2_b_src(a, c, j);
    return p ? *reinterpret_cast<const uint4 *>(p) : zero4();
}

// Row-major operand rows (8 consecutive reduction entries of row r).
__device__ __forceinline__ const __nv_bfloat16 *rows_src(const __nv_bfloat16 *base, int rows, int ld,
                                                         int r, int j) {
    if (r >= rows || j >= ld) return nullptr;
    return base + (size_t)r * ld + j;
}
__device__ __forceinline__ uint4 rows_b(const __nv_bfloat16 *base, int rows, int ld, int r, int j) {
    const __nv_bfloat16 *p = rows_src(base, rows, ld, r, j);
    return p ? *reinterpret_cast<const uint4 *>(p) : zero4();
}

// Filter gradient: A(k, pixel) = dY[pixel][k..k+7] (a vector across 8 rows
// of the A tile); B(j, pixel) = X(im2col)[pixel][j..j+7] (across 8 rows of
// the B tile).
__device__ __forceinline__ uint4 wgrad_a(const Args &a, int k, int pix) {
    if (k >= a.M || pix >= a.Kred) return zero4();
    return *reinterpret_cast<const uint4 *>(a.x + (size_t)pix * a.g.K + k);
}
__device__ __forceinline__ uint4 wgrad_b(const Args &a, int j, int pix) {
    const Geo &g = a.g;
    if (j >= a.Ncols || pix >= a.Kred) return zero4();
    const int q = pix % g.Q, t = pix / g.Q, p = t % g.P, n = t / g.P;
    const int rs = j / g.C, c = j - rs * g.C, r = rs / g.S, s = rs - r * g.S;
    const int h = p * g.stride + r - g.pad, w = q * g.stride + s - g.pad;
    if (h < 0 || h >= g.H || w < 0 || w >= g.W) return zero4();
    return *reinterpret_cast<const uint4 *>(a.w + (((size_t)n * g.H + h) * g.W + w) * g.C + c);
}

// Output of two adjacent columns (col, col + 1) of GEMM row `row`.
template <int PASS>
__device__ __forceinline__ void epilogue_pair(const Args &a, int row, int col, float v0, float v1) {
    size_t o = (size_t)row * a.Ncols + col;
    if constexpr (PASS == kDgrad2) {  // class pixel -> input pixel
        const int wi = row % a.Wc, t = row / a.Wc, hi = t % a.Hc, n = t / a.Hc;
        o = (((size_t)n * a.g.H + 2 * hi + a.ph) * a.g.W + 2 * wi + a.pw) * a.Ncols + col;
    }
    if constexpr (PASS == kFwd) {
        v0 += a.bias[col];
        v1 += a.bias[col + 1];
        if (a.relu) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
        }
        *reinterpret_cast<__nv_bfloat162 *>(a.y + o) = __floats2bfloat162_rn(v0, v1);
        if (a.y32) *reinterpret_cast<float2 *>(a.y32 + o) = make_float2(v0, v1);
    } else if constexpr (PASS == kDgrad || PASS == kDgrad2) {
        if (a.mask) {
            const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(a.mask + o);
            if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
            if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
        }
        *reinterpret_cast<__nv_bfloat162 *>(a.y + o) = __floats2bfloat162_rn(v0, v1);
    } else {
        *reinterpret_cast<float2 *>(a.part + (size_t)blockIdx.z * a.M * a.Ncols + o) =
            make_float2(v0, v1);
    }
}

// Output of eight consecutive columns col .. col + 7 (col a multiple of 8)
// of GEMM row `row`, forward or data gradient, as 16-byte accesses.
template <int PASS>
__device__ __forceinline__ void epilogue_vec8(const Args &a, int row, int col, const float *v) {
    size_t o = (size_t)row * a.Ncols + col;
    if constexpr (PASS == kDgrad2) {
        const int wi = row % a.Wc, t = row / a.Wc, hi = t % a.Hc, n = t / a.Hc;
        o = (((size_t)n * a.g.H + 2 * hi + a.ph) * a.g.W + 2 * wi + a.pw) * a.Ncols + col;
    }
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = v[j];
    if constexpr (PASS == kFwd) {
        const float4 b0 = *reinterpret_cast<const float4 *>(a.bias + col);
        const float4 b1 = *reinterpret_cast<const float4 *>(a.bias + col + 4);
        const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            x[j] += bb[j];
            if (a.relu) x[j] = fmaxf(x[j], 0.f);
        }
        if (a.y32) {
            *reinterpret_cast<float4 *>(a.y32 + o) = make_float4(x[0], x[1], x[2], x[3]);
            *reinterpret_cast<float4 *>(a.y32 + o + 4) = make_float4(x[4], x[5], x[6], x[7]);
        }
    } else if (a.mask) {
        const uint4 mk = *reinterpret_cast<const uint4 *>(a.mask + o);
        const __nv_bfloat16 *m8 = reinterpret_cast<const __nv_bfloat16 *>(&mk);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (!(__bfloat162float(m8[j]) > 0.f)) x[j] = 0.f;
    }
    uint4 out;
    __nv_bfloat162 *o2 = reinterpret_cast<__nv_bfloat162 *>(&out);
#pragma unroll
    for (int j = 0; j < 4; ++j) o2[j] = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
    *reinterpret_cast<uint4 *>(a.y + o) = out;
}

// ---------------------------------------------------------------- GEMM
// The filter gradient reduces over pixels, the outer index of both NHWC
// operands: its tiles are kept as [pixel][row] (16-byte vector stores) and
// its fragments are read transposed (ldmatrix .trans).
constexpr int LDT = BM + 8;  // 72 bf16 = 144 bytes per pixel row

template <int PASS>
__global__ void __launch_bounds__(NT) k_conv_gemm(const __grid_constant__ Args a) {
    constexpr bool T = PASS == kWgrad;
    __shared__ __align__(16) __nv_bfloat16 smA[2 * (T ? BK * LDT : BM * LDS)];
    __shared__ __align__(16) __nv_bfloat16 smB[2 * (T ? BK * LDT : BN * LDS)];
    // element (row, k) of stage buf: [row][k] tiles, or [k][row] for T
    auto As = [&](int buf, int row, int k) -> __nv_bfloat16 * {
        return T ? smA + buf * BK * LDT + k * LDT + row : smA + buf * BM * LDS + row * LDS + k;
    };
    auto Bs = [&](int buf, int row, int k) -> __nv_bfloat16 * {
        return T ? smB + buf * BK * LDT + k * LDT + row : smB + buf * BN * LDS + row * LDS + k;
    };
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    int kbeg = 0, kend = a.Kred;
    if constexpr (PASS == kWgrad) {
        kbeg = blockIdx.z * kSplitPixels;
        kend = min(a.Kred, kbeg + kSplitPixels);
    }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = warp & 1, wn = warp >> 1;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
    uint4 ra[2], rb[2];

    auto load = [&](int k0) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int v = tid + i * NT;
            if constexpr (PASS == kWgrad) {
                const int kc = v & 31, rg = v >> 5;
                ra[i] = wgrad_a(a, m0 + rg * 8, k0 + kc);
                rb[i] = wgrad_b(a, n0 + rg * 8, k0 + kc);
            } else {
                const int row = v >> 2, kv = v & 3;
                if constexpr (PASS == kDgrad2) {
                    ra[i] = dgrad2_a(a, m0 + row, k0 + kv * 8);
                    rb[i] = dgrad2_b(a, n0 + row, k0 + kv * 8);
                } else {
                    ra[i] = PASS == kFwd ? fwd_a(a, m0 + row, k0 + kv * 8)
                                         : dgrad_a(a, m0 + row, k0 + kv * 8);
                    rb[i] = rows_b(a.w, a.Ncols, a.Kred, n0 + row, k0 + kv * 8);
                }
            }
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int v = tid + i * NT;
            if constexpr (PASS == kWgrad) {
                const int kc = v & 31, rg = v >> 5;
                *reinterpret_cast<uint4 *>(As(buf, rg * 8, kc)) = ra[i];
                *reinterpret_cast<uint4 *>(Bs(buf, rg * 8, kc)) = rb[i];
            } else {
                const int row = v >> 2, kv = v & 3;
                *reinterpret_cast<uint4 *>(As(buf, row, kv * 8)) = ra[i];
                *reinterpret_cast<uint4 *>(Bs(buf, row, kv * 8)) = rb[i];
            }
        }
    };

    load(kbeg);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        const bool more = k0 + BK < kend;
        if (more) load(k0 + BK);  // global loads in flight during the MMAs
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[2][4], bf[4][2];
            const int q = lane >> 3, r8 = lane & 7;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                if constexpr (T)  // 8x8 blocks (m 0-7 | 8-15) x (k 0-7 | 8-15), stored [k][m]
                    ldsm_x4_t(af[mt][0], af[mt][1], af[mt][2], af[mt][3],
                              As(buf, wm * 32 + mt * 16 + (q & 1) * 8, kk + r8 + (q >> 1) * 8));
                else
                    ldsm_x4(af[mt][0], af[mt][1], af[mt][2], af[mt][3],
                            As(buf, wm * 32 + mt * 16 + (lane & 15), kk + (lane >> 4) * 8));
            }
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                if constexpr (T)  // (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
                    ldsm_x4_t(bf[2 * np][0], bf[2 * np][1], bf[2 * np + 1][0], bf[2 * np + 1][1],
                              Bs(buf, wn * 32 + np * 16 + (q >> 1) * 8, kk + r8 + (q & 1) * 8));
                else
                    ldsm_x4(bf[2 * np][0], bf[2 * np][1], bf[2 * np + 1][0], bf[2 * np + 1][1],
                            Bs(buf, wn * 32 + np * 16 + (lane & 7) + (lane >> 4) * 8,
                               kk + ((lane >> 3) & 1) * 8));
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bf[nt][0], bf[nt][1]);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }

    // epilogue: thread holds rows (lane / 4) and (lane / 4 + 8) of each
    // 16 x 8 tile, columns 2 (lane % 4) and +1
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int row = m0 + wm * 32 + mt * 16 + (lane >> 2) + half * 8;
                const int col = n0 + wn * 32 + nt * 8 + (lane & 3) * 2;
                if (row >= a.M || col >= a.Ncols) continue;
                epilogue_pair<PASS>(a, row, col, acc[mt][nt][half * 2], acc[mt][nt][half * 2 + 1]);
            }
}

// ---------------------------------------------------------------- tcgen05
// Forward and data-gradient convolutions on the fifth-generation tensor
// cores.  A CTA of UNT threads owns a tile of UM = 128 GEMM rows (pixels) by
// BNU columns (output channels rounded up to 16, at most 128); the FP32
// accumulator lives in tensor memory (TMEM, one lane per row).  Each
// reduction slice of UBK = 64 is copied by all threads (cp.async, 16 bytes,
// zero-filled outside the image) into one of UST shared stages in the
// canonical K-major layout without swizzle -- 8-row x 16-byte
// core matrices, contiguous along K (LBO = 128 bytes) and 8-row groups
// UBK / 8 core matrices apart (SBO = 1024 bytes) -- then one thread issues
// four tcgen05.mma (M 128, N BNU, K 16) with shared-memory descriptors and
// commits them to the stage's mbarrier; a stage is refilled once its
// multiplications are done, while the next stage's are already queued, so
// copies of UST - 1 stages overlap the multiplications.  Waits are bounded: a timeout latches
// g_cnn_status and the kernel still releases its tensor memory.
constexpr int UM = 128, UBK = 64, UST = 3, UKC = UBK / 8, UNT = 256;
constexpr int kUStage = UM * UBK * 2;   // bytes of one operand stage (B <= 128 rows)
constexpr int kSpinLimit = 1 << 22;

__device__ int g_cnn_status;
// Failure-detection test (osog_conv_test_wait_limit): when positive, every
// tcgen05 convolution CTA also waits, for this many polls, on a barrier that
// nothing arrives on, so the bounded wait runs out and latches g_cnn_status.
__device__ int g_cnn_probe_polls;

__device__ __forceinline__ int canon(int row, int k) {  // byte offset in a stage
    return (row >> 3) * (UKC * 128) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)((UKC * 128) >> 4) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: FP32 D, BF16 A and B, both K-major,
// N >> 3 and M >> 4.
__device__ __forceinline__ uint32_t umma_idesc(int n, bool mn_major = false) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (mn_major ? (1u << 15) | (1u << 16) : 0u) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);
}

// MN-major canonical layout (both operands of the filter gradient): core
// matrices of 8 reduction rows x 16 bytes (8 consecutive MN elements),
// contiguous along the reduction (LBO 128 bytes), 8-element MN groups
// UKC core matrices apart (SBO 1024 bytes) -- the same strides as the
// K-major tiles, with the transpose bits of the instruction descriptor set.
__device__ __forceinline__ int canon_mn(int mn, int k) {
    return (mn >> 3) * (UKC * 128) + (k >> 3) * 128 + (k & 7) * 16 + (mn & 7) * 2;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit = kSpinLimit) {
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        __nanosleep(32);
    }
    return false;
}

// 16-byte asynchronous copy to shared memory; a NULL source writes zeros.
__device__ __forceinline__ void cp16(void *dst, const __nv_bfloat16 *src, const void *any) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n"
                 :: "r"(smem_u32(dst)), "l"(src ? (const void *)src : any), "r"(src ? 16 : 0)
                 : "memory");
}

// The operand copies of one thread.  Thread t copies the 8-element column
// kv = t % 8 of every slice for the A rows t / 8 + 32 i (i < 4) and the B
// rows t / 8 + 32 i below BNU.  The pixel of each A row is decoded once; the
// tap and channel of the reduction entry j = k0 + 8 kv advance by UBK per
// slice without divisions.
template <int PASS>
struct UGather {
    int kv;
    int n[UM * UKC / UNT], y[UM * UKC / UNT], x[UM * UKC / UNT];  // n < 0: row past M
    int t0, t1, ch;  // (r, s, c) forward, (r, s, k) data gradient, (ri, si, k) stride-2 class

    __device__ __forceinline__ void init(const Args &a, int m0, int tid) {
        const Geo &g = a.g;
        kv = tid & 7;
        const int cch = PASS == kFwd ? g.C : g.K, t1n = PASS == kDgrad2 ? a.ns : g.S;
        const int j = kv * 8, tap = j / cch;
        ch = j - tap * cch;
        if (t1n > 0) {
            t0 = tap / t1n;
            t1 = tap - t0 * t1n;
        } else {  // a parity class without taps: nothing to copy
            t0 = 1 << 20;
            t1 = 0;
        }
#pragma unroll
        for (int i = 0; i < UM * UKC / UNT; ++i) {
            const int m = m0 + (tid >> 3) + 32 * i;
            n[i] = -1;
            if (m >= a.M) continue;
            if constexpr (PASS == kFwd) {
                const int q = m % g.Q, t = m / g.Q, p = t % g.P;
                n[i] = t / g.P;
                y[i] = p * g.stride - g.pad;
                x[i] = q * g.stride - g.pad;
            } else if constexpr (PASS == kDgrad) {  // stride 1
                const int w = m % g.W, t = m / g.W, h = t % g.H;
                n[i] = t / g.H;
                y[i] = h + g.pad;
                x[i] = w + g.pad;
            } else {
                const int wi = m % a.Wc, t = m / a.Wc, hi = t % a.Hc;
                n[i] = t / a.Hc;
                y[i] = 2 * hi + a.ph + g.pad;
                x[i] = 2 * wi + a.pw + g.pad;
            }
        }
    }

    __device__ __forceinline__ void advance(const Args &a) {
        const int cch = PASS == kFwd ? a.g.C : a.g.K, t1n = PASS == kDgrad2 ? a.ns : a.g.S;
        ch += UBK;
        while (ch >= cch) {
            ch -= cch;
            if (++t1 == t1n) {
                t1 = 0;
                ++t0;
            }
        }
    }

    __device__ __forceinline__ void load(const Args &a, unsigned char *A, unsigned char *B, int n0,
                                         int k0, int BNU, int tid) const {
        const Geo &g = a.g;
        const bool live = t0 < (PASS == kDgrad2 ? a.nr : g.R);  // j < Kred
        const int r = PASS == kDgrad2 ? a.rtap[live ? t0 : 0] : t0;
        const int sx = PASS == kDgrad2 ? a.stap[t1] : t1;
#pragma unroll
        for (int i = 0; i < UM * UKC / UNT; ++i) {
            const int row = (tid >> 3) + 32 * i;
            const __nv_bfloat16 *src = nullptr;
            if (live && n[i] >= 0) {
                if constexpr (PASS == kFwd) {
                    const int h = y[i] + r, w = x[i] + sx;
                    if (h >= 0 && h < g.H && w >= 0 && w < g.W)
                        src = a.x + (((size_t)n[i] * g.H + h) * g.W + w) * g.C + ch;
                } else {
                    const int p = PASS == kDgrad ? y[i] - r : (y[i] - r) >> 1;
                    const int q = PASS == kDgrad ? x[i] - sx : (x[i] - sx) >> 1;
                    if (p >= 0 && p < g.P && q >= 0 && q < g.Q)
                        src = a.x + (((size_t)n[i] * g.P + p) * g.Q + q) * g.K + ch;
                }
            }
            cp16(A + canon(row, kv * 8), src, a.x);
        }
        for (int row = tid >> 3; row < BNU; row += UNT / 8) {
            const int b = n0 + row;
            const __nv_bfloat16 *src = nullptr;
            if (live && b < a.Ncols) {
                if constexpr (PASS == kDgrad2)
                    src = a.w + (((size_t)b * g.R + r) * g.S + sx) * g.K + ch;
                else
                    src = a.w + (size_t)b * a.Kred + k0 + kv * 8;
            }
            cp16(B + canon(row, kv * 8), src, a.w);
        }
    }
};

template <int PASS>
__global__ void __launch_bounds__(UNT) k_conv_umma(const __grid_constant__ Args a, int BNU) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int bstage = BNU * UBK * 2;  // bytes of one B stage
    unsigned char *stA = sm, *stB = sm + UST * kUStage;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(stB + UST * bstage);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + UST);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * UM, n0 = blockIdx.y * BNU;
    const uint32_t ncols = BNU <= 32 ? 32u : BNU <= 64 ? 64u : 128u;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     :: "r"(smem_u32(tslot)), "r"(ncols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int st = 0; st < UST; ++st)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(smem_u32(mbar + st)), "r"(1));
        // the failure-detection probe's barrier (after tslot): nothing arrives on it
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(smem_u32(mbar + UST + 1)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    const int nk = (a.Kred + UBK - 1) / UBK;
    UGather<PASS> ga;
    ga.init(a, m0, tid);
    // prologue: stages 0 .. UST-2 in flight, one commit group each
    for (int kt = 0; kt < UST - 1; ++kt) {
        if (kt < nk) {
            ga.load(a, stA + kt * kUStage, stB + kt * bstage, n0, kt * UBK, BNU, tid);
            ga.advance(a);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t taddr = *tslot;
    const uint32_t idesc = umma_idesc(BNU);
    bool ok = true;
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt % UST;
        // this thread's copies of stage kt have landed (UST-2 newer groups may pend)
        asm volatile("cp.async.wait_group %0;\n" :: "n"(UST - 2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            unsigned char *A = stA + st * kUStage, *B = stB + st * bstage;
#pragma unroll
            for (int s = 0; s < UBK / 16; ++s) {
                const uint64_t ad = umma_desc(smem_u32(A) + s * 256);
                const uint64_t bd = umma_desc(smem_u32(B) + s * 256);
                const uint32_t acc = (kt > 0 || s > 0) ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             :: "r"(taddr), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                         :: "r"(smem_u32(mbar + st)) : "memory");
        }
        // refill the stage of step kt-1 with step kt+UST-1 once its
        // multiplications are done (those of step kt are queued behind them)
        const int nx = kt + UST - 1;
        if (nx < nk) {
            const int sx = nx % UST;
            if (kt >= 1) ok = mbar_wait(smem_u32(mbar + sx), (uint32_t)(((kt - 1) / UST) & 1)) && ok;
            ga.load(a, stA + sx * kUStage, stB + sx * bstage, n0, nx * UBK, BNU, tid);
            ga.advance(a);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    // the last commit covers every multiplication issued before it (a
    // reduction of length 0 issues none: the result is zero)
    if (nk > 0) {
        const int last = nk - 1;
        ok = mbar_wait(smem_u32(mbar + last % UST), (uint32_t)((last / UST) & 1)) && ok;
    }
    if (tid == 0 && g_cnn_probe_polls > 0)  // a wait made to run out (test hook)
        ok = mbar_wait(smem_u32(mbar + UST + 1), 0u, g_cnn_probe_polls) && ok;
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (!ok && lane == 0) atomicExch(&g_cnn_status, 1);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows) and the
    // 32-column chunks c with c % (UNT / 128) == w / 4
    const int quarter = warp & 3, group = warp >> 2;
    const int row = m0 + quarter * 32 + lane;
    for (int c0 = group * 32; c0 < BNU; c0 += 32 * (UNT / 128)) {
        uint32_t v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
              "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
              "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
              "=r"(v[31])
            : "r"(taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (nk == 0) {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = 0u;
        }
        if (row < a.M) {
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
                const int col = n0 + c0 + j;
                if (c0 + j < BNU && col < a.Ncols) {
                    float f[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) f[i] = __uint_as_float(v[j + i]);
                    epilogue_vec8<PASS>(a, row, col, f);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(taddr), "r"(ncols)
                     : "memory");
}

// Filter gradient on tcgen05: dW[k][j] = sum over pixels of dY[pixel][k]
// X(im2col)[pixel][j] with the output channels k as the 128 GEMM rows
// (zero past K), the filter entries j = (r, s, c) as up to 128 columns and
// the pixels as the reduction, in chunks of kSplitPixels per CTA (grid.z)
// whose partial tiles are summed in chunk order.  Both operands are copied
// from NHWC rows as 16-byte vectors (8 channels of one pixel) into the
// MN-major layout.  SWAP (fewer than 128 output channels): the roles are
// exchanged, the filter entries are the 128 rows and the output channels
// the BNU columns (K rounded up to 16), so that few output channels do not
// pad the rows; the partial tiles are written in the same [k][j] layout.
template <bool SWAP>
__global__ void __launch_bounds__(UNT) k_wgrad_umma(const __grid_constant__ Args a, int BNU) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int bstage = BNU * UBK * 2;
    unsigned char *stA = sm, *stB = sm + UST * kUStage;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(stB + UST * bstage);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + UST);
    const Geo &g = a.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * UM, n0 = blockIdx.y * BNU;
    const int pbeg = blockIdx.z * kSplitPixels;
    const int pend = min(a.Kred, pbeg + kSplitPixels);
    const uint32_t ncols = BNU <= 32 ? 32u : BNU <= 64 ? 64u : 128u;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     :: "r"(smem_u32(tslot)), "r"(ncols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int st = 0; st < UST; ++st)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(smem_u32(mbar + st)), "r"(1));
        // the failure-detection probe's barrier (after tslot): nothing arrives on it
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(smem_u32(mbar + UST + 1)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    const int nk = (pend - pbeg + UBK - 1) / UBK;
    // Copies of slice kt.  Thread t owns channel group t % 16 of the 128
    // rows (A: 8 output channels) and of the 128 columns (B: 8 channels of
    // one tap, decoded once) and the pixels t / 16 + 16 i (i < 4) of every
    // slice, whose coordinates advance by UBK per slice without divisions;
    // consecutive threads read consecutive channel groups of one pixel.
    constexpr int NV = UBK * 16 / UNT;  // pixels per thread and slice
    const int grp = tid & 15, kq = tid >> 4;
    // m: this thread's 8 output channels (of dY); j: its 8 filter entries
    // (one tap of X); the row group is A's, the column group B's
    const int m = SWAP ? n0 + grp * 8 : m0 + grp * 8;
    const int j = SWAP ? m0 + grp * 8 : n0 + grp * 8;
    const bool jok = j < a.Ncols;
    const bool bcol = !SWAP || grp * 8 < BNU;  // B columns past BNU are not in the stage
    int tr = 0, ts = 0, tc = 0;
    if (jok) {
        const int rs = j / g.C;
        tc = j - rs * g.C;
        tr = rs / g.S;
        ts = rs - tr * g.S;
    }
    int pn[NV], pp[NV], pq[NV];  // image, output row, output column of each pixel
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const int pix = pbeg + kq + 16 * i;
        pq[i] = pix % g.Q;
        const int t = pix / g.Q;
        pp[i] = t % g.P;
        pn[i] = t / g.P;
    }
    auto load = [&](int kt, int st) {
        unsigned char *A = stA + st * kUStage, *B = stB + st * bstage;
        const int p0 = pbeg + kt * UBK;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const int k = kq + 16 * i, pix = p0 + k;
            const bool live = pix < pend;
            const __nv_bfloat16 *sy = live && m < a.M ? a.x + (size_t)pix * g.K + m : nullptr;
            const __nv_bfloat16 *sx = nullptr;
            if (live && jok) {
                const int h = pp[i] * g.stride + tr - g.pad, w = pq[i] * g.stride + ts - g.pad;
                if (h >= 0 && h < g.H && w >= 0 && w < g.W)
                    sx = a.w + (((size_t)pn[i] * g.H + h) * g.W + w) * g.C + tc;
            }
            cp16(A + canon_mn(grp * 8, k), SWAP ? sx : sy, a.x);
            if (bcol) cp16(B + canon_mn(grp * 8, k), SWAP ? sy : sx, a.w);
            // next slice: UBK pixels further
            pq[i] += UBK;
            while (pq[i] >= g.Q) {
                pq[i] -= g.Q;
                if (++pp[i] == g.P) {
                    pp[i] = 0;
                    ++pn[i];
                }
            }
        }
    };
    for (int kt = 0; kt < UST - 1; ++kt) {
        if (kt < nk) load(kt, kt);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t taddr = *tslot;
    const uint32_t idesc = umma_idesc(BNU, true);
    bool ok = true;
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt % UST;
        asm volatile("cp.async.wait_group %0;\n" :: "n"(UST - 2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            unsigned char *A = stA + st * kUStage, *B = stB + st * bstage;
#pragma unroll
            for (int s = 0; s < UBK / 16; ++s) {
                const uint64_t ad = umma_desc(smem_u32(A) + s * 256);
                const uint64_t bd = umma_desc(smem_u32(B) + s * 256);
                const uint32_t acc = (kt > 0 || s > 0) ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             :: "r"(taddr), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                         :: "r"(smem_u32(mbar + st)) : "memory");
        }
        const int nx = kt + UST - 1;
        if (nx < nk) {
            const int sx = nx % UST;
            if (kt >= 1) ok = mbar_wait(smem_u32(mbar + sx), (uint32_t)(((kt - 1) / UST) & 1)) && ok;
            load(nx, sx);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    if (nk > 0) {
        const int last = nk - 1;
        ok = mbar_wait(smem_u32(mbar + last % UST), (uint32_t)((last / UST) & 1)) && ok;
    }
    if (tid == 0 && g_cnn_probe_polls > 0)  // a wait made to run out (test hook)
        ok = mbar_wait(smem_u32(mbar + UST + 1), 0u, g_cnn_probe_polls) && ok;
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (!ok && lane == 0) atomicExch(&g_cnn_status, 1);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const int quarter = warp & 3, group = warp >> 2;
    const int row = m0 + quarter * 32 + lane;  // output channel (SWAP: filter entry)
    float *part = a.part + (size_t)blockIdx.z * a.M * a.Ncols;
    for (int c0 = group * 32; c0 < BNU; c0 += 32 * (UNT / 128)) {
        uint32_t v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
              "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
              "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
              "=r"(v[31])
            : "r"(taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if constexpr (SWAP) {  // lanes hold consecutive filter entries: coalesced per column
            if (row < a.Ncols) {
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    const int k = n0 + c0 + jj;
                    if (c0 + jj < BNU && k < a.M)
                        part[(size_t)k * a.Ncols + row] = nk ? __uint_as_float(v[jj]) : 0.f;
                }
            }
        } else if (row < a.M) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                const int col = n0 + c0 + j;
                if (c0 + j < BNU && col < a.Ncols) {  // Ncols is a multiple of 8
                    const float f0 = nk ? __uint_as_float(v[j]) : 0.f;
                    const float f1 = nk ? __uint_as_float(v[j + 1]) : 0.f;
                    const float f2 = nk ? __uint_as_float(v[j + 2]) : 0.f;
                    const float f3 = nk ? __uint_as_float(v[j + 3]) : 0.f;
                    *reinterpret_cast<float4 *>(part + (size_t)row * a.Ncols + col) =
                        make_float4(f0, f1, f2, f3);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(taddr), "r"(ncols)
                     : "memory");
}

constexpr int kUmmaSmem = 2 * UST * kUStage + 64;  // the largest (BNU = 128)
__host__ __device__ constexpr int umma_smem(int bnu) { return UST * (kUStage + bnu * UBK * 2) + 64; }

// One-time opt-in to the stages' dynamic shared memory.
cudaError_t umma_prepare() {
    static const cudaError_t e = [] {
        cudaError_t r = cudaFuncSetAttribute(k_conv_umma<kFwd>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kUmmaSmem);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_conv_umma<kDgrad>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kUmmaSmem);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_conv_umma<kDgrad2>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kUmmaSmem);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_wgrad_umma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kUmmaSmem);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_wgrad_umma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kUmmaSmem);
        return r;
    }();
    return e;
}

template <int PASS>
cudaError_t launch_umma(const Args &a, cudaStream_t st) {
    cudaError_t e = umma_prepare();
    if (e != cudaSuccess) return e;
    const int bnu = ((a.Ncols + 15) / 16) * 16 < 128 ? ((a.Ncols + 15) / 16) * 16 : 128;
    dim3 grid((a.M + UM - 1) / UM, (a.Ncols + bnu - 1) / bnu);
    k_conv_umma<PASS><<<grid, UNT, umma_smem(bnu), st>>>(a, bnu);
    return cudaGetLastError();
}

// Sum of the filter-gradient partial tiles over the pixel splits, in split
// order.
// out[i] = sum over z of part[z][i] for i < count, in a fixed order: a CTA
// takes 32 consecutive outputs (one per lane); warp w adds the splits z = w,
// w + kSumWarps, ... in ascending order (four loads in flight per lane), and
// warp 0 adds the warps' sums in warp order.  Coalesced 128-byte loads and
// count / 32 CTAs, where one thread per output walked every split alone.
constexpr int kSumWarps = 16;

__global__ void __launch_bounds__(32 * kSumWarps)
k_sum_splits(const float *part, int splits, int64_t count, float *out) {
    __shared__ float red[kSumWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 32 + lane;
    float s = 0.f;
    if (i < count) {
        int z = warp;
        for (; z + 3 * kSumWarps < splits; z += 4 * kSumWarps) {
            const float a0 = part[(int64_t)z * count + i];
            const float a1 = part[(int64_t)(z + kSumWarps) * count + i];
            const float a2 = part[(int64_t)(z + 2 * kSumWarps) * count + i];
            const float a3 = part[(int64_t)(z + 3 * kSumWarps) * count + i];
            s += a0;
            s += a1;
            s += a2;
            s += a3;
        }
        for (; z < splits; z += kSumWarps) s += part[(int64_t)z * count + i];
    }
    red[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && i < count) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < kSumWarps; ++w) t += red[w][lane];
        out[i] = t;
    }
}

// Launch of k_sum_splits over count outputs.
static void sum_splits(const float *part, int splits, int64_t count, float *out, cudaStream_t st) {
    if (count > 0)
        k_sum_splits<<<(unsigned)((count + 31) / 32), 32 * kSumWarps, 0, st>>>(part, splits, count, out);
}

// Partial bias gradients for K dividing 256: CTA c sums the pixels
// [c chunk, (c + 1) chunk), chunk = kBiasIter 256 / K, with 256 / K pixel
// lanes per channel (coalesced rows), then a fixed tree over the lanes:
// part[c][k].
constexpr int kBiasIter = 64;
__host__ __device__ constexpr int bias_chunk(int K) { return kBiasIter * (256 / K); }
__global__ void k_bias_partial(const __nv_bfloat16 *dy, int64_t pixels, int K, float *part) {
    __shared__ float red[256];
    const int lanes = 256 / K, t = threadIdx.x, k = t % K, pl = t / K;
    const int64_t p0 = (int64_t)blockIdx.x * bias_chunk(K);
    const int64_t p1 = p0 + bias_chunk(K) < pixels ? p0 + bias_chunk(K) : pixels;
    float acc = 0.f;
    for (int64_t p = p0 + pl; p < p1; p += lanes) acc += __bfloat162float(dy[p * K + k]);
    red[t] = acc;
    __syncthreads();
    for (int d = lanes / 2; d > 0; d >>= 1) {
        if (pl < d) red[t] += red[t + d * K];
        __syncthreads();
    }
    if (pl == 0) part[(int64_t)blockIdx.x * K + k] = red[t];
}

// dbias[k] = sum over pixels of dy[pixel][k] for other K: one CTA per
// channel, a fixed strided partition and a fixed tree.
__global__ void k_bias_grad(const __nv_bfloat16 *dy, int64_t pixels, int K, float *db) {
    __shared__ float red[256];
    const int k = blockIdx.x;
    float s = 0.f;
    for (int64_t p = threadIdx.x; p < pixels; p += blockDim.x) s += __bfloat162float(dy[p * K + k]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int d = blockDim.x / 2; d > 0; d >>= 1) {
        if (threadIdx.x < d) red[threadIdx.x] += red[threadIdx.x + d];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[k] = red[0];
}

// W [K][R][S][C] -> Wt [C][R][S][K].
__global__ void k_filter_transpose(const __nv_bfloat16 *w, int K, int RS, int C, __nv_bfloat16 *wt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)K * RS * C;
    if (i >= total) return;
    const int c = i % C;
    const int64_t t = i / C;
    const int rs = t % RS, k = t / RS;
    wt[((int64_t)c * RS + rs) * K + k] = w[i];
}

__global__ void k_relu_backward(const __nv_bfloat16 *dy, const __nv_bfloat16 *act, int64_t n,
                                __nv_bfloat16 *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __bfloat162float(act[i]) > 0.f ? dy[i] : __float2bfloat16(0.f);
}

}  // namespace
}  // namespace cnn
}  // namespace osog

using namespace osog::cnn;

namespace {

bool shape_ok(const osog_conv_shape_t *s) {
    return s && s->N > 0 && s->H > 0 && s->W > 0 && s->C > 0 && s->C % 8 == 0 && s->K > 0 &&
           s->K % 8 == 0 && s->R > 0 && s->S > 0 && s->R <= 8 && s->S <= 8 &&
           (s->stride == 1 || s->stride == 2) &&
           s->pad >= 0 && s->H + 2 * s->pad >= s->R && s->W + 2 * s->pad >= s->S;
}

Geo geo_of(const osog_conv_shape_t *s) {
    Geo g;
    g.N = s->N;
    g.H = s->H;
    g.W = s->W;
    g.C = s->C;
    g.K = s->K;
    g.R = s->R;
    g.S = s->S;
    g.stride = s->stride;
    g.pad = s->pad;
    g.P = (s->H + 2 * s->pad - s->R) / s->stride + 1;
    g.Q = (s->W + 2 * s->pad - s->S) / s->stride + 1;
    return g;
}

int splits_of(const Geo &g) {
    const int64_t pix = (int64_t)g.N * g.P * g.Q;
    return (int)((pix + kSplitPixels - 1) / kSplitPixels);
}

int status_of(cudaError_t e) { return e == cudaSuccess ? OSOG_OK : OSOG_ERR_CUDA; }

// Engine of the forward and data-gradient convolutions: the tcgen05 kernel
// (1, default) or the warp-level MMA kernel (0).
int g_use_tcgen05 = 1;
// Filter gradients with fewer than 128 output channels on tcgen05 with the
// roles exchanged (k_wgrad_umma<true>); 0 keeps them on the warp-level MMA.
int g_wgrad_swap = 1;

const __nv_bfloat16 *bf(const uint16_t *p) { return reinterpret_cast<const __nv_bfloat16 *>(p); }
__nv_bfloat16 *bf(uint16_t *p) { return reinterpret_cast<__nv_bfloat16 *>(p); }

}  // namespace

extern "C" {

int32_t osog_conv_out_h(const osog_conv_shape_t *s) { return shape_ok(s) ? geo_of(s).P : 0; }
int32_t osog_conv_out_w(const osog_conv_shape_t *s) { return shape_ok(s) ? geo_of(s).Q : 0; }

int osog_conv2d_forward(const osog_conv_shape_t *shape, const uint16_t *x, const uint16_t *w,
                        const float *bias, int32_t relu, uint16_t *y, float *y_f32,
                        osog_stream_t stream) {
    if (!shape_ok(shape) || !x || !w || !bias || !y) return OSOG_ERR_INVALID_ARG;
    Args a{};
    a.g = geo_of(shape);
    a.x = bf(x);
    a.w = bf(w);
    a.bias = bias;
    a.y = bf(y);
    a.y32 = y_f32;
    a.relu = relu;
    a.M = a.g.N * a.g.P * a.g.Q;
    a.Ncols = a.g.K;
    a.Kred = a.g.R * a.g.S * a.g.C;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // reductions shorter than two slices feed the tensor cores too little per
    // copied row (measured: the 8-channel first layer is faster on mma.sync)
    if (g_use_tcgen05 && a.Kred >= 2 * UBK) return status_of(launch_umma<kFwd>(a, st));
    dim3 grid((a.M + BM - 1) / BM, (a.Ncols + BN - 1) / BN);
    k_conv_gemm<kFwd><<<grid, NT, 0, st>>>(a);
    return status_of(cudaGetLastError());
}

int osog_conv2d_backward_data(const osog_conv_shape_t *shape, const uint16_t *dy,
                              const uint16_t *w, const uint16_t *x_act, uint16_t *dx,
                              uint16_t *w_t, osog_stream_t stream) {
    if (!shape_ok(shape) || !dy || !w || !dx || !w_t) return OSOG_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const Geo g = geo_of(shape);
    const int64_t nw = (int64_t)g.K * g.R * g.S * g.C;
    k_filter_transpose<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(bf(w), g.K, g.R * g.S, g.C, bf(w_t));
    Args a{};
    a.g = g;
    a.x = bf(dy);
    a.w = bf(w_t);
    a.mask = x_act ? bf(x_act) : nullptr;
    a.y = bf(dx);
    a.Ncols = g.C;
    if (g.stride == 2) {  // four parity classes, each over its own taps
        for (int ph = 0; ph < 2; ++ph)
            for (int pw = 0; pw < 2; ++pw) {
                a.ph = ph;
                a.pw = pw;
                a.Hc = (g.H - ph + 1) / 2;
                a.Wc = (g.W - pw + 1) / 2;
                a.nr = a.ns = 0;
                for (int r = 0; r < g.R; ++r)
                    if (((ph + g.pad - r) & 1) == 0) a.rtap[a.nr++] = r;
                for (int sx = 0; sx < g.S; ++sx)
                    if (((pw + g.pad - sx) & 1) == 0) a.stap[a.ns++] = sx;
                a.M = g.N * a.Hc * a.Wc;
                a.Kred = a.nr * a.ns * g.K;
                if (a.M == 0) continue;
                if (g_use_tcgen05) {
                    const cudaError_t e = launch_umma<kDgrad2>(a, st);
                    if (e != cudaSuccess) return status_of(e);
                    continue;
                }
                dim3 grid((a.M + BM - 1) / BM, (a.Ncols + BN - 1) / BN);
                k_conv_gemm<kDgrad2><<<grid, NT, 0, st>>>(a);
            }
        return status_of(cudaGetLastError());
    }
    a.M = g.N * g.H * g.W;
    a.Kred = g.R * g.S * g.K;
    if (g_use_tcgen05) return status_of(launch_umma<kDgrad>(a, st));
    dim3 grid((a.M + BM - 1) / BM, (a.Ncols + BN - 1) / BN);
    k_conv_gemm<kDgrad><<<grid, NT, 0, st>>>(a);
    return status_of(cudaGetLastError());
}

static int bias_chunks(const Geo &g) {
    if (256 % g.K) return 0;
    return (int)(((int64_t)g.N * g.P * g.Q + bias_chunk(g.K) - 1) / bias_chunk(g.K));
}

size_t osog_conv2d_backward_filter_workspace(const osog_conv_shape_t *shape) {
    if (!shape_ok(shape)) return 0;
    const Geo g = geo_of(shape);
    return ((size_t)splits_of(g) * g.K * g.R * g.S * g.C + (size_t)bias_chunks(g) * g.K) *
           sizeof(float);
}

int osog_conv2d_backward_filter(const osog_conv_shape_t *shape, const uint16_t *dy,
                                const uint16_t *x, float *dw, float *dbias, void *ws,
                                size_t ws_bytes, osog_stream_t stream) {
    if (!shape_ok(shape) || !dy || !x || !dw || !dbias) return OSOG_ERR_INVALID_ARG;
    if (!ws || ws_bytes < osog_conv2d_backward_filter_workspace(shape)) return OSOG_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const Geo g = geo_of(shape);
    Args a{};
    a.g = g;
    a.x = bf(dy);
    a.w = bf(x);
    a.part = static_cast<float *>(ws);
    a.M = g.K;
    a.Ncols = g.R * g.S * g.C;
    a.Kred = g.N * g.P * g.Q;
    const int splits = splits_of(g);
    // tcgen05: output channels as the 128 rows when there are at least 128,
    // else, with at least 64 filter entries, the filter entries as the rows
    // and the output channels (rounded up to 16) as the columns
    if (g_use_tcgen05 && a.M >= UM) {
        const cudaError_t e = umma_prepare();
        if (e != cudaSuccess) return status_of(e);
        dim3 grid((a.M + UM - 1) / UM, (a.Ncols + 127) / 128, splits);
        k_wgrad_umma<false><<<grid, UNT, umma_smem(128), st>>>(a, 128);
    } else if (g_use_tcgen05 && g_wgrad_swap && a.Ncols >= 64) {
        const cudaError_t e = umma_prepare();
        if (e != cudaSuccess) return status_of(e);
        const int bnu = (a.M + 15) / 16 * 16;
        dim3 grid((a.Ncols + UM - 1) / UM, 1, splits);
        k_wgrad_umma<true><<<grid, UNT, umma_smem(bnu), st>>>(a, bnu);
    } else {
        dim3 grid((a.M + BM - 1) / BM, (a.Ncols + BN - 1) / BN, splits);
        k_conv_gemm<kWgrad><<<grid, NT, 0, st>>>(a);
    }
    const int64_t count = (int64_t)a.M * a.Ncols;
    sum_splits(a.part, splits, count, dw, st);
    const int64_t pixels = (int64_t)g.N * g.P * g.Q;
    if (256 % g.K == 0) {
        float *bpart = a.part + (size_t)splits * count;
        const int chunks = bias_chunks(g);
        k_bias_partial<<<chunks, 256, 0, st>>>(bf(dy), pixels, g.K, bpart);
        sum_splits(bpart, chunks, g.K, dbias, st);
    } else {
        k_bias_grad<<<g.K, 256, 0, st>>>(bf(dy), pixels, g.K, dbias);
    }
    return status_of(cudaGetLastError());
}

int osog_relu_backward(const uint16_t *dy, const uint16_t *act, uint16_t *dy_out, int64_t count,
                       osog_stream_t stream) {
    if (!dy || !act || !dy_out || count < 0) return OSOG_ERR_INVALID_ARG;
    if (count == 0) return OSOG_OK;
    k_relu_backward<<<(unsigned)((count + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        bf(dy), bf(act), count, bf(dy_out));
    return status_of(cudaGetLastError());
}

void osog_conv_use_tcgen05(int32_t enable) { g_use_tcgen05 = enable ? 1 : 0; }

int osog_conv_test_wait_limit(int32_t polls) {
    const int v = polls > 0 ? polls : 0;
    return cudaMemcpyToSymbol(g_cnn_probe_polls, &v, sizeof v) == cudaSuccess ? OSOG_OK : OSOG_ERR_CUDA;
}

int osog_conv_sync_status(osog_stream_t stream) {
    if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return OSOG_ERR_CUDA;
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_cnn_status, sizeof v) != cudaSuccess) return OSOG_ERR_CUDA;
    if (!v) return OSOG_OK;
    const int zero = 0;
    if (cudaMemcpyToSymbol(g_cnn_status, &zero, sizeof zero) != cudaSuccess) return OSOG_ERR_CUDA;
    return OSOG_ERR_TIMEOUT;
}

}  // extern "C"
