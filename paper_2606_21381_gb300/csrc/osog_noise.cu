// Sensor noise epilogue (Sec. III.C: the digitised output carries Poisson
// photon shot noise plus Gaussian read noise).
//
// out_i = (Poisson(g max(I_i, 0)) + sigma Z_i) / g, g photo-electrons per
// unit intensity, sigma the read noise in electrons, Z_i standard normal.
// Random numbers come from the counter-based Philox4x32-10 generator
// (Salmon, Moraes, Dror and Shaw, SC 2011) keyed by the 64-bit seed, one
// counter (i, round, tag) per element and round, so every element's draw is
// independent of the launch shape and reproducible.  Round 0 gives the two
// uniforms of the Box-Muller normal and the first Poisson attempt; rounds
// 1.. two more attempts each.  Poisson: inversion by sequential search for
// rates below 10, Hormann's transformed rejection with squeeze (PTRS, 1993)
// above.  Decisions and the normal are taken in double precision.
#include <math.h>
#include <stdint.h>

#include "osog.h"

namespace osog {
namespace noise {
namespace {

constexpr uint32_t kTag = 0x6E6F6973u;  // fourth counter word
constexpr int kRounds = 64;            // attempts cap (2 per round)

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ double unit_open(uint32_t x) {
    return ((double)x + 0.5) * (1.0 / 4294967296.0);
}

__device__ __forceinline__ void uniforms(uint64_t seed, int64_t i, uint32_t round, double u[4]) {
    uint32_t c[4] = {(uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32), round, kTag};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
#pragma unroll
    for (int k = 0; k < 4; ++k) u[k] = unit_open(c[k]);
}

__device__ int64_t poisson(double lam, uint64_t seed, int64_t i, const double u0[4]) {
    if (!(lam > 0.0)) return 0;
    if (lam < 10.0) {
        double p = exp(-lam), F = p;
        int64_t k = 0;
        while (u0[2] > F && k < 1000) {
            ++k;
            p *= lam / (double)k;
            F += p;
        }
        return k;
    }
    const double slam = sqrt(lam), loglam = log(lam);
    const double b = 0.931 + 2.53 * slam;
    const double a = -0.059 + 0.02483 * b;
    const double invalpha = 1.1239 + 1.1328 / (b - 3.4);
    const double vr = 0.9277 - 3.6224 / (b - 2.0);
    double u[4] = {u0[0], u0[1], u0[2], u0[3]};
    for (int r = 0; r < kRounds; ++r) {
        if (r > 0) uniforms(seed, i, (uint32_t)r, u);
        for (int h = (r == 0 ? 1 : 0); h < 2; ++h) {
            const double U = u[2 * h] - 0.5, V = u[2 * h + 1];
            const double us = 0.5 - fabs(U);
            const double k = floor((2.0 * a / us + b) * U + lam + 0.43);
            if (us >= 0.07 && V <= vr) return (int64_t)k;
            if (k < 0.0 || (us < 0.013 && V > us)) continue;
            if (log(V * invalpha / (a / (us * us) + b)) <= -lam + k * loglam - lgamma(k + 1.0))
                return (int64_t)k;
        }
    }
    return (int64_t)floor(lam);
}

__global__ void k_sensor_noise(const float *__restrict__ img, int64_t count, double g,
                               double sigma, uint64_t seed, float *__restrict__ out) {
    const double pi2 = 6.283185307179586476925286766559;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        double u[4];
        uniforms(seed, i, 0, u);
        const float v = img[i];
        const double lam = g * (v > 0.f ? (double)v : 0.0);
        const double z = sqrt(-2.0 * log(u[0])) * cos(pi2 * u[1]);
        out[i] = (float)(((double)poisson(lam, seed, i, u) + sigma * z) / g);
    }
}

}  // namespace
}  // namespace noise
}  // namespace osog

extern "C" int osog_sensor_noise(const float *image, int64_t count, double photons_per_unit,
                                 double read_sigma, uint64_t seed, float *out,
                                 osog_stream_t stream) {
    if (count < 0 || (count > 0 && (!image || !out))) return OSOG_ERR_INVALID_ARG;
    if (!(photons_per_unit > 0.0) || !(photons_per_unit <= 1e12) || !(read_sigma >= 0.0) ||
        !isfinite(read_sigma))
        return OSOG_ERR_INVALID_ARG;
    if (count == 0) return OSOG_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return OSOG_ERR_CUDA;
    const int64_t want = (count + 255) / 256;
    const int blocks = (int)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
    osog::noise::k_sensor_noise<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        image, count, photons_per_unit, read_sigma, seed, out);
    return cudaGetLastError() == cudaSuccess ? OSOG_OK : OSOG_ERR_CUDA;
}
