// Device building blocks of the SCH particle-filter kernels (sm_103a).
//
// * Philox4x64-10 and Philox4x32-10 counter-based generators (Salmon et al.,
//   SC'11) and the Box-Muller transform, so that every draw is a pure function of
//   (seed, purpose, block, step, particle, stream counter).
// * Reciprocal and warp-reduction helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sch {

constexpr unsigned FULL = 0xffffffffu;

// --------------------------------------------------------------------------
// Philox4x64-10
// --------------------------------------------------------------------------
constexpr uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t PHILOX_M1 = 0xCA5A826395121157ull;
constexpr uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t PHILOX_W1 = 0xBB67AE8584CAA73Bull;

struct U64x4 { uint64_t v0, v1, v2, v3; };

__device__ __forceinline__ U64x4 philox4x64(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                            uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t lo0 = PHILOX_M0 * c0, hi0 = __umul64hi(PHILOX_M0, c0);
        const uint64_t lo1 = PHILOX_M1 * c2, hi1 = __umul64hi(PHILOX_M1, c2);
        const uint64_t n0 = hi1 ^ c1 ^ k0;
        const uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += PHILOX_W0; k1 += PHILOX_W1;
    }
    return {c0, c1, c2, c3};
}

// Box-Muller on two raw words: u1 = ((a >> 11) + 1) 2^-53 in (0, 1],
// u2 = (b >> 11) 2^-53 in [0, 1); z0 = r cos(2 pi u2), z1 = r sin(2 pi u2).
__device__ __forceinline__ void box_muller(uint64_t a, uint64_t b, double& z0, double& z1) {
    const double u1 = (double)((a >> 11) + 1ull) * 0x1.0p-53;
    const double u2 = (double)(b >> 11) * 0x1.0p-53;
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// A 53-bit integer v times 2^-53 in float, from its high 32 and low 21 bits: two
// 32-bit conversions (a 64-bit integer conversion would run on the narrow FP64 pipe).
__device__ __forceinline__ float u53_to_float(uint64_t v) {
    const float hi = __uint2float_rn((unsigned)(v >> 21));
    const float lo = __uint2float_rn((unsigned)(v & 0x1FFFFFull));
    return fmaf(hi, 0x1.0p-32f, lo * 0x1.0p-53f);
}

// The FP32 transform keeps to the FP32 pipes.  r^2 = -2 ln u1: for u1 <= 15/16 from the
// __logf intrinsic (absolute error below 2^-21.4 on [1/2, 2], so below 6e-6 relative
// here); nearer one, where that bound is large against the value, from the series
// -ln(1 - x) = x + x^2/2 + x^3/3 + x^4/4 + x^5/5 on x = 1 - u1, which the integer gives
// exactly (truncation below 2e-7 relative for x < 1/16).  The angle 2 pi u2 is taken
// as theta + pi with theta = 2 pi (u2 - 1/2) in [-pi, pi), where __sincosf is accurate
// to 2^-21.4, and the signs flipped back.  |z| is within about 4e-6 of the FP64 transform.
__device__ __forceinline__ void box_muller(uint64_t a, uint64_t b, float& z0, float& z1) {
    const uint64_t v = (a >> 11) + 1ull;           // u1 = v 2^-53 in (0, 1]
    const uint64_t w = (1ull << 53) - v;           // 1 - u1 = w 2^-53
    float r2;
    if (w < (1ull << 49)) {
        const float x = u53_to_float(w);
        r2 = 2.0f * x * (1.0f + x * (0.5f + x * (1.0f / 3.0f + x * (0.25f + x * 0.2f))));
    } else {
        r2 = -2.0f * __logf(u53_to_float(v));
    }
    const float r = sqrtf(r2);
    float s, c;
    __sincosf(6.28318531f * (u53_to_float(b >> 11) - 0.5f), &s, &c);
    z0 = -r * c;
    z1 = -r * s;
}

// --------------------------------------------------------------------------
// Philox4x32-10 (the same paper): ten rounds of two 32 x 32 -> 64-bit products on a
// 4 x 32-bit counter, the 2 x 32-bit key bumped by two Weyl constants between rounds.
// The FP32 Matern kernels draw one normal per cell and step from it, where the
// 64-bit products of Philox4x64 would take a third of the step.  Key (seed mod 2^32,
// (seed >> 32) mod 2^16 + tag 2^16), counter words taken mod 2^32.
// --------------------------------------------------------------------------
constexpr uint32_t PHILOX32_M0 = 0xD2511F53u;
constexpr uint32_t PHILOX32_M1 = 0xCD9E8D57u;
constexpr uint32_t PHILOX32_W0 = 0x9E3779B9u;
constexpr uint32_t PHILOX32_W1 = 0xBB67AE85u;

struct U32x4 { uint32_t v0, v1, v2, v3; };

__device__ __forceinline__ U32x4 philox4x32(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                            uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = PHILOX32_M0 * c0, hi0 = __umulhi(PHILOX32_M0, c0);
        const uint32_t lo1 = PHILOX32_M1 * c2, hi1 = __umulhi(PHILOX32_M1, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += PHILOX32_W0; k1 += PHILOX32_W1;
    }
    return {c0, c1, c2, c3};
}

// Box-Muller in FP32 on two 32-bit words: u1 = (a + 1) 2^-32 in (0, 1], u2 = b 2^-32 in
// [0, 1).  As the 53-bit transform: r^2 from __logf where u1 <= 15/16, from the series of
// -ln(1 - x) on x = 1 - u1 = (~a) 2^-32 (exact as an integer) nearer one; the angle as
// theta + pi with theta = 2 pi (u2 - 1/2).
__device__ __forceinline__ void box_muller32(uint32_t a, uint32_t b, float& z0, float& z1) {
    const uint32_t w = ~a;   // (1 - u1) 2^32
    float r2;
    if (w < (1u << 28)) {
        const float x = __uint2float_rn(w) * 0x1.0p-32f;
        r2 = 2.0f * x * (1.0f + x * (0.5f + x * (1.0f / 3.0f + x * (0.25f + x * 0.2f))));
    } else {
        r2 = -2.0f * __logf(fmaf(__uint2float_rn(a), 0x1.0p-32f, 0x1.0p-32f));
    }
    const float r = sqrtf(r2);
    float s, c;
    __sincosf(6.28318531f * fmaf(__uint2float_rn(b), 0x1.0p-32f, -0.5f), &s, &c);
    z0 = -r * c;
    z1 = -r * s;
}

// Four FP32 normals of Philox4x32 block (blk, c1, c2, c3) under (seed, tag)
__device__ __forceinline__ void normal4_32(uint64_t seed, uint64_t tag, uint64_t blk, uint64_t c1, uint64_t c2,
                                           uint64_t c3, float z[4]) {
    const uint32_t k1 = ((uint32_t)(seed >> 32) & 0xFFFFu) | ((uint32_t)tag << 16);
    const U32x4 r = philox4x32((uint32_t)blk, (uint32_t)c1, (uint32_t)c2, (uint32_t)c3, (uint32_t)seed, k1);
    box_muller32(r.v0, r.v1, z[0], z[1]);
    box_muller32(r.v2, r.v3, z[2], z[3]);
}

// Four normals of block (blk, c1, c2, c3) under key (seed, tag).
template <typename R>
__device__ __forceinline__ void normal4(uint64_t seed, uint64_t tag, uint64_t blk, uint64_t c1,
                                        uint64_t c2, uint64_t c3, R z[4]) {
    const U64x4 r = philox4x64(blk, c1, c2, c3, seed, tag);
    box_muller(r.v0, r.v1, z[0], z[1]);
    box_muller(r.v2, r.v3, z[2], z[3]);
}

// PCN proposal rho dW + sqrt(1 - rho^2) sqrt(dt) z, rounded the same way wherever it
// is formed (a window's noise and the stored accepted proposal agree bit for bit)
template <typename R>
__device__ __forceinline__ R pcn_value(R rho, R cur, R sq, R z) {
    return fma(rho, cur, sq * z);
}

// Uniform in (0, 1] from word 0 of block (0, 0, c2, c3).
__device__ __forceinline__ double uniform_open0(uint64_t seed, uint64_t tag, uint64_t c2, uint64_t c3) {
    const U64x4 r = philox4x64(0, 0, c2, c3, seed, tag);
    return (double)((r.v0 >> 11) + 1ull) * 0x1.0p-53;
}

// --------------------------------------------------------------------------
// arithmetic helpers
// --------------------------------------------------------------------------
// FP32: the hardware reciprocal approximation (relative error ~2^-23), ample
// for the 1e-6 Picard tolerance of the FP32 path; FP64: correctly rounded.
__device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

template <typename R> __device__ __forceinline__ R rabs(R x) { return x < R(0) ? -x : x; }
template <typename R> __device__ __forceinline__ bool finite_(R x) { return isfinite(x); }

// --------------------------------------------------------------------------
// warp reductions (every lane receives the result)
// --------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R warp_max(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
    return v;
}
template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

}  // namespace sch
