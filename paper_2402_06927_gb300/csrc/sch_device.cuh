// Device building blocks of the SCH particle-filter kernels (sm_103a).
//
// * Philox4x64-10 counter-based generator (Salmon et al., SC'11) and the
//   Box-Muller transform, so that every draw is a pure function of
//   (seed, purpose, block, step, particle, stream counter).
// * CTA-wide helpers for the "one particle per CTA" layout: each of the TP
//   threads owns C consecutive nodes of the periodic mesh in registers;
//   neighbours at chunk ends are exchanged with warp shuffles plus a shared
//   memory hop between warps.
// * Cyclic parallel cyclic reduction (PCR) over one row per thread.
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

__device__ __forceinline__ void box_muller(uint64_t a, uint64_t b, float& z0, float& z1) {
    const float u1 = (float)((a >> 11) + 1ull) * 0x1.0p-53f;
    const float u2 = (float)(b >> 11) * 0x1.0p-53f;
    const float r = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// Four normals of block (blk, c1, c2, c3) under key (seed, tag).
template <typename R>
__device__ __forceinline__ void normal4(uint64_t seed, uint64_t tag, uint64_t blk, uint64_t c1,
                                        uint64_t c2, uint64_t c3, R z[4]) {
    const U64x4 r = philox4x64(blk, c1, c2, c3, seed, tag);
    box_muller(r.v0, r.v1, z[0], z[1]);
    box_muller(r.v2, r.v3, z[2], z[3]);
}

// Uniform in (0, 1] from word 0 of block (0, 0, c2, c3).
__device__ __forceinline__ double uniform_open0(uint64_t seed, uint64_t tag, uint64_t c2, uint64_t c3) {
    const U64x4 r = philox4x64(0, 0, c2, c3, seed, tag);
    return (double)((r.v0 >> 11) + 1ull) * 0x1.0p-53;
}

// --------------------------------------------------------------------------
// arithmetic helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

template <typename R> __device__ __forceinline__ R rabs(R x) { return x < R(0) ? -x : x; }
template <typename R> __device__ __forceinline__ bool finite_(R x) { return isfinite(x); }

// --------------------------------------------------------------------------
// CTA exchange helpers.  `base` holds two phases of EXCH_SLOTS 8-byte slots;
// successive exchanges alternate phases, so a slot is rewritten only after a
// later barrier that every reader of its previous value has passed.
// --------------------------------------------------------------------------
constexpr int EXCH_SLOTS = 128;
constexpr int EXCH_BYTES = 2 * EXCH_SLOTS * 8;

struct Exch {
    unsigned char* base;   // shared scratch for neighbour exchange (EXCH_BYTES)
    int phase;
    int tp;                // threads per particle (power of two, >= 32)

    template <typename R>
    __device__ __forceinline__ R* slots() const {
        return reinterpret_cast<R*>(base + (phase & 1) * EXCH_SLOTS * 8);
    }
};

// prev thread's `last` and next thread's `first` (cyclic over tp threads)
template <typename R>
__device__ __forceinline__ void halo(Exch& x, R first, R last, R& prev_last, R& next_first) {
    const int lane = threadIdx.x & 31;
    prev_last = __shfl_sync(FULL, last, (lane + 31) & 31);
    next_first = __shfl_sync(FULL, first, (lane + 1) & 31);
    if (x.tp > 32) {
        const int nw = x.tp >> 5;
        const int warp = threadIdx.x >> 5;
        R* buf = x.slots<R>();
        if (lane == 31) buf[warp] = last;
        if (lane == 0) buf[32 + warp] = first;
        __syncthreads();
        if (lane == 0) prev_last = buf[(warp + nw - 1) & (nw - 1)];
        if (lane == 31) next_first = buf[32 + ((warp + 1) & (nw - 1))];
        x.phase++;
    }
}

// next thread's values of a small tuple (cyclic)
template <typename R, int V>
__device__ __forceinline__ void from_next(Exch& x, const R (&mine)[V], R (&nxt)[V]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int v = 0; v < V; ++v) nxt[v] = __shfl_sync(FULL, mine[v], (lane + 1) & 31);
    if (x.tp > 32) {
        const int nw = x.tp >> 5;
        const int warp = threadIdx.x >> 5;
        R* buf = x.slots<R>();
        if (lane == 0) {
#pragma unroll
            for (int v = 0; v < V; ++v) buf[warp * V + v] = mine[v];
        }
        __syncthreads();
        if (lane == 31) {
            const int w = (warp + 1) & (nw - 1);
#pragma unroll
            for (int v = 0; v < V; ++v) nxt[v] = buf[w * V + v];
        }
        x.phase++;
    }
}

// prev and next thread's single value (cyclic)
template <typename R>
__device__ __forceinline__ void both_neighbours(Exch& x, R mine, R& prev, R& next) {
    halo(x, mine, mine, prev, next);
}

// Block-wide reductions; all threads receive the result.
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

// max of two values across the tp threads of the CTA
template <typename R>
__device__ __forceinline__ void block_max2(Exch& x, R& a, R& b) {
    a = warp_max(a);
    b = warp_max(b);
    if (x.tp > 32) {
        const int nw = x.tp >> 5;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        R* buf = x.slots<R>();
        if (lane == 0) { buf[warp] = a; buf[32 + warp] = b; }
        __syncthreads();
        a = buf[0]; b = buf[32];
        for (int w = 1; w < nw; ++w) { a = fmax(a, buf[w]); b = fmax(b, buf[32 + w]); }
        x.phase++;
    }
}

// sum across the CTA in double
__device__ __forceinline__ double block_sum(Exch& x, double v) {
    v = warp_sum(v);
    if (x.tp > 32) {
        const int nw = x.tp >> 5;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        double* buf = x.slots<double>();
        if (lane == 0) buf[warp] = v;
        __syncthreads();
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += buf[w];
        v = s;
        x.phase++;
    }
    return v;
}

// --------------------------------------------------------------------------
// Cyclic PCR on one row per thread: A_t E_{t-1} + B_t E_t + C_t E_{t+1} = D_t,
// t = 0..tp-1 (indices mod tp, tp a power of two >= 32).  Levels with stride
// s < tp/2 eliminate the neighbours at distance s; at stride tp/2 the two
// neighbours coincide and a 2x2 system closes the solve.
// `pbuf` holds 2 * tp rows of 4 values (double-buffered).
// --------------------------------------------------------------------------
template <typename R>
struct Row4 { R a, c, d, rb; };

template <typename R>
__device__ __forceinline__ R pcr_cyclic(R A, R B, R Cc, R D, Row4<R>* pbuf, int tp) {
    const int t = threadIdx.x;
    int ph = 0;
    for (int s = 1; s < (tp >> 1); s <<= 1) {
        const R rb = rcp(B);
        Row4<R>* buf = pbuf + ph * tp;
        R Am, Cm, Dm, rbm, Ap, Cp, Dp, rbp;
        buf[t] = Row4<R>{A, Cc, D, rb};
        __syncthreads();
        const Row4<R> lo = buf[(t - s) & (tp - 1)];
        const Row4<R> hi = buf[(t + s) & (tp - 1)];
        Am = lo.a; Cm = lo.c; Dm = lo.d; rbm = lo.rb;
        Ap = hi.a; Cp = hi.c; Dp = hi.d; rbp = hi.rb;
        const R k1 = A * rbm;
        const R k2 = Cc * rbp;
        // B' = B - C_{t-s} k1 - A_{t+s} k2
        const R nB = B - Cm * k1 - Ap * k2;
        const R nD = D - Dm * k1 - Dp * k2;
        A = -Am * k1;
        Cc = -Cp * k2;
        B = nB;
        D = nD;
        ph ^= 1;
    }
    // closing 2x2 with the row half a period away
    Row4<R>* buf = pbuf + ph * tp;
    const R e = A + Cc;
    buf[t] = Row4<R>{e, B, D, R(0)};
    __syncthreads();
    const Row4<R> o = buf[t ^ (tp >> 1)];
    // rows: B E_t + e E_j = D ;  o.c E_j + o.a E_t = o.d   (o.a = e_j, o.c = B_j)
    const R det = B * o.c - e * o.a;
    const R E = (D * o.c - e * o.d) / det;
    __syncthreads();   // pbuf may be reused right after
    return E;
}

// Same for a circulant system whose A, B, C are the same on every row at every
// level: only D travels.  k1[l], k2[l] are the level multipliers and
// f1 E = f1 D + f2 D_{t + tp/2} closes the solve.
template <typename R>
__device__ __forceinline__ R pcr_cyclic_const(R D, const R* k1, const R* k2, R f1, R f2, R* dbuf,
                                              int tp) {
    const int t = threadIdx.x;
    int ph = 0, l = 0;
    for (int s = 1; s < (tp >> 1); s <<= 1, ++l) {
        R* buf = dbuf + ph * tp;
        buf[t] = D;
        __syncthreads();
        const R Dm = buf[(t - s) & (tp - 1)];
        const R Dp = buf[(t + s) & (tp - 1)];
        D = D - k1[l] * Dm - k2[l] * Dp;
        ph ^= 1;
    }
    R* buf = dbuf + ph * tp;
    buf[t] = D;
    __syncthreads();
    const R Dj = buf[t ^ (tp >> 1)];
    __syncthreads();
    return f1 * D + f2 * Dj;
}

}  // namespace sch
