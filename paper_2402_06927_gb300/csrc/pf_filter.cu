// Filter kernels on sm_103a: adaptive tempering by ESS bisection, systematic
// resampling on exact integers, and the row gather that copies resampled
// particles (Sec. 3.1.1 and 3.1.2 of the paper).  Weights and cumulative sums
// are FP64 / uint64 regardless of the field precision.
#include "sch_internal.h"

namespace sch {

constexpr int TEMPER_THREADS = 1024;
constexpr int TEMPER_PER_THREAD = 16;   // N <= 16384
constexpr int RESAMPLE_THREADS = 1024;

__device__ __forceinline__ double block_reduce_sum1024(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    s = warp_sum(s);
    return s;
}

__device__ __forceinline__ double block_reduce_min1024(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(FULL, v, o));
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmin(s, __shfl_xor_sync(FULL, s, o));
    return s;
}

// ESS of the weights exp(-d phi_i) (shifted by their maximum -d phi_min):
// ESS = (sum w)^2 / sum w^2  (Eq. ess).
__device__ __forceinline__ double ess_at(double d, const double (&phi)[TEMPER_PER_THREAD], int cnt,
                                         double phimin, double* sh1, double* sh2, double& s1out) {
    const double mx = -d * phimin;
    double s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int e = 0; e < TEMPER_PER_THREAD; ++e) {
        if (e < cnt) {
            const double w = exp(-d * phi[e] - mx);
            s1 += w;
            s2 += w * w;
        }
    }
    s1 = block_reduce_sum1024(s1, sh1);
    s2 = block_reduce_sum1024(s2, sh2);
    s1out = s1;
    return s1 * s1 / s2;
}

__global__ void __launch_bounds__(TEMPER_THREADS) temper_kernel(int N, const double* __restrict__ nll,
                                                                const double* __restrict__ logG,
                                                                double theta, double ess_min,
                                                                double* __restrict__ wbar,
                                                                double* __restrict__ out) {
    __shared__ double sh1[32], sh2[32];
    const int t = threadIdx.x;
    // thread t owns particles t, t + 1024, ... (strided for coalescing)
    double phi[TEMPER_PER_THREAD];
    int cnt = 0;
    double lmin = INFINITY;
#pragma unroll
    for (int e = 0; e < TEMPER_PER_THREAD; ++e) {
        const int i = t + e * TEMPER_THREADS;
        if (i < N) {
            phi[e] = logG ? nll[i] - logG[i] : nll[i];
            lmin = fmin(lmin, phi[e]);
            cnt = e + 1;
        } else {
            phi[e] = 0.0;
        }
    }
    const double phimin = block_reduce_min1024(lmin, sh1);
    const double rest = 1.0 - theta;
    double s1;
    double d;
    double ess = ess_at(rest, phi, cnt, phimin, sh1, sh2, s1);
    if (ess >= ess_min) {
        d = rest;
    } else {
        double lo = 0.0, hi = rest;
        for (int it = 0; it < 60; ++it) {
            const double mid = 0.5 * (lo + hi);
            const double e_mid = ess_at(mid, phi, cnt, phimin, sh1, sh2, s1);
            if (e_mid >= ess_min) lo = mid; else hi = mid;
        }
        d = (lo > 0.0) ? lo : hi;
    }
    ess = ess_at(d, phi, cnt, phimin, sh1, sh2, s1);
    const double mx = -d * phimin;
#pragma unroll
    for (int e = 0; e < TEMPER_PER_THREAD; ++e) {
        const int i = t + e * TEMPER_THREADS;
        if (i < N) wbar[i] = exp(-d * phi[e] - mx) / s1;
    }
    if (t == 0) {
        out[0] = d;
        out[1] = ess;
        out[2] = (d >= 1.0 - theta) ? 1.0 : theta + d;
        out[3] = (ess == ess) ? 0.0 : 1.0;
    }
}

// Offspring indices of systematic resampling on integers:
// q_i = floor(wbar_i 2^50), C = inclusive scan, T = C_{N-1},
// slot i -> smallest j with C_j > t_i = (i T + floor(U T / 2^53)) / N
// (equal to floor((i 2^53 + U) T / (N 2^53)) since 2^53 divides i 2^53 T).
__global__ void __launch_bounds__(RESAMPLE_THREADS) resample_kernel(int N, const double* __restrict__ wbar,
                                                                    uint64_t seed, uint64_t stage_ctr,
                                                                    int32_t* __restrict__ idx) {
    extern __shared__ __align__(16) unsigned long long Cs[];   // N inclusive sums
    __shared__ unsigned long long wsum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (N + RESAMPLE_THREADS - 1) / RESAMPLE_THREADS;
    const int beg = t * per;
    const int end = min(N, beg + per);
    unsigned long long loc = 0;
    for (int i = beg; i < end; ++i) {
        const unsigned long long q = __double2ull_rd(wbar[i] * 0x1.0p50);
        loc += q;
        Cs[i] = loc;
    }
    // exclusive scan of per-thread totals
    unsigned long long v = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long n = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += n;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long n = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += n;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    const unsigned long long off = (v - loc) + (warp > 0 ? wsum[warp - 1] : 0ull);
    for (int i = beg; i < end; ++i) Cs[i] += off;
    __syncthreads();
    const unsigned long long T = Cs[N - 1];
    const U64x4 r = philox4x64(0, 0, 0, stage_ctr, seed, SCH_TAG_RESAMPLE);
    const unsigned long long U = r.v0 >> 11;
    const unsigned long long ut_hi = __umul64hi(U, T), ut_lo = U * T;
    const unsigned long long ut53 = (ut_hi << 11) | (ut_lo >> 53);
    for (int i = t; i < N; i += blockDim.x) {
        const unsigned long long thr = ((unsigned long long)i * T + ut53) / (unsigned long long)N;
        int lo = 0, hi = N - 1;   // smallest j with C_j > thr (C_{N-1} = T > thr)
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (Cs[mid] > thr) hi = mid; else lo = mid + 1;
        }
        idx[i] = lo;
    }
}

template <typename V>
__global__ void gather_kernel(int N, const int32_t* __restrict__ idx, const V* __restrict__ src,
                              V* __restrict__ dst, size_t rowv) {
    const size_t tot = (size_t)N * rowv;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
        const size_t row = q / rowv, col = q % rowv;
        dst[q] = src[(size_t)idx[row] * rowv + col];
    }
}

__global__ void copy_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t n16) {
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n16; q += (size_t)gridDim.x * blockDim.x)
        dst[q] = src[q];
}

int launch_temper(int N, const double* nll, const double* logG, double theta, double ess_min, double* wbar,
                  double* out, cudaStream_t st) {
    temper_kernel<<<1, TEMPER_THREADS, 0, st>>>(N, nll, logG, theta, ess_min, wbar, out);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

int launch_resample_idx(int N, const double* wbar, uint64_t seed, uint64_t stage_ctr, int32_t* idx,
                        cudaStream_t st) {
    const size_t sm = (size_t)N * sizeof(unsigned long long);
    if (sm > 48 * 1024)
        cudaFuncSetAttribute(resample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    resample_kernel<<<1, RESAMPLE_THREADS, sm, st>>>(N, wbar, seed, stage_ctr, idx);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

static int grid_for(size_t work) {
    size_t b = (work + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    return (int)b;
}

int launch_gather(int N, const int32_t* idx, const void* src, void* dst, size_t row_bytes, cudaStream_t st) {
    if (row_bytes % 16 == 0) {
        const size_t rv = row_bytes / 16;
        gather_kernel<uint4><<<grid_for((size_t)N * rv), 256, 0, st>>>(N, idx, (const uint4*)src, (uint4*)dst, rv);
    } else if (row_bytes % 8 == 0) {
        const size_t rv = row_bytes / 8;
        gather_kernel<uint2><<<grid_for((size_t)N * rv), 256, 0, st>>>(N, idx, (const uint2*)src, (uint2*)dst, rv);
    } else {
        const size_t rv = row_bytes / 4;
        gather_kernel<unsigned><<<grid_for((size_t)N * rv), 256, 0, st>>>(N, idx, (const unsigned*)src,
                                                                         (unsigned*)dst, rv);
    }
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

int launch_copy(const void* src, void* dst, size_t bytes, cudaStream_t st) {
    const size_t n16 = bytes / 16;
    copy_kernel<<<grid_for(n16), 256, 0, st>>>((const uint4*)src, (uint4*)dst, n16);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

}  // namespace sch
