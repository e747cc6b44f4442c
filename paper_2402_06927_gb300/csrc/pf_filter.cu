// Filter kernels on sm_103a: adaptive tempering by an ESS root search, systematic
// resampling on exact integers, and the row gather that copies resampled
// particles (Sec. 3.1.1 and 3.1.2 of the paper).  Weights and cumulative sums
// are FP64 / uint64 regardless of the field precision.
#include <cooperative_groups.h>

#include "sch_internal.h"

namespace sch {

constexpr int TEMPER_CTAS = 8;          // one thread-block cluster
constexpr int TEMPER_PER_THREAD = 8;    // N <= 8 * 256 * 8 = 16384
// threads per CTA: 128 up to N = 8 * 128 = 1024 (one particle per thread, every CTA
// busy), else 256.  The FP64 pipe bounds an evaluation, and every thread's share of
// the reductions runs on it; above N = 1024 the wider CTA shortens each thread's
// serial chain of exponentials.
constexpr int TEMPER_THREADS_SMALL = 128, TEMPER_THREADS_LARGE = 256;
constexpr int RESAMPLE_THREADS = 1024;

// Adaptive tempering on one cluster of TEMPER_CTAS CTAs: every CTA holds a
// slice of the particles, ESS evaluations reduce (sum w, sum w^2) in the CTA,
// then across the cluster through distributed shared memory.  Every CTA sums
// the partials in the same order, so all CTAs take identical root-search
// decisions.  Partials are double-buffered by evaluation parity, so one
// cluster barrier per evaluation suffices.
struct TemperShm {
    double part[2][2];      // [parity][s1, s2] of this CTA
    double warp[2][8];      // per-warp partials (s1, s2)
    double minw[8];
};

template <int TPT>
__device__ __forceinline__ double cta_min(double v, TemperShm* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(FULL, v, o));
    if (lane == 0) sh->minw[warp] = v;
    __syncthreads();
    double m = sh->minw[0];
    for (int w = 1; w < TPT / 32; ++w) m = fmin(m, sh->minw[w]);
    __syncthreads();
    return m;
}

// The sums S1 = sum w_e and S2 = sum w_e^2 of the weights w_e = exp(-d phi_e - max),
// max = -d phi_min, over the cluster (ESS = S1^2 / S2, Eq. ess); the thread's weights
// are returned in w.  Every thread sums the CTAs' partials in rank order, so all CTAs
// take identical decisions.  (Folding them over 8 lanes with shuffles instead, each
// lane reading another CTA, measured slower at 256 threads: 216 us against 165 per
// search at N = 8192.)
template <int TPT>
__device__ __forceinline__ void ess_sums(double d, const double (&phi)[TEMPER_PER_THREAD], int cnt, double phimin,
                                         TemperShm* sh, int& parity, double& S1, double& S2,
                                         double (&w)[TEMPER_PER_THREAD]) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const double mx = -d * phimin;
    double s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int e = 0; e < TEMPER_PER_THREAD; ++e) {
        w[e] = 0.0;
        if (e < cnt) {
            w[e] = exp(-d * phi[e] - mx);
            s1 += w[e];
            s2 += w[e] * w[e];
        }
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sh->warp[0][warp] = s1;
        sh->warp[1][warp] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < TPT / 32; ++w) {
            a += sh->warp[0][w];
            b += sh->warp[1][w];
        }
        sh->part[parity][0] = a;
        sh->part[parity][1] = b;
    }
    cl.sync();
    double t1 = 0.0, t2 = 0.0;
    for (int r = 0; r < TEMPER_CTAS; ++r) {
        const TemperShm* o = cl.map_shared_rank(sh, r);
        t1 += o->part[parity][0];
        t2 += o->part[parity][1];
    }
    parity ^= 1;
    S1 = t1;
    S2 = t2;
}

template <int TPT>
__global__ void __cluster_dims__(TEMPER_CTAS, 1, 1) __launch_bounds__(TPT)
    temper_kernel(int N, const double* __restrict__ nll, const double* __restrict__ logG, double theta,
                  const double* __restrict__ theta_dev, double ess_min, int halving, double* __restrict__ wbar,
                  double* __restrict__ out) {
    namespace cg = cooperative_groups;
    __shared__ TemperShm shm;
    TemperShm* sh = &shm;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    // device-gated stage: the temperature comes from the previous stage's result; a
    // stage that starts at theta = 1 is inactive and only says so (out[4] = 0)
    if (theta_dev) {
        theta = *theta_dev;
        if (theta >= 1.0) {
            if (rank == 0 && threadIdx.x == 0) {
                out[0] = 0.0;
                out[1] = 0.0;
                out[2] = 1.0;
                out[3] = 0.0;
                out[4] = 0.0;
            }
            return;
        }
    }
    const int gt = rank * TPT + threadIdx.x;                  // global thread index in the cluster
    constexpr int STRIDE = TEMPER_CTAS * TPT;
    // thread gt owns particles gt, gt + STRIDE, ... (coalesced)
    double phi[TEMPER_PER_THREAD];
    int cnt = 0;
    double lmin = INFINITY;
#pragma unroll
    for (int e = 0; e < TEMPER_PER_THREAD; ++e) {
        const int i = gt + e * STRIDE;
        if (i < N) {
            phi[e] = logG ? nll[i] - logG[i] : nll[i];
            lmin = fmin(lmin, phi[e]);
            cnt = e + 1;
        } else {
            phi[e] = 0.0;
        }
    }
    // cluster-wide minimum of phi
    double cmin = cta_min<TPT>(lmin, sh);
    if (threadIdx.x == 0) sh->part[1][0] = cmin;
    cl.sync();
    double phimin = INFINITY;
    for (int r = 0; r < TEMPER_CTAS; ++r) phimin = fmin(phimin, cl.map_shared_rank(sh, r)->part[1][0]);
    int parity = 0;   // the next evaluation writes parity 0; parity 1 is free again after its barrier
    const double rest = 1.0 - theta;
    // (s1, s2, wk): the sums and this thread's weights at the current answer, so that
    // the normalised weights need no further pass.  Whether the whole step passes is
    // tested as S1^2 >= ess_min S2 (S2 > 0), without a division.
    double s1, s2, wk[TEMPER_PER_THREAD], wc[TEMPER_PER_THREAD];
    ess_sums<TPT>(rest, phi, cnt, phimin, sh, parity, s1, s2, wk);
    const double s1_rest = s1, s2_rest = s2;
    // The largest dtheta with ESS >= ess_min.  ESS(d) falls monotonically in d
    // (its log-derivative is 2 (E_{w^2}[phi] - E_w[phi]) <= 0), so the root of
    // g(d) = ESS(d) - ess_min is bracketed by [0, rest] (g(0) = N - ess_min >= 0)
    // and found by the Illinois variant of regula falsi: the secant point of the
    // bracket, with the function value at an end kept twice in a row halved, and a
    // midpoint whenever the bracket failed to halve over three steps.  It stops at a
    // relative width of 2^-46 and returns the passing end.  A root below rest 2^-60
    // (astronomically spread phi) gives rest 2^-60, the smallest point 60 bisection
    // steps would try.  (Run on S1^2 - ess_min S2 instead, which has the same root and
    // saves the division, the secant steps needed more evaluations, and a searching call
    // at N = 1024 took 20% longer.)
    double d;
    if (s1 * s1 >= ess_min * s2) {
        d = rest;
    } else if (halving) {
        // the paper's search read literally: halve dtheta until the ESS passes, at most
        // 60 times (the last point tried is kept if none passes)
        d = rest;
        for (int k = 1; k <= 60; ++k) {
            d = ldexp(rest, -k);
            ess_sums<TPT>(d, phi, cnt, phimin, sh, parity, s1, s2, wk);
            if (s1 * s1 >= ess_min * s2) break;
        }
    } else {
        const double dmin = rest * 0x1.0p-60;
        double lo = 0.0, glo = (double)N - ess_min, hi = rest, ghi = s1 * s1 / s2 - ess_min;
        double w3 = rest, w2 = rest, w1 = rest;   // bracket widths of the last three steps
        int side = 0;
        for (int it = 0; it < 200; ++it) {
            const double w = hi - lo;
            if (w <= hi * 0x1.0p-46 || hi < dmin) break;
            double c = (lo * ghi - hi * glo) / (ghi - glo);
            if (!(c > lo && c < hi) || w > 0.5 * w3) c = 0.5 * (lo + hi);
            w3 = w2;
            w2 = w1;
            w1 = w;
            double sc, s2c;
            ess_sums<TPT>(c, phi, cnt, phimin, sh, parity, sc, s2c, wc);
            const double gc = sc * sc / s2c - ess_min;
            if (gc >= 0.0) {
                lo = c;
                glo = gc;
                s1 = sc;
                s2 = s2c;
#pragma unroll
                for (int e = 0; e < TEMPER_PER_THREAD; ++e) wk[e] = wc[e];
                if (side == 1) ghi *= 0.5;
                side = 1;
            } else {
                hi = c;
                ghi = gc;
                if (side == -1) glo *= 0.5;
                side = -1;
            }
        }
        if (lo > 0.0) {
            d = lo;
        } else {
            d = fmax(hi, dmin);
            ess_sums<TPT>(d, phi, cnt, phimin, sh, parity, s1, s2, wk);
        }
    }
    const double ess = s1 * s1 / s2;
    const double ess_rest = s1_rest * s1_rest / s2_rest;
#pragma unroll
    for (int e = 0; e < TEMPER_PER_THREAD; ++e) {
        const int i = gt + e * STRIDE;
        if (i < N) wbar[i] = wk[e] / s1;
    }
    if (rank == 0 && threadIdx.x == 0) {
        out[0] = d;
        out[1] = ess;
        out[2] = (d >= 1.0 - theta) ? 1.0 : theta + d;
        out[3] = ess_rest;
        if (theta_dev) out[4] = 1.0;
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

// Offspring indices of systematic resampling on integers:
// q_i = floor(wbar_i 2^50), C = inclusive scan, T = C_{N-1},
// slot i -> smallest j with C_j > t_i = (i T + floor(U T / 2^53)) / N
// (equal to floor((i 2^53 + U) T / (N 2^53)) since 2^53 divides i 2^53 T).
__global__ void __launch_bounds__(RESAMPLE_THREADS) resample_kernel(int N, const double* __restrict__ wbar,
                                                                    uint64_t seed, uint64_t stage_ctr,
                                                                    const double* __restrict__ gate,
                                                                    int32_t* __restrict__ idx) {
    extern __shared__ __align__(16) unsigned long long Cs[];   // N inclusive sums
    __shared__ unsigned long long wsum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // an inactive device-gated stage keeps every particle in place
    if (gate && *gate == 0.0) {
        for (int i = t; i < N; i += blockDim.x) idx[i] = i;
        return;
    }
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

// Row gathers of several arrays in one launch: blockIdx.y picks the array, whose rows
// move in the widest vector (16, 8 or 4 bytes) that divides the row length.
struct GatherSet {
    const void* src[GATHER_MAX_ARRAYS];
    void* dst[GATHER_MAX_ARRAYS];
    size_t rowv[GATHER_MAX_ARRAYS];
    int vw[GATHER_MAX_ARRAYS];
};

template <typename V>
__device__ __forceinline__ void gather_rows(int N, const int32_t* __restrict__ idx, const V* __restrict__ src,
                                            V* __restrict__ dst, size_t rowv) {
    const size_t tot = (size_t)N * rowv;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
        const size_t row = q / rowv, col = q % rowv;
        dst[q] = src[(size_t)idx[row] * rowv + col];
    }
}

__global__ void gather_multi_kernel(int N, const int32_t* __restrict__ idx, GatherSet g) {
    const int a = blockIdx.y;
    if (g.vw[a] == 16) gather_rows<uint4>(N, idx, (const uint4*)g.src[a], (uint4*)g.dst[a], g.rowv[a]);
    else if (g.vw[a] == 8) gather_rows<uint2>(N, idx, (const uint2*)g.src[a], (uint2*)g.dst[a], g.rowv[a]);
    else gather_rows<unsigned>(N, idx, (const unsigned*)g.src[a], (unsigned*)g.dst[a], g.rowv[a]);
}

__global__ void copy_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t n16) {
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n16; q += (size_t)gridDim.x * blockDim.x)
        dst[q] = src[q];
}

int launch_temper(int N, const double* nll, const double* logG, double theta, const double* theta_dev,
                  double ess_min, int halving, double* wbar, double* out, cudaStream_t st) {
    if (N <= TEMPER_CTAS * TEMPER_THREADS_SMALL)
        temper_kernel<TEMPER_THREADS_SMALL><<<TEMPER_CTAS, TEMPER_THREADS_SMALL, 0, st>>>(
            N, nll, logG, theta, theta_dev, ess_min, halving, wbar, out);
    else
        temper_kernel<TEMPER_THREADS_LARGE><<<TEMPER_CTAS, TEMPER_THREADS_LARGE, 0, st>>>(
            N, nll, logG, theta, theta_dev, ess_min, halving, wbar, out);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

int launch_resample_idx(int N, const double* wbar, uint64_t seed, uint64_t stage_ctr, const double* gate,
                        int32_t* idx, cudaStream_t st) {
    const size_t sm = (size_t)N * sizeof(unsigned long long);
    if (sm > 48 * 1024)
        cudaFuncSetAttribute(resample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    resample_kernel<<<1, RESAMPLE_THREADS, sm, st>>>(N, wbar, seed, stage_ctr, gate, idx);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

static int grid_for(size_t work) {
    size_t b = (work + 255) / 256;
    if (b > (size_t)device_sms() * 8) b = (size_t)device_sms() * 8;
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

int launch_gather_multi(int N, const int32_t* idx, int n, const void* const* src, void* const* dst,
                        const size_t* row_bytes, cudaStream_t st) {
    if (n < 1 || n > GATHER_MAX_ARRAYS) return SCH_ERR_ARG;
    GatherSet g{};
    size_t most = 0;
    for (int a = 0; a < n; ++a) {
        const int vw = row_bytes[a] % 16 == 0 ? 16 : (row_bytes[a] % 8 == 0 ? 8 : 4);
        g.src[a] = src[a];
        g.dst[a] = dst[a];
        g.vw[a] = vw;
        g.rowv[a] = row_bytes[a] / vw;
        most = most > (size_t)N * g.rowv[a] ? most : (size_t)N * g.rowv[a];
    }
    gather_multi_kernel<<<dim3(grid_for(most), n), 256, 0, st>>>(N, idx, g);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

int launch_copy(const void* src, void* dst, size_t bytes, cudaStream_t st) {
    const size_t n16 = bytes / 16;
    copy_kernel<<<grid_for(n16), 256, 0, st>>>((const uint4*)src, (uint4*)dst, n16);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

}  // namespace sch
