// Small kernels around the propagation: Philox draws of the window noise,
// the standalone likelihood / Girsanov weight, synthetic observations of a
// truth trajectory and the EMRE / RB / RES diagnostics of Sec. 4.1.1.
#include <type_traits>

#include "sch_internal.h"

namespace sch {

// dW[p][s][k] = sqrt(dt) z, z from block (k/4, s, particle0 + p, ctr): Philox4x32-10 when
// gen32 (R float), else Philox4x64-10
template <typename R>
__global__ void draw_kernel(int N, int Ns, int K, R sqdt, uint64_t seed, uint64_t tag, uint64_t ctr,
                            int particle0, int gen32, R* dW) {
    const int nblk = (K + 3) >> 2;
    const long long tot = (long long)N * Ns * nblk;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot;
         q += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(q % nblk);
        const int s = (int)((q / nblk) % Ns);
        const int p = (int)(q / ((long long)nblk * Ns));
        R z[4];
        if constexpr (std::is_same<R, float>::value) {
            if (gen32)
                normal4_32(seed, tag, (uint64_t)b, (uint64_t)s, (uint64_t)(particle0 + p), ctr, z);
            else
                normal4<R>(seed, tag, (uint64_t)b, (uint64_t)s, (uint64_t)(particle0 + p), ctr, z);
        } else {
            normal4<R>(seed, tag, (uint64_t)b, (uint64_t)s, (uint64_t)(particle0 + p), ctr, z);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = 4 * b + e;
            if (k < K) dW[((size_t)p * Ns + s) * K + k] = sqdt * z[e];
        }
    }
}

// one warp per particle: nll and logG of given end states
template <typename R>
__global__ void loglik_kernel(ModelArgs<R> A, int N, const R* u, const R* y, const R* dW,
                              const R* lam, int Ns, double* nll, double* logG) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= N) return;
    const R* up = u + (size_t)warp * A.n;
    double acc = 0.0;
    for (int j = lane; j < A.M; j += 32) {
        const R yj = y[j];
        if (yj != yj) continue;   // NaN: not observed
        const R r = (up[j * A.stride] - yj) * A.sigma_inv;
        acc += (double)r * (double)r;
    }
    acc = warp_sum(acc);
    double g = 0.0;
    if (lam) {
        const int NK = Ns * A.K;
        for (int q = lane; q < NK; q += 32) {
            const double l = lam[(size_t)warp * NK + q], w = dW[(size_t)warp * NK + q];
            g += l * w + 0.5 * l * l * A.dt_d;
        }
    }
    g = warp_sum(g);
    if (lane == 0) {
        nll[warp] = 0.5 * acc;
        if (logG) logG[warp] = -g;
    }
}

template <typename R>
int launch_draw(int N, int Ns, int K, R sqdt, uint64_t seed, uint64_t tag, uint64_t ctr, int particle0,
                int gen32, R* dW, cudaStream_t st) {
    const long long tot = (long long)N * Ns * ((K + 3) / 4);
    const int threads = 256;
    long long blocks = (tot + threads - 1) / threads;
    if (blocks > (long long)device_sms() * 16) blocks = (long long)device_sms() * 16;
    if (blocks < 1) blocks = 1;
    draw_kernel<R><<<(int)blocks, threads, 0, st>>>(N, Ns, K, sqdt, seed, tag, ctr, particle0, gen32, dW);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

template <typename R>
int launch_loglik(const ModelArgs<R>& A, int N, const R* u, const R* y, const R* dW, const R* lam, int Ns,
                  double* nll, double* logG, cudaStream_t st) {
    const int threads = 256;
    const int blocks = (N * 32 + threads - 1) / threads;
    loglik_kernel<R><<<blocks, threads, 0, st>>>(A, N, u, y, dW, lam, Ns, nll, logG);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

template int launch_draw<float>(int, int, int, float, uint64_t, uint64_t, uint64_t, int, int, float*,
                                 cudaStream_t);
template int launch_draw<double>(int, int, int, double, uint64_t, uint64_t, uint64_t, int, int, double*,
                                 cudaStream_t);
template int launch_loglik<float>(const ModelArgs<float>&, int, const float*, const float*, const float*,
                                  const float*, int, double*, double*, cudaStream_t);
template int launch_loglik<double>(const ModelArgs<double>&, int, const double*, const double*,
                                   const double*, const double*, int, double*, double*, cudaStream_t);

// y_j = u(x_j) + sigma z_j, z_j keyed (seed, SCH_TAG_OBS, (j / 4, 0, 0, ctr))
template <typename R>
__global__ void synth_obs_kernel(ModelArgs<R> A, const R* u, uint64_t seed, uint64_t ctr, R sigma, R* y) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= A.M) return;
    R z[4];
    normal4<R>(seed, SCH_TAG_OBS, (uint64_t)(j >> 2), 0, 0, ctr, z);
    y[j] = u[j * A.stride] + sigma * z[j & 3];
}

// ensemble sum per node, particles split over gridDim.y groups: ws[i] += sum_p u[p][i]
// (in double: the mean's error enters RB and the RMSE through u_a - mean, which is
// small against u)
template <typename R>
__global__ void diag_sum_kernel(ModelArgs<R> A, int N, const R* u, double* ws) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    double s = 0.0;
    for (int p = blockIdx.y; p < N; p += gridDim.y) s += (double)u[(size_t)p * A.n + i];
    atomicAdd(&ws[i], s);
}

// ensemble mean per node and the truth-based node sums:
// ws[i] <- mean_p u[p][i]; out[4] += u_a^2; out[5] += (u_a - mean)^2
template <typename R>
__global__ void diag_mean_kernel(ModelArgs<R> A, int N, const R* ua, double* ws, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double a = 0.0, b = 0.0;
    if (i < A.n) {
        const double mean = ws[i] / N;
        ws[i] = mean;
        const double t = (double)ua[i];
        a = t * t;
        b = (t - mean) * (t - mean);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[4], a);
        atomicAdd(&out[5], b);
    }
}

// one warp per particle: out[6] += |u_p - u_a|, out[7] += |u_p - mean|
template <typename R>
__global__ void diag_particle_kernel(ModelArgs<R> A, int N, const R* u, const R* ua, const double* ws,
                                     double* out) {
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= N) return;
    double e = 0.0, f = 0.0;
    for (int i = lane; i < A.n; i += 32) {
        const double v = (double)u[(size_t)p * A.n + i];
        const double d1 = v - (double)ua[i], d2 = v - ws[i];
        e += d1 * d1;
        f += d2 * d2;
    }
    e = warp_sum(e);
    f = warp_sum(f);
    if (lane == 0) {
        atomicAdd(&out[6], sqrt(e));
        atomicAdd(&out[7], sqrt(f));
    }
}

// The same for float fields, with the arithmetic in float: each warp takes particles
// w, w + W, ... and holds its lanes' nodes' mean and truth in registers (NPL = n / 32
// nodes a lane, n <= 32 NPL); a particle's sums of squares run in float over the lane's
// nodes and a 5-level warp tree (relative error below (NPL + 5) 2^-24), and only their
// square roots are accumulated in double, then added once per block.
template <int NPL>
__global__ void diag_particle_f32_kernel(ModelArgs<float> A, int N, const float* u, const float* ua,
                                         const double* ws, double* out) {
    __shared__ double part[2][8];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = blockIdx.x * (blockDim.x >> 5) + wib;
    const int W = gridDim.x * (blockDim.x >> 5);
    float t[NPL], mn[NPL];
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
        const int i = lane + 32 * k;
        t[k] = i < A.n ? ua[i] : 0.f;
        mn[k] = i < A.n ? (float)ws[i] : 0.f;
    }
    double e = 0.0, f = 0.0;
    for (int p = warp; p < N; p += W) {
        float se = 0.f, sf = 0.f;
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            const int i = lane + 32 * k;
            if (i < A.n) {
                const float v = u[(size_t)p * A.n + i];
                const float d1 = v - t[k], d2 = v - mn[k];
                se = fmaf(d1, d1, se);
                sf = fmaf(d2, d2, sf);
            }
        }
        se = warp_sum(se);
        sf = warp_sum(sf);
        e += (double)sqrtf(se);
        f += (double)sqrtf(sf);
    }
    if (lane == 0) {
        part[0][wib] = e;
        part[1][wib] = f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += part[0][w];
            b += part[1][w];
        }
        atomicAdd(&out[6], a);
        atomicAdd(&out[7], b);
    }
}

// The same for float fields of any n up to DIAG_SMEM_N: the truth and the mean staged in
// shared memory as float (the block's threads load them once), then each warp as above.
constexpr int DIAG_SMEM_N = 4096;   // 32 KB of shared memory, within the default limit
__global__ void diag_particle_f32_smem_kernel(ModelArgs<float> A, int N, const float* u, const float* ua,
                                              const double* ws, double* out) {
    extern __shared__ float tm[];   // [n] truth, [n] mean
    __shared__ double part[2][8];
    const int n = A.n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        tm[i] = ua[i];
        tm[n + i] = (float)ws[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = blockIdx.x * (blockDim.x >> 5) + wib;
    const int W = gridDim.x * (blockDim.x >> 5);
    double e = 0.0, f = 0.0;
    for (int p = warp; p < N; p += W) {
        const float* up = u + (size_t)p * n;
        float se = 0.f, sf = 0.f;
        for (int i = lane; i < n; i += 32) {
            const float v = up[i];
            const float d1 = v - tm[i], d2 = v - tm[n + i];
            se = fmaf(d1, d1, se);
            sf = fmaf(d2, d2, sf);
        }
        se = warp_sum(se);
        sf = warp_sum(sf);
        e += (double)sqrtf(se);
        f += (double)sqrtf(sf);
    }
    if (lane == 0) {
        part[0][wib] = e;
        part[1][wib] = f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += part[0][w];
            b += part[1][w];
        }
        atomicAdd(&out[6], a);
        atomicAdd(&out[7], b);
    }
}

__global__ void diag_zero_kernel(int n, double* ws, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 8) out[i] = 0.0;
    if (i < n) ws[i] = 0.0;
}

template <typename R>
__global__ void diag_final_kernel(ModelArgs<R> A, int N, double* out) {
    if (threadIdx.x != 0) return;
    const double na = sqrt(out[4]);
    out[0] = out[6] / N / na;                 // EMRE
    out[1] = sqrt(out[5]) / na;               // RB
    out[2] = out[7] / (N - 1) / na;           // RES
    out[3] = sqrt(out[5] / A.n);              // RMSE of the ensemble mean
}

template <typename R>
int launch_synth_obs(const ModelArgs<R>& A, const R* u, uint64_t seed, uint64_t ctr, R* y, cudaStream_t st) {
    synth_obs_kernel<R><<<(A.M + 127) / 128, 128, 0, st>>>(A, u, seed, ctr, R(1) / A.sigma_inv, y);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

// per-particle norms: double fields one warp per particle in double; float fields in
// float with the mean and truth in registers for n up to 32 * 32, in shared memory up to
// DIAG_SMEM_N (else as double)
template <typename R>
void launch_diag_particle(const ModelArgs<R>& A, int N, const R* u, const R* ua, const double* ws, double* out,
                          cudaStream_t st) {
    if constexpr (std::is_same<R, float>::value) {
        // 8 warps a block, blocks enough for one or two particles a warp
        const int blocks = (N + 15) / 16 < 1 ? 1 : (N + 15) / 16;
        if (A.n <= 256) {
            diag_particle_f32_kernel<8><<<blocks, 256, 0, st>>>(A, N, u, ua, ws, out);
            return;
        }
        if (A.n <= 1024) {
            diag_particle_f32_kernel<32><<<blocks, 256, 0, st>>>(A, N, u, ua, ws, out);
            return;
        }
        if (A.n <= DIAG_SMEM_N) {
            // one pass over the ensemble at the memory's pace: a few warps a particle-row in flight
            // on every SM, each block staging the truth and the mean once
            int b2 = device_sms() * 4;
            if (b2 > (N + 7) / 8) b2 = (N + 7) / 8;
            if (b2 < 1) b2 = 1;
            diag_particle_f32_smem_kernel<<<b2, 256, 2 * A.n * sizeof(float), st>>>(A, N, u, ua, ws, out);
            return;
        }
    }
    diag_particle_kernel<R><<<(N * 32 + 255) / 256, 256, 0, st>>>(A, N, u, ua, ws, out);
}

template <typename R>
int launch_diag(const ModelArgs<R>& A, int N, const R* u, const R* ua, double* ws, double* out, cudaStream_t st) {
    const int nb = (A.n + 255) / 256;
    diag_zero_kernel<<<nb, 256, 0, st>>>(A.n, ws, out);
    // particles split over up to 512 groups: short chains of dependent adds per thread
    const int groups = N < 512 ? N : 512;
    diag_sum_kernel<R><<<dim3(nb, groups), 256, 0, st>>>(A, N, u, ws);
    diag_mean_kernel<R><<<nb, 256, 0, st>>>(A, N, ua, ws, out);
    launch_diag_particle<R>(A, N, u, ua, ws, out, st);
    diag_final_kernel<R><<<1, 32, 0, st>>>(A, N, out);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

template int launch_synth_obs<float>(const ModelArgs<float>&, const float*, uint64_t, uint64_t, float*, cudaStream_t);
template int launch_synth_obs<double>(const ModelArgs<double>&, const double*, uint64_t, uint64_t, double*,
                                      cudaStream_t);
template int launch_diag<float>(const ModelArgs<float>&, int, const float*, const float*, double*, double*,
                                cudaStream_t);
template int launch_diag<double>(const ModelArgs<double>&, int, const double*, const double*, double*, double*,
                                 cudaStream_t);

}  // namespace sch
