// Window and jitter kernels with the paper's Matern SALT noise (Eq. noise_solve2):
// one Brownian motion per cell, so a window's noise is Ns x n values per particle.
// Unlike the mode-expansion kernels, which stage a window's K weights per step in
// shared memory, these compute the n cell weights of one step at a time into an
// n-value buffer: thread t writes the weights eta sqrt(h)/8 (dW_c + lambda_c dt) of
// its own cells c in [tC, tC + C), and matern_nodes reads its cells and the one
// before them.  The jitter kernel regenerates each PCN proposal from its Philox
// counter where it needs it (once per step, and once more to store an accepted
// proposal), so dW in global memory is the only copy of the current noise.  Shared
// memory is then the CTA's solver scratch plus n values, and occupancy is set by
// registers.
#pragma once

#include <type_traits>

#include "sch_kernels.cuh"

namespace sch {

// normals of cells [i0, i0 + C) of step s under (seed, tag) at particle counter pc:
// Philox4x32-10 in FP32, Philox4x64-10 in FP64
template <typename R, int C>
__device__ __forceinline__ void cell_normals(uint64_t seed, int i0, int s, uint64_t pc, uint64_t ctr, R (&z)[C]) {
    static_assert(C % 4 == 0, "a chunk covers whole Philox blocks");
#pragma unroll
    for (int b = 0; b < C / 4; ++b) {
        R zb[4];
        if constexpr (std::is_same<R, float>::value)
            normal4_32(seed, SCH_TAG_PCN, (uint64_t)((i0 >> 2) + b), (uint64_t)s, pc, ctr, zb);
        else
            normal4<R>(seed, SCH_TAG_PCN, (uint64_t)((i0 >> 2) + b), (uint64_t)s, pc, ctr, zb);
#pragma unroll
        for (int e = 0; e < 4; ++e) z[4 * b + e] = zb[e];
    }
}

template <typename R, int C, int TP, int S>
__global__ void __launch_bounds__(TP, Occ<R, TP>::minb) matern_window_kernel(ModelArgs<R> A, WindowIO<R> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shm<R, TP>* sh = reinterpret_cast<Shm<R, TP>*>(smem_raw);
    R* wbuf = reinterpret_cast<R*>(smem_raw + shm_base_bytes<R, TP>());
    const int p = blockIdx.x;
    const int n = A.n;
    const size_t NQ = (size_t)io.Ns * n;
    const R* dW = io.dW + p * NQ;
    const R* lam = io.lam ? io.lam + p * NQ : nullptr;
    const int i0 = threadIdx.x * C;
    Field<R, C> f;
    field_start<R, C, TP>(A, sh, io.m_in + (size_t)p * n, f);
    int iters = 0, flags = 0;
    double gl = 0.0;
    for (int s = 0; s < io.Ns; ++s) {
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const size_t q = (size_t)s * n + i0 + i;
            R v = dW[q];
            if (lam) {
                const R l = lam[q];
                gl += (double)l * (double)v + 0.5 * (double)l * (double)l * A.dt_d;
                v += l * A.dt;
            }
            wbuf[i0 + i] = A.mz * v;
        }
        __syncthreads();
        step_any<S, R, C, TP, SCH_NOISE_MATERN>(A, sh, f, wbuf, R(0), R(0), iters, flags);
    }
#pragma unroll
    for (int i = 0; i < C; ++i) {
        io.m_out[(size_t)p * n + i0 + i] = f.m[i];
        io.u_out[(size_t)p * n + i0 + i] = f.u[i];
    }
    if (io.y) {
        double mis = chunk_misfit<R, C>(A, f.u, io.y);
        block_sum2<R, TP>(sh, mis, gl);
        if (threadIdx.x == 0) {
            io.nll[p] = 0.5 * mis;
            if (io.logG) io.logG[p] = -gl;
        }
    }
    if (threadIdx.x == 0) {
        if (io.iters) io.iters[p] = iters;
        if (io.status) io.status[p] = flags;
    }
}

// PCN jittering with the Matern noise: n_iter proposals of the window noise, each run
// through the whole window from m_start and accepted with probability min(1, exp(w0 - w1)).
template <typename R, int C, int TP, int S>
__global__ void __launch_bounds__(TP, Occ<R, TP>::minb) matern_jitter_kernel(ModelArgs<R> A, JitterIO<R> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shm<R, TP>* sh = reinterpret_cast<Shm<R, TP>*>(smem_raw);
    R* wbuf = reinterpret_cast<R*>(smem_raw + shm_base_bytes<R, TP>());
    // a device-gated stage reads its temperature, and does nothing when inactive
    if (io.tstate && io.tstate[4] == 0.0) return;
    const double theta = io.tstate ? io.tstate[2] : io.theta;
    const int p = blockIdx.x;
    const int Ns = io.Ns, n = A.n;
    const size_t NQ = (size_t)Ns * n;
    R* dW = io.dW + p * NQ;
    const R* lam = io.lam ? io.lam + p * NQ : nullptr;
    const uint64_t pc = (uint64_t)(io.particle0 + p);
    __shared__ double sh_state[2];
    __shared__ int sh_acc;
    if (threadIdx.x == 0) {
        sh_state[0] = io.nll[p];
        sh_state[1] = io.logG ? io.logG[p] : 0.0;
    }
    const R sq = io.sq1mr2 * (R)sqrt(A.dt_d);
    const int i0 = threadIdx.x * C;
    int iters = 0, flags = 0, n_acc = 0;
    for (int j = 0; j < io.n_iter; ++j) {
        const uint64_t ctr = io.ctr + (uint64_t)j;
        Field<R, C> f;
        field_start<R, C, TP>(A, sh, io.m_start + (size_t)p * n, f);
        int fl = 0;
        double gl = 0.0;
        for (int s = 0; s < Ns; ++s) {
            R z[C];
            cell_normals<R, C>(io.seed, i0, s, pc, ctr, z);
#pragma unroll
            for (int i = 0; i < C; ++i) {
                const size_t q = (size_t)s * n + i0 + i;
                R v = pcn_value(io.rho, dW[q], sq, z[i]);
                if (lam) {
                    const R l = lam[q];
                    gl += (double)l * (double)v + 0.5 * (double)l * (double)l * A.dt_d;
                    v += l * A.dt;
                }
                wbuf[i0 + i] = A.mz * v;
            }
            __syncthreads();
            step_any<S, R, C, TP, SCH_NOISE_MATERN>(A, sh, f, wbuf, R(0), R(0), iters, fl);
        }
        double mis = chunk_misfit<R, C>(A, f.u, io.y);
        block_sum2<R, TP>(sh, mis, gl);
        if (threadIdx.x == 0) {
            const double nll1 = 0.5 * mis, lg1 = -gl;
            const double w0 = theta * (sh_state[0] - sh_state[1]);
            const double w1 = theta * (nll1 - lg1);
            const double logU = log(uniform_open0(io.seed, SCH_TAG_PCN_ACCEPT, pc, ctr));
            const int acc = (fl == 0) && (logU < w0 - w1);
            sh_acc = acc;
            if (acc) {
                sh_state[0] = nll1;
                sh_state[1] = lg1;
            }
        }
        __syncthreads();
        if (sh_acc) {
            // store the accepted proposal: each thread rewrites its own cells of every step
            for (int s = 0; s < Ns; ++s) {
                R z[C];
                cell_normals<R, C>(io.seed, i0, s, pc, ctr, z);
#pragma unroll
                for (int i = 0; i < C; ++i) {
                    const size_t q = (size_t)s * n + i0 + i;
                    dW[q] = pcn_value(io.rho, dW[q], sq, z[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < C; ++i) {
                io.m_end[(size_t)p * n + i0 + i] = f.m[i];
                io.u_end[(size_t)p * n + i0 + i] = f.u[i];
            }
            n_acc++;
        }
        flags |= fl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        io.nll[p] = sh_state[0];
        if (io.logG) io.logG[p] = sh_state[1];
        if (io.accepts) io.accepts[p] = n_acc;
        if (io.iters) io.iters[p] = iters;
        if (io.status) io.status[p] = flags;
    }
}

template <typename R, int C, int TP>
struct LaunchMatern {
    static size_t smem(int n) { return shm_base_bytes<R, TP>() + (size_t)n * sizeof(R); }

    template <typename Kern>
    static void prep(Kern k, size_t sm) {
        if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    }
    template <int S>
    static int window(const ModelArgs<R>& A, const WindowIO<R>& io, int N, cudaStream_t st) {
        const size_t sm = smem(A.n);
        prep(matern_window_kernel<R, C, TP, S>, sm);
        matern_window_kernel<R, C, TP, S><<<N, TP, sm, st>>>(A, io);
        return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
    }
    template <int S>
    static int jitter(const ModelArgs<R>& A, const JitterIO<R>& io, int N, cudaStream_t st) {
        const size_t sm = smem(A.n);
        prep(matern_jitter_kernel<R, C, TP, S>, sm);
        matern_jitter_kernel<R, C, TP, S><<<N, TP, sm, st>>>(A, io);
        return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
    }
};

}  // namespace sch
