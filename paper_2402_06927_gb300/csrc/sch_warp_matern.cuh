// Warp-per-particle window and jitter kernels with the paper's Matern SALT noise
// (Eq. noise_solve2), FP32, n = 64 P CS.  Lane l holds nodes [LN l, LN (l + 1)),
// LN = 2 P CS, in the paired layout of sch_warp.cuh, and the cells with the same
// indices (cell c = [x_c, x_{c+1}]).  Each step the lane forms its cells' weights in
// registers (from dW, or for the jitter from the PCN proposal regenerated from its
// Philox counter), and the k solves of the Matern operator run as warp-partitioned
// constant solves, like the Helmholtz solve of every Picard iteration.  Shared
// memory holds the step's R0 scratch and a column of PCN normals per lane; dW in
// global memory is the only copy of the current noise.  The loop over a step's
// Philox blocks and the k solves are not unrolled: each is one copy of its code,
// which keeps the step within the instruction cache.
#pragma once

#include "sch_warp.cuh"

namespace sch {

// dU/4 at this lane's nodes from its cells' weights wq = (6/h) eta sqrt(h)/8 (dW_c +
// lambda_c dt): the load (6/h) eta (dW_h, phi_i) / 4 = wq_{i-1} + wq_i, then mk solves
// of (6/h)(M + kappa^-2 K), each later one loaded with U_{i-1} + 4 U_i + U_{i+1} =
// (6/h) M U.  MM: how the operator's reduced system is solved (RED_*).
template <int CS, int P, int MM>
__device__ __forceinline__ void wmatern_noise(const ModelArgs<float>& A, const WArgs& W, const float2 (&wq)[P][CS],
                                              float2 (&nq)[P][CS]) {
    float2 pd[P], de[P], E[P], F[P];
    float Ep = 0.f, Fn = 0.f;
    const float2 four = f2b(4.f);
#pragma unroll 1
    for (int j = 0; j < A.mk; ++j) {
        float2 lo, hi, x[P][CS];
        if (j == 0) {
            whalo<CS, P>(wq, lo, hi);
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int i = 0; i < CS; ++i) x[p][i] = f2add(wleft<CS, P>(wq, p, i, lo), wq[p][i]);
        } else {
            wsolved_halo<P>(E, F, Ep, Fn, lo, hi);
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int i = 0; i < CS; ++i)
                    x[p][i] = f2fma(four, nq[p][i], f2add(wleft<CS, P>(nq, p, i, lo), wright<CS, P>(nq, p, i, hi)));
        }
        wsweep<CS, P>(W.mat, x, pd, de);
        wreduced<P, MM>(W.mat, W.rmat, pd, de, E, F, Ep, Fn);
        wback<CS, P>(W.mat, x, F, E, nq);
    }
}

// PCN normals of this lane's cells at step s: Philox4x32-10 (seed, SCH_TAG_PCN) block c / 4
// gives the normals of cells c .. c + 3 (a sub-chunk holds whole blocks).  The blocks
// are drawn in a rolled loop into the lane's column of zsm (cell k of the lane at
// zsm[32 k + lane]; the lane reads back only what it wrote).
template <int CS, int P>
__device__ __forceinline__ void wcell_normals(uint64_t seed, int s, uint64_t pc, uint64_t ctr, float* zsm,
                                              float2 (&z)[P][CS]) {
    static_assert(CS % 4 == 0, "a sub-chunk covers whole Philox blocks");
    constexpr int NB = 2 * P * CS / 4;
    const int lane = threadIdx.x & 31;
    const int b0 = lane * NB;
#pragma unroll 1
    for (int b = 0; b < NB; ++b) {
        float zb[4];
        normal4_32(seed, SCH_TAG_PCN, (uint64_t)(b0 + b), (uint64_t)s, pc, ctr, zb);
#pragma unroll
        for (int e = 0; e < 4; ++e) zsm[(4 * b + e) * 32 + lane] = zb[e];
    }
#pragma unroll
    for (int t = 0; t < 2 * P; ++t)
#pragma unroll
        for (int i = 0; i < CS; ++i) {
            const float v = zsm[(t * CS + i) * 32 + lane];
            if (t < P)
                z[t][i].x = v;
            else
                z[t - P][i].y = v;
        }
}

// shared memory of the Matern warp jitter kernel: R0 scratch, then the normals' columns
template <int CS, int P>
__host__ __device__ constexpr size_t wmatern_smem() {
    return wsmem_base<CS, P>() + (size_t)2 * P * CS * 32 * sizeof(float);
}

// the step's cell weights from the increments v (in: dW or the proposal, out: the
// scaled weights), adding the drift row lam_s (may be null) and its Girsanov terms
template <int CS, int P>
__device__ __forceinline__ void wmatern_weights(const ModelArgs<float>& A, const WArgs& W, const float* lam_s,
                                                float2 (&v)[P][CS], double& gl) {
    if (lam_s) {
        float2 l[P][CS];
        wload<CS, P>(lam_s, l);
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int i = 0; i < CS; ++i) {
                gl += (double)l[p][i].x * (double)v[p][i].x + 0.5 * (double)l[p][i].x * (double)l[p][i].x * A.dt_d;
                gl += (double)l[p][i].y * (double)v[p][i].y + 0.5 * (double)l[p][i].y * (double)l[p][i].y * A.dt_d;
                v[p][i] = f2fma(l[p][i], f2b(A.dt), v[p][i]);
            }
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
        for (int i = 0; i < CS; ++i) v[p][i] = f2mul(v[p][i], f2b(W.mzw));
}

template <int CS, int P, int PM, int HM, int MM>
__global__ void __launch_bounds__(32, WMINB) wmatern_window_kernel(ModelArgs<float> A, WArgs W, WindowIO<float> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* R0sm = reinterpret_cast<float2*>(smem_raw);
    const int p = blockIdx.x;
    const int n = A.n;
    const size_t NQ = (size_t)io.Ns * n;
    const float* dW = io.dW + p * NQ;
    const float* lam = io.lam ? io.lam + p * NQ : nullptr;
    float2 m[P][CS], u[P][CS];
    wload<CS, P>(io.m_in + (size_t)p * n, m);
    wu_from_m<CS, P, HM>(W, m, u);
    int iters = 0, flags = 0;
    double gl = 0.0;
    for (int s = 0; s < io.Ns; ++s) {
        float2 v[P][CS], nq[P][CS];
        wload<CS, P>(dW + (size_t)s * n, v);
        wmatern_weights<CS, P>(A, W, lam ? lam + (size_t)s * n : nullptr, v, gl);
        wmatern_noise<CS, P, MM>(A, W, v, nq);
        wstep_core<CS, P, PM, HM>(A, W, m, u, R0sm, nq, iters, flags);
    }
    wstore<CS, P>(io.m_out + (size_t)p * n, m);
    wstore<CS, P>(io.u_out + (size_t)p * n, u);
    if (io.y) {
        const double mis = warp_sum(wmisfit<CS, P>(A, u, io.y));
        gl = warp_sum(gl);
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

// PCN jittering with the Matern noise (Sec. 3.1.2): n_iter proposals of the window noise,
// each run through the window from m_start and accepted with probability
// min(1, exp(w0 - w1)), w = theta (NLL - log G).
template <int CS, int P, int PM, int HM, int MM>
__global__ void __launch_bounds__(32, WMINB) wmatern_jitter_kernel(ModelArgs<float> A, WArgs W, JitterIO<float> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* R0sm = reinterpret_cast<float2*>(smem_raw);
    float* zsm = reinterpret_cast<float*>(smem_raw + wsmem_base<CS, P>());
    // a device-gated stage reads its temperature, and does nothing when inactive
    if (io.tstate && io.tstate[4] == 0.0) return;
    const double theta = io.tstate ? io.tstate[2] : io.theta;
    const int p = blockIdx.x;
    const int lane = threadIdx.x;
    const int Ns = io.Ns, n = A.n;
    const size_t NQ = (size_t)Ns * n;
    float* dW = io.dW + p * NQ;
    const float* lam = io.lam ? io.lam + p * NQ : nullptr;
    const uint64_t pc = (uint64_t)(io.particle0 + p);
    double nll0 = io.nll[p], lg0 = io.logG ? io.logG[p] : 0.0;
    const float sq = io.sq1mr2 * (float)sqrt(A.dt_d);
    int iters = 0, flags = 0, n_acc = 0;
    for (int j = 0; j < io.n_iter; ++j) {
        const uint64_t ctr = io.ctr + (uint64_t)j;
        float2 m[P][CS], u[P][CS];
        wload<CS, P>(io.m_start + (size_t)p * n, m);
        wu_from_m<CS, P, HM>(W, m, u);
        int fl = 0;
        double gl = 0.0;
        for (int s = 0; s < Ns; ++s) {
            float2 v[P][CS], z[P][CS], nq[P][CS];
            wload<CS, P>(dW + (size_t)s * n, v);
            wcell_normals<CS, P>(io.seed, s, pc, ctr, zsm, z);
#pragma unroll
            for (int q = 0; q < P; ++q)
#pragma unroll
                for (int i = 0; i < CS; ++i)
                    v[q][i] = make_float2(pcn_value(io.rho, v[q][i].x, sq, z[q][i].x),
                                          pcn_value(io.rho, v[q][i].y, sq, z[q][i].y));
            wmatern_weights<CS, P>(A, W, lam ? lam + (size_t)s * n : nullptr, v, gl);
            wmatern_noise<CS, P, MM>(A, W, v, nq);
            wstep_core<CS, P, PM, HM>(A, W, m, u, R0sm, nq, iters, fl);
        }
        const double mis = warp_sum(wmisfit<CS, P>(A, u, io.y));
        gl = warp_sum(gl);
        const double nll1 = 0.5 * mis, lg1 = -gl;
        int acc = 0;
        if (lane == 0) {
            const double w0 = theta * (nll0 - lg0);
            const double w1 = theta * (nll1 - lg1);
            const double logU = log(uniform_open0(io.seed, SCH_TAG_PCN_ACCEPT, pc, ctr));
            acc = (fl == 0) && (logU < w0 - w1);
        }
        acc = __shfl_sync(FULL, acc, 0);
        if (acc) {
            nll0 = nll1;
            lg0 = lg1;
            // store the accepted proposal: each lane rewrites its own cells of every step
            for (int s = 0; s < Ns; ++s) {
                float2 v[P][CS], z[P][CS];
                wload<CS, P>(dW + (size_t)s * n, v);
                wcell_normals<CS, P>(io.seed, s, pc, ctr, zsm, z);
#pragma unroll
                for (int q = 0; q < P; ++q)
#pragma unroll
                    for (int i = 0; i < CS; ++i)
                        v[q][i] = make_float2(pcn_value(io.rho, v[q][i].x, sq, z[q][i].x),
                                              pcn_value(io.rho, v[q][i].y, sq, z[q][i].y));
                wstore<CS, P>(dW + (size_t)s * n, v);
            }
            wstore<CS, P>(io.m_end + (size_t)p * n, m);
            wstore<CS, P>(io.u_end + (size_t)p * n, u);
            n_acc++;
        }
        flags |= fl;
        __syncwarp();
    }
    if (lane == 0) {
        io.nll[p] = nll0;
        if (io.logG) io.logG[p] = lg0;
        if (io.accepts) io.accepts[p] = n_acc;
        if (io.iters) io.iters[p] = iters;
        if (io.status) io.status[p] = flags;
    }
}

}  // namespace sch
