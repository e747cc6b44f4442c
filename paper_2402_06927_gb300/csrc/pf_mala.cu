// MALA jitter of the window noise: the gradient-informed move that Sec. 5 of the
// paper lists as future work, on the target of the PCN jitter of Sec. 3.1.2:
//   U(dW) = theta (NLL(dW) - log G(dW)) + |dW|^2 / (2 dt)
//         = theta (J(dW) + sum lambda dW) + |dW|^2 / (2 dt),
// J = NLL + 1/2 dt |lambda|^2 the window cost whose gradient dJ/ddW the adjoint
// returns, grad U = theta (dJ/ddW + lambda) + dW / dt.  Preconditioner C = dt:
//   dW' = dW - (h/2) dt grad U(dW) + sqrt(h dt) z.
// Both kernels read and write each noise entry once (HBM-bound, a few bytes per
// entry); the window runs between them are the adjoint's.
#include "sch_internal.h"

namespace sch {

template <typename R>
__global__ void mala_propose_kernel(int N, int Ns, int K, double theta, double h, double dt, const R* __restrict__ dW,
                                    const R* __restrict__ lam, const R* __restrict__ gJ, uint64_t seed, uint64_t ctr,
                                    int particle0, R* __restrict__ dWp) {
    const int nblk = (K + 3) >> 2;
    const size_t tot = (size_t)N * Ns * nblk;
    const double a = 0.5 * h * dt, b = sqrt(h * dt);
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < tot; q += (size_t)gridDim.x * blockDim.x) {
        const int blk = (int)(q % nblk);
        const int s = (int)((q / nblk) % Ns);
        const int p = (int)(q / ((size_t)nblk * Ns));
        double z[4];
        normal4<double>(seed, SCH_TAG_MALA, (uint64_t)blk, (uint64_t)s, (uint64_t)(particle0 + p), ctr, z);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = 4 * blk + e;
            if (k >= K) break;
            const size_t i = ((size_t)p * Ns + s) * K + k;
            const double x = dW[i], l = lam ? (double)lam[i] : 0.0;
            const double g = theta * ((double)gJ[i] + l) + x / dt;
            dWp[i] = (R)(x - a * g + b * z[e]);
        }
    }
}

// one warp per particle: the Metropolis-Hastings decision; on acceptance the
// proposal's noise, cost and gradient replace the current ones
template <typename R>
__global__ void mala_accept_kernel(int N, int NK, double theta, double h, double dt, uint64_t seed, uint64_t ctr,
                                   int particle0, R* __restrict__ dW, const R* __restrict__ dWp,
                                   const R* __restrict__ lam, double* __restrict__ J, const double* __restrict__ Jp,
                                   R* __restrict__ gJ, const R* __restrict__ gJp, int32_t* __restrict__ accepts) {
    const int p = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (p >= N) return;
    const size_t o = (size_t)p * NK;
    const double a = 0.5 * h * dt;
    // lambda.x and |x|^2 at both points, and the two proposal exponents
    double lx = 0.0, lxp = 0.0, xx = 0.0, xpxp = 0.0, qf = 0.0, qb = 0.0;
    for (int i = lane; i < NK; i += 32) {
        const double x = dW[o + i], xp = dWp[o + i], l = lam ? (double)lam[o + i] : 0.0;
        const double g = theta * ((double)gJ[o + i] + l) + x / dt;
        const double gp = theta * ((double)gJp[o + i] + l) + xp / dt;
        const double f = xp - x + a * g;    // exponent of q(x' | x)
        const double r = x - xp + a * gp;   // exponent of q(x | x')
        lx += l * x;
        lxp += l * xp;
        xx += x * x;
        xpxp += xp * xp;
        qf += f * f;
        qb += r * r;
    }
    lx = warp_sum(lx);
    lxp = warp_sum(lxp);
    xx = warp_sum(xx);
    xpxp = warp_sum(xpxp);
    qf = warp_sum(qf);
    qb = warp_sum(qb);
    int acc = 0;
    if (lane == 0) {
        const double U0 = theta * (J[p] + lx) + xx / (2.0 * dt);
        const double U1 = theta * (Jp[p] + lxp) + xpxp / (2.0 * dt);
        const double log_alpha = U0 - U1 + (qf - qb) / (2.0 * h * dt);
        const double logu = log(uniform_open0(seed, SCH_TAG_MALA_ACCEPT, (uint64_t)(particle0 + p), ctr));
        acc = (logu < log_alpha) && isfinite(U1);
    }
    acc = __shfl_sync(FULL, acc, 0);
    if (acc) {
        for (int i = lane; i < NK; i += 32) {
            dW[o + i] = dWp[o + i];
            gJ[o + i] = gJp[o + i];
        }
        if (lane == 0) {
            J[p] = Jp[p];
            if (accepts) accepts[p] += 1;
        }
    }
}

template <typename R>
int launch_mala_propose(int N, int Ns, int K, double theta, double h, double dt, const R* dW, const R* lam,
                        const R* gJ, uint64_t seed, uint64_t ctr, int particle0, R* dWp, cudaStream_t st) {
    const size_t tot = (size_t)N * Ns * ((K + 3) >> 2);
    const size_t blocks = (tot + 255) / 256;
    const int cap = device_sms() * 16;
    const int grid = (int)(blocks < (size_t)cap ? blocks : (size_t)cap);
    mala_propose_kernel<R><<<grid, 256, 0, st>>>(N, Ns, K, theta, h, dt, dW, lam, gJ, seed, ctr, particle0, dWp);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

template <typename R>
int launch_mala_accept(int N, int NK, double theta, double h, double dt, uint64_t seed, uint64_t ctr, int particle0,
                       R* dW, const R* dWp, const R* lam, double* J, const double* Jp, R* gJ, const R* gJp,
                       int32_t* accepts, cudaStream_t st) {
    mala_accept_kernel<R><<<(N + 7) / 8, 256, 0, st>>>(N, NK, theta, h, dt, seed, ctr, particle0, dW, dWp, lam, J, Jp,
                                                      gJ, gJp, accepts);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

template int launch_mala_propose<float>(int, int, int, double, double, double, const float*, const float*,
                                        const float*, uint64_t, uint64_t, int, float*, cudaStream_t);
template int launch_mala_propose<double>(int, int, int, double, double, double, const double*, const double*,
                                         const double*, uint64_t, uint64_t, int, double*, cudaStream_t);
template int launch_mala_accept<float>(int, int, double, double, double, uint64_t, uint64_t, int, float*,
                                       const float*, const float*, double*, const double*, float*, const float*,
                                       int32_t*, cudaStream_t);
template int launch_mala_accept<double>(int, int, double, double, double, uint64_t, uint64_t, int, double*,
                                        const double*, const double*, double*, const double*, double*,
                                        const double*, int32_t*, cudaStream_t);

}  // namespace sch
