// Reverse-mode adjoint of the window and batched L-BFGS nudging (Sec. 3.1.3 of
// the paper: nudging drifts chosen by a gradient optimiser whose gradient is
// computed by the adjoint technique).  One CTA per particle, same chunk layout
// as the forward kernels.
//
// Adjoint of one converged implicit-midpoint step.  With
//   R(m1; m0, dU) = M (m1 - m0) + mu dt K mbar + A(mbar, dv),
//   dv = dt (u0 + u1)/2 + dU,  u = H^{-1} M m,
// the Jacobians are
//   J1 = dR/dm1 = P + (dt/2) B H^{-1} M,   P = M + mu dt/2 K + 1/2 A_dv,
//   J0 = dR/dm0 = -N + (dt/2) B H^{-1} M,  N = M - mu dt/2 K - 1/2 A_dv,
//   dR/d(dU) = B,
// where B is the map v -> A(mbar, v): (B v)_i = 1/2 [S_i v_{i+1} - S_{i-1} v_{i-1}],
// S_i = mbar_i + mbar_{i+1}.  Given g = dJ/dm1, psi solves J1^T psi = g by the
// fixed point P^T psi = g - (dt/2) M H^{-1} B^T psi (the transpose of the
// forward Picard contraction), and
//   dJ/dm0 = N^T psi - (dt/2) M H^{-1} B^T psi,   dJ/d(dU) = -B^T psi.
// All operators are tridiagonal, so every solve reuses the chunk partition.
#pragma once

#include "sch_kernels.cuh"

namespace sch {

// the adjoint and optimiser kernels keep more live state: no occupancy push
template <int TP>
struct OccAdj {
    static constexpr int minb = TP <= 32 ? 16 : (TP <= 64 ? 8 : (TP <= 128 ? 4 : (TP <= 256 ? 2 : 1)));
};

// --------------------------------------------------------------------------
// generic variable cyclic tridiagonal solve: row i reads
// a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i.  Two CTA barriers.
// --------------------------------------------------------------------------
template <typename R, int C, int TP>
__device__ __forceinline__ void var_solve(const R (&a)[C], const R (&b)[C], const R (&c)[C], const R (&d)[C],
                                          R (&x)[C], R& xp, R& xn, Shm<R, TP>* sh) {
    const int t = threadIdx.x;
    R al[C], ga[C], de[C];
    al[0] = R(-1);
    ga[0] = R(0);
    de[0] = R(0);
#pragma unroll
    for (int i = 1; i < C; ++i) {
        const R q = rcp(b[i] - a[i] * ga[i - 1]);
        ga[i] = c[i] * q;
        al[i] = -a[i] * al[i - 1] * q;
        de[i] = (d[i] - a[i] * de[i - 1]) * q;
    }
    sh->ae[t] = al[C - 1];
    sh->ge[t] = ga[C - 1];
    sh->de[t] = de[C - 1];
    {
        R dp = R(0), ap = R(0), gp = R(-1);
#pragma unroll
        for (int i = C - 2; i >= 1; --i) {
            dp = de[i] - ga[i] * dp;
            ap = al[i] - ga[i] * ap;
            gp = -ga[i] * gp;
            de[i] = dp;
            al[i] = ap;
            ga[i] = gp;
        }
    }
    R BF, CF, DF;
    if (C == 2) {
        BF = b[0]; CF = c[0]; DF = d[0];
    } else {
        BF = b[0] - c[0] * al[1];
        CF = -c[0] * ga[1];
        DF = d[0] - c[0] * de[1];
    }
    const R qF = rcp(BF);
    sh->pa[t] = a[0] * qF;
    sh->pc[t] = CF * qF;
    sh->pd[t] = DF * qF;
    __syncthreads();
    if (t < 32) warp_reduce_var<R, TP>(sh);
    __syncthreads();
    const R E = sh->E[t], F = sh->F[t];
    xp = sh->E[(t - 1) & (TP - 1)];
    xn = sh->F[(t + 1) & (TP - 1)];
    x[0] = F;
    x[C - 1] = E;
#pragma unroll
    for (int i = 1; i < C - 1; ++i) x[i] = de[i] - al[i] * F - ga[i] * E;
}

// neighbours of two chunk fields at once (E/F and hE/hF as exchange slots)
template <typename R, int C, int TP>
__device__ __forceinline__ void chunk_halo2(const R (&v)[C], R& vp, R& vn, const R (&w)[C], R& wp, R& wn,
                                           Shm<R, TP>* sh) {
    const int t = threadIdx.x;
    sh->E[t] = v[C - 1];
    sh->F[t] = v[0];
    sh->hE[t] = w[C - 1];
    sh->hF[t] = w[0];
    __syncthreads();
    vp = sh->E[(t - 1) & (TP - 1)];
    vn = sh->F[(t + 1) & (TP - 1)];
    wp = sh->hE[(t - 1) & (TP - 1)];
    wn = sh->hF[(t + 1) & (TP - 1)];
    __syncthreads();
}

// max over the CTA (all threads receive it); one barrier pair
template <typename R, int TP>
__device__ __forceinline__ void block_max2_all(Shm<R, TP>* sh, R& a, R& b) {
    a = warp_max(a);
    b = warp_max(b);
    const int t = threadIdx.x;
    if ((t & 31) == 0) {
        sh->wred[0][t >> 5] = a;
        sh->wred[1][t >> 5] = b;
    }
    __syncthreads();
    a = sh->wred[0][0];
    b = sh->wred[1][0];
    for (int w = 1; w < TP / 32; ++w) {
        a = fmax(a, sh->wred[0][w]);
        b = fmax(b, sh->wred[1][w]);
    }
    __syncthreads();
}

// --------------------------------------------------------------------------
// Adjoint of one converged step.  In: the step's states (m0, u0) -> (m1, u1)
// with chunk-end neighbours, dU/4 at nodes i0-1 .. i0+C, and g = dJ/dm1 (with
// neighbours).  Out: g = dJ/dm0 (with neighbours) and gdu = dJ/d(dU) at the
// chunk's nodes.
// --------------------------------------------------------------------------
template <typename R, int C>
struct StepState {
    R m0[C], u0[C], m1[C], u1[C];
    R m0p, m0n, u0p, u0n, m1p, m1n, u1p, u1n;
};

template <typename R, int C, int TP>
__device__ __forceinline__ void adjoint_step(const ModelArgs<R>& A, Shm<R, TP>* sh, const StepState<R, C>& st,
                                             const R (&nq)[C + 2], R (&g)[C], R& gp, R& gn, R (&gdu)[C],
                                             int& iters, int& flags) {
    // w = dv/4 and S_i = mbar_i + mbar_{i+1} at the chunk and its neighbours
    R w[C], S[C];
    R wp, wn, Sp;
#pragma unroll
    for (int i = 0; i < C; ++i) w[i] = A.dt8 * (st.u0[i] + st.u1[i]) + nq[i + 1];
    wp = A.dt8 * (st.u0p + st.u1p) + nq[0];
    wn = A.dt8 * (st.u0n + st.u1n) + nq[C + 1];
    {
        R mb[C];
#pragma unroll
        for (int i = 0; i < C; ++i) mb[i] = R(0.5) * (st.m0[i] + st.m1[i]);
        const R mbp = R(0.5) * (st.m0p + st.m1p), mbn = R(0.5) * (st.m0n + st.m1n);
#pragma unroll
        for (int i = 0; i < C; ++i) S[i] = mb[i] + ((i == C - 1) ? mbn : mb[i + 1]);
        Sp = mbp + mb[0];
    }
    // rows of P^T: (c0 + w_i) x_{i-1} + (b0 + w_{i+1} - w_{i-1}) x_i + (c0 - w_i) x_{i+1}
    R pa_[C], pb_[C], pc_[C];
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const R wl = (i == 0) ? wp : w[i - 1];
        const R wr = (i == C - 1) ? wn : w[i + 1];
        pa_[i] = A.c0 + w[i];
        pb_[i] = A.b0 + wr - wl;
        pc_[i] = A.c0 - w[i];
    }
    R psi[C], psip = R(0), psin = R(0), corr[C], BT[C];
#pragma unroll
    for (int i = 0; i < C; ++i) { psi[i] = R(0); corr[i] = R(0); BT[i] = R(0); }
    for (int it = 1; it <= A.max_iter; ++it) {
        R rhs[C], pn[C], pnp, pnn;
#pragma unroll
        for (int i = 0; i < C; ++i) rhs[i] = g[i] - corr[i];
        var_solve<R, C, TP>(pa_, pb_, pc_, rhs, pn, pnp, pnn, sh);
        // B^T psi: (B^T x)_j = 1/2 S_{j-1} x_{j-1} - 1/2 S_j x_{j+1}
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const R xl = (i == 0) ? pnp : pn[i - 1];
            const R xr = (i == C - 1) ? pnn : pn[i + 1];
            const R Sl = (i == 0) ? Sp : S[i - 1];
            BT[i] = R(0.5) * (Sl * xl - S[i] * xr);
        }
        // corr = (dt/2) M H^{-1} B^T psi
        R q[C], qp, qn, r[C];
        const_solve<R, C, TP>(A.hel, A.rhel, BT, q, qp, qn, sh);
        mass_apply<R, C>(A.h6, q, qp, qn, r);
        R dmax = R(0), pmax = R(0);
#pragma unroll
        for (int i = 0; i < C; ++i) {
            corr[i] = R(0.5) * A.dt * r[i];
            R dd = rabs(pn[i] - psi[i]);
            if (!(dd == dd)) dd = R(INFINITY);
            dmax = fmax(dmax, dd);
            pmax = fmax(pmax, rabs(pn[i]));
            psi[i] = pn[i];
        }
        psip = pnp;
        psin = pnn;
        block_max2_all<R, TP>(sh, dmax, pmax);
        iters++;
        if (!(dmax < R(INFINITY)) || !(pmax < R(INFINITY))) {
            flags |= SCH_DEV_NONFINITE;
            break;
        }
        if (dmax <= A.tol * pmax) break;
        if (it == A.max_iter) flags |= SCH_DEV_NOCONVERGE;
    }
    // dJ/dm0 = N^T psi - corr,  N^T rows: (c0p - w_i) x_{i-1} + (b0p - w_{i+1} + w_{i-1}) x_i + (c0p + w_i) x_{i+1}
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const R wl = (i == 0) ? wp : w[i - 1];
        const R wr = (i == C - 1) ? wn : w[i + 1];
        const R xl = (i == 0) ? psip : psi[i - 1];
        const R xr = (i == C - 1) ? psin : psi[i + 1];
        g[i] = (A.c0p - w[i]) * xl + (A.b0p - wr + wl) * psi[i] + (A.c0p + w[i]) * xr - corr[i];
        gdu[i] = -BT[i];
    }
    chunk_halo<R, C, TP>(g, gp, gn, sh);
}

// sum over the CTA of sin(j theta_i) x_i and cos(j theta_i) x_i, j = 1 .. K/2:
// each warp reduces with shuffles and lane 0 writes red[warp * K + 2(j-1) (+1)];
// the caller sums over warps after a barrier.  (s1, c1): angle of node i0.
template <typename R, int C>
__device__ __forceinline__ void mode_sums_warp(const ModelArgs<R>& A, R s1, R c1, const R (&x)[C], double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const R twoc = R(2) * c1;
    R sj = s1, cj = c1, sjm = R(0), cjm = R(1);
    for (int j = 0; j < A.K2; ++j) {
        const R rc = A.rot_c[j], rs = A.rot_s[j];
        R sn = sj, cs = cj, as = R(0), ac = R(0);
#pragma unroll
        for (int q = 0; q < C; ++q) {
            as += sn * x[q];
            ac += cs * x[q];
            const R s2 = sn * rc + cs * rs;
            cs = cs * rc - sn * rs;
            sn = s2;
        }
        const double das = warp_sum((double)as), dac = warp_sum((double)ac);
        if (lane == 0) {
            red[warp * A.K + 2 * j] = das;
            red[warp * A.K + 2 * j + 1] = dac;
        }
        const R sn2 = twoc * sj - sjm, cn2 = twoc * cj - cjm;
        sjm = sj;
        cjm = cj;
        sj = sn2;
        cj = cn2;
    }
}

template <typename R, int C>
__device__ __forceinline__ void store_field(R* dst, const R (&v)[C]) {
    const int i0 = threadIdx.x * C;
#pragma unroll
    for (int i = 0; i < C; ++i) dst[i0 + i] = v[i];
}
template <typename R, int C>
__device__ __forceinline__ void load_field(const R* src, R (&v)[C]) {
    const int i0 = threadIdx.x * C;
#pragma unroll
    for (int i = 0; i < C; ++i) v[i] = src[i0 + i];
}

// Matern noise (Eq. noise_solve2): this thread's cell weights eta sqrt(h)/8 (dW_c +
// lambda_c dt) of step s into the n-value buffer wbuf, published by a barrier
template <typename R, int C>
__device__ __forceinline__ void matern_stage_step(const ModelArgs<R>& A, R* wbuf, const R* dW, const R* lam, int s) {
    const int i0 = threadIdx.x * C;
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const size_t q = (size_t)s * A.n + i0 + i;
        R v = dW[q];
        if (lam) v += lam[q] * A.dt;
        wbuf[i0 + i] = A.mz * v;
    }
    __syncthreads();
}

// dJ/dw for this thread's cells c = i0 .. i0 + C - 1 from dJ/ddU at its nodes: the
// transpose of dU = (G^{-1} M)^{k-1} G^{-1} B w, i.e. B^T G^{-1} (M G^{-1})^{k-1}, with
// G = M + kappa^-2 K symmetric and (B^T t)_c = eta sqrt(h)/2 (t_c + t_{c+1})
template <typename R, int C, int TP>
__device__ __forceinline__ void matern_adjoint_cells(const ModelArgs<R>& A, Shm<R, TP>* sh, const R (&gdu)[C],
                                                     R (&gw)[C]) {
    R t[C], x[C], xp, xn;
#pragma unroll
    for (int i = 0; i < C; ++i) t[i] = gdu[i];
    for (int j = 1; j < A.mk; ++j) {
        const_solve<R, C, TP>(A.matern, A.rmatern, t, x, xp, xn, sh);
        mass_apply<R, C>(A.h6, x, xp, xn, t);
    }
    const_solve<R, C, TP>(A.matern, A.rmatern, t, x, xp, xn, sh);
    const R b = R(4) * A.mz;
#pragma unroll
    for (int i = 0; i < C; ++i) gw[i] = b * (x[i] + ((i == C - 1) ? xn : x[i + 1]));
}

// --------------------------------------------------------------------------
// Forward window from step n0 (state at `start`) to Ns, storing the state at
// steps n0, n0 + ck, ... into ckp; returns J = NLL(u_end) + 1/2 dt sum_s sum_k
// lam^2 (all steps) in every thread, and the end state in f.  segst (may be null):
// when the window is one segment (ck >= Ns - n0), every state (m, u) is also stored
// there in backward_ck's segment layout, so that the reverse sweep need not
// recompute it.
// noise: the weights a_j/4 (dW + lam dt) of all Ns steps (staged by the caller); with
// the Matern noise (NZ) an n-value buffer for one step's cell weights, formed here from
// dW and lam.
// --------------------------------------------------------------------------
template <typename R, int C, int TP, int S, int NZ = SCH_NOISE_MODES>
__device__ __forceinline__ double forward_ck(const ModelArgs<R>& A, Shm<R, TP>* sh, R* noise, const R* start,
                                             int n0, int Ns, int ck, R* ckp, const R* lam, const R* y, R s0, R c0,
                                             Field<R, C>& f, int& iters, int& flags, const R* dW = nullptr,
                                             R* segst = nullptr) {
    field_start<R, C, TP>(A, sh, start, f);
    if (segst) {
        store_field<R, C>(segst, f.m);
        store_field<R, C>(segst + A.n, f.u);
    }
    for (int s = n0; s < Ns; ++s) {
        if ((s - n0) % ck == 0) store_field<R, C>(ckp + (size_t)((s - n0) / ck) * A.n, f.m);
        if constexpr (NZ == SCH_NOISE_MATERN) {
            matern_stage_step<R, C>(A, noise, dW, lam, s);
            step_any<S, R, C, TP, NZ>(A, sh, f, noise, s0, c0, iters, flags);
        } else {
            step_any<S, R, C, TP>(A, sh, f, noise + s * A.K, s0, c0, iters, flags);
        }
        if (segst) {
            store_field<R, C>(segst + (size_t)(s - n0 + 1) * 2 * A.n, f.m);
            store_field<R, C>(segst + (size_t)(s - n0 + 1) * 2 * A.n + A.n, f.u);
        }
    }
    double mis = chunk_misfit<R, C>(A, f.u, y);
    double reg = 0.0;
    if (lam)
        for (int q = threadIdx.x; q < Ns * A.K; q += TP) reg += (double)lam[q] * (double)lam[q];
    block_sum2<R, TP>(sh, mis, reg);
    if (threadIdx.x == 0) sh->dsum[0][0] = 0.5 * mis + 0.5 * A.dt_d * reg;
    __syncthreads();
    const double J = sh->dsum[0][0];
    __syncthreads();
    return J;
}

// --------------------------------------------------------------------------
// Reverse sweep after forward_ck: dJ/dlambda for steps [v0, v1) into
// glam[(s - v0) K + k] (and dJ/d dW into gdw when non-null), dJ/dm(n0) into g.
// glam, gdw: any address space, written by threads k < K.  seg_ready: forward_ck
// stored the window's states in seg (one segment), so none is recomputed.
// --------------------------------------------------------------------------
template <typename R, int C, int TP, int S, typename GL, typename GW, int NZ = SCH_NOISE_MODES>
__device__ __forceinline__ void backward_ck(const ModelArgs<R>& A, Shm<R, TP>* sh, R* noise, int n0, int Ns,
                                            int ck, const R* ckp, R* seg, const R* lam, const R* y, R s0, R c0,
                                            R s1, R c1, const Field<R, C>& fend, int v0, int v1, double* red,
                                            GL glam, GW gdw, R (&g)[C], int& iters, int& flags,
                                            const R* dW = nullptr, bool seg_ready = false) {
    const int t = threadIdx.x;
    const int i0 = t * C;
    const int K = A.K;
    // terminal: dJ/du_end = (u - y) / sigma^2 at the observation nodes; dJ/dm = M H^{-1} dJ/du
    R gu[C];
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const int node = i0 + i;
        const R yj = (node % A.stride == 0) ? y[node / A.stride] : R(NAN);
        gu[i] = (yj == yj) ? (fend.u[i] - yj) * A.sigma_inv * A.sigma_inv : R(0);   // NaN: not observed
    }
    R q[C], qp, qn, gp, gn;
    const_solve<R, C, TP>(A.hel, A.rhel, gu, q, qp, qn, sh);
    mass_apply<R, C>(A.h6, q, qp, qn, g);
    chunk_halo<R, C, TP>(g, gp, gn, sh);
    const int ncp = (Ns - n0 + ck - 1) / ck;
    for (int k = ncp - 1; k >= 0; --k) {
        const int sa = n0 + k * ck;
        const int sb = min(sa + ck, Ns);
        if (!(seg_ready && ncp == 1)) {
            Field<R, C> h;
            int dummy_it = 0, dummy_fl = 0;
            field_start<R, C, TP>(A, sh, ckp + (size_t)k * A.n, h);
            store_field<R, C>(seg, h.m);
            store_field<R, C>(seg + A.n, h.u);
            for (int s = sa; s < sb; ++s) {
                if constexpr (NZ == SCH_NOISE_MATERN) {
                    matern_stage_step<R, C>(A, noise, dW, lam, s);
                    step_any<S, R, C, TP, NZ>(A, sh, h, noise, s0, c0, dummy_it, dummy_fl);
                } else {
                    step_any<S, R, C, TP>(A, sh, h, noise + s * K, s0, c0, dummy_it, dummy_fl);
                }
                store_field<R, C>(seg + (size_t)(s - sa + 1) * 2 * A.n, h.m);
                store_field<R, C>(seg + (size_t)(s - sa + 1) * 2 * A.n + A.n, h.u);
            }
        }
        for (int s = sb - 1; s >= sa; --s) {
            StepState<R, C> st;
            const R* sl0 = seg + (size_t)(s - sa) * 2 * A.n;
            const R* sl1 = sl0 + 2 * A.n;
            load_field<R, C>(sl0, st.m0);
            load_field<R, C>(sl0 + A.n, st.u0);
            load_field<R, C>(sl1, st.m1);
            load_field<R, C>(sl1 + A.n, st.u1);
            chunk_halo2<R, C, TP>(st.m0, st.m0p, st.m0n, st.u0, st.u0p, st.u0n, sh);
            chunk_halo2<R, C, TP>(st.m1, st.m1p, st.m1n, st.u1, st.u1p, st.u1n, sh);
            R nq[C + 2];
            if constexpr (NZ == SCH_NOISE_MATERN) {
                matern_stage_step<R, C>(A, noise, dW, lam, s);
                matern_nodes<R, C, TP>(A, sh, noise, nq);
            } else {
                noise_nodes<R, C>(A, noise + s * K, s0, c0, nq);
            }
            R gdu[C];
            adjoint_step<R, C, TP>(A, sh, st, nq, g, gp, gn, gdu, iters, flags);
            if constexpr (NZ == SCH_NOISE_MATERN) {
                // one drift per cell: dJ/dlambda_c = dt dJ/dw_c + dt lambda_c, dJ/ddW_c = dJ/dw_c
                R gw[C];
                matern_adjoint_cells<R, C, TP>(A, sh, gdu, gw);
                if (s >= v0 && s < v1) {
#pragma unroll
                    for (int i = 0; i < C; ++i) {
                        const size_t q = (size_t)(s - v0) * A.n + i0 + i;
                        const double l = lam ? (double)lam[(size_t)s * A.n + i0 + i] : 0.0;
                        glam[q] = A.dt_d * (double)gw[i] + l * A.dt_d;
                        if (gdw) gdw[q] = gw[i];
                    }
                }
            } else if (s >= v0 && s < v1) {
                mode_sums_warp<R, C>(A, s1, c1, gdu, red);
                __syncthreads();
                for (int k = t; k < K; k += TP) {
                    double sum = 0.0;
                    for (int w = 0; w < TP / 32; ++w) sum += red[w * K + k];
                    const double aj = 4.0 * (double)A.amp4[k >> 1];
                    const double l = lam ? (double)lam[s * K + k] : 0.0;
                    glam[(s - v0) * K + k] = A.dt_d * aj * sum + l * A.dt_d;
                    if (gdw) gdw[(s - v0) * K + k] = aj * sum;
                }
                __syncthreads();
            }
        }
    }
}

// --------------------------------------------------------------------------
// kernels
// --------------------------------------------------------------------------
template <typename R, int TP>
__host__ __device__ inline size_t adj_smem_bytes(int Ns, int K) {
    size_t b = shm_base_bytes<R, TP>();
    b += ((size_t)Ns * K * sizeof(R) + 15) / 16 * 16;            // noise weights
    b += (size_t)(TP / 32) * K * sizeof(double);                  // mode-sum partials
    return b;
}

// J and dJ/dlambda, dJ/ddW, dJ/dm0 of a whole window for every particle.  With the
// Matern noise (NZ) the shared noise buffer holds one step's n cell weights, formed per
// step from dW and lambda, and the gradients have one entry per cell.
template <typename R, int C, int TP, int S, int NZ = SCH_NOISE_MODES>
__global__ void __launch_bounds__(TP, OccAdj<TP>::minb) adjoint_kernel(ModelArgs<R> A, AdjointIO<R> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shm<R, TP>* sh = reinterpret_cast<Shm<R, TP>*>(smem_raw);
    R* noise = reinterpret_cast<R*>(smem_raw + shm_base_bytes<R, TP>());
    double* red = reinterpret_cast<double*>(smem_raw + shm_base_bytes<R, TP>() +
                                            ((size_t)io.Ns * A.K * sizeof(R) + 15) / 16 * 16);
    const int p = blockIdx.x;
    const int NK = io.Ns * A.K;
    const R* dWp = io.dW + (size_t)p * NK;
    const R* lamp = io.lam ? io.lam + (size_t)p * NK : nullptr;
    if constexpr (NZ != SCH_NOISE_MATERN) stage_noise(A, noise, dWp, lamp, io.Ns);
    R s0, c0, s1, c1;
    node_angle<R>((int)threadIdx.x * C - 1, A.n, s0, c0);
    node_angle<R>((int)threadIdx.x * C, A.n, s1, c1);
    const int ncp = (io.Ns + io.ck - 1) / io.ck;
    R* ckp = io.ws + (size_t)p * io.ws_per;
    R* seg = ckp + (size_t)ncp * A.n;
    int iters = 0, flags = 0;
    Field<R, C> f;
    // a window of one segment keeps every state from the forward pass
    const bool one = io.ck >= io.Ns;
    const double J = forward_ck<R, C, TP, S, NZ>(A, sh, noise, io.m_start + (size_t)p * A.n, 0, io.Ns, io.ck, ckp,
                                                 lamp, io.y, s0, c0, f, iters, flags, dWp, one ? seg : nullptr);
    if (threadIdx.x == 0) io.J[p] = J;
    R g[C];
    backward_ck<R, C, TP, S, R*, R*, NZ>(A, sh, noise, 0, io.Ns, io.ck, ckp, seg, lamp, io.y, s0, c0, s1, c1, f, 0,
                                         io.Ns, red, io.g_lam + (size_t)p * NK,
                                         io.g_dW ? io.g_dW + (size_t)p * NK : (R*)nullptr, g, iters, flags, dWp, one);
    if (io.g_m0) store_field<R, C>(io.g_m0 + (size_t)p * A.n, g);
    if (threadIdx.x == 0) {
        if (io.iters) io.iters[p] = iters;
        if (io.status) io.status[p] = flags;
    }
}

enum { NUDGE_SEQUENTIAL = 0, NUDGE_OPEN_LOOP = 1 };

template <typename R, int TP>
__host__ __device__ inline size_t nudge_smem_bytes(int Ns, int K) {
    const int nv = Ns * K;
    size_t b = adj_smem_bytes<R, TP>(Ns, K);
    b += 2 * (((size_t)nv * sizeof(R) + 15) / 16 * 16);           // dW and lambda of the window
    b += (size_t)(5 + 2 * LBFGS_M) * nv * sizeof(double) + 2 * LBFGS_M * sizeof(double);
    return b;
}

template <typename R, int TP>
__device__ __forceinline__ double block_dot(Shm<R, TP>* sh, const double* a, const double* b, int nv) {
    double v = 0.0;
    for (int q = threadIdx.x; q < nv; q += TP) v += a[q] * b[q];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh->dsum[1][threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < TP / 32; ++w) s += sh->dsum[1][w];
    __syncthreads();
    return s;
}

template <typename R, int TP>
__device__ __forceinline__ double block_absmax(Shm<R, TP>* sh, const double* a, int nv) {
    double v = 0.0;
    for (int q = threadIdx.x; q < nv; q += TP) v = fmax(v, fabs(a[q]));
    v = warp_max(v);
    if ((threadIdx.x & 31) == 0) sh->dsum[1][threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < TP / 32; ++w) s = fmax(s, sh->dsum[1][w]);
    __syncthreads();
    return s;
}

// Per-particle nudging (Sec. 3.1.3): minimise J = NLL + 1/2 dt sum lambda^2 by
// L-BFGS (two-loop recursion, Armijo backtracking), gradient by the adjoint.
// Sequential schedule: for n = 0..Ns-1 optimise lambda^n with later increments
// and drifts zero, then reveal dW^n (Philox, SCH_TAG_NUDGE, counter
// (k/4, n, particle, ctr)) and advance the start state one step.
// Open loop: optimise all drifts with every increment zero, then reveal all.
//
// With the Matern noise (NZ) the drift has one entry per cell (K = n), the shared noise
// buffer holds one step's cell weights, and the window's drifts, increments and L-BFGS
// vectors live in the particle's workspace (nudge_matern_ws_elems).
template <typename R, int C, int TP, int S, int NZ = SCH_NOISE_MODES>
__global__ void __launch_bounds__(TP, OccAdj<TP>::minb) nudge_kernel(ModelArgs<R> A, NudgeIO<R> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shm<R, TP>* sh = reinterpret_cast<Shm<R, TP>*>(smem_raw);
    const int Ns = io.Ns, K = A.K, NK = Ns * K;
    unsigned char* base = smem_raw + shm_base_bytes<R, TP>();
    R* noise = reinterpret_cast<R*>(base);
    double* red = nullptr;
    R* dWl;
    R* laml;
    if constexpr (NZ == SCH_NOISE_MATERN) {
        // after the adjoint's region: start (n), checkpoints, segment states
        const size_t ws_adj = (size_t)A.n * (1 + (Ns + io.ck - 1) / io.ck + 2 * (io.ck + 1));
        base = reinterpret_cast<unsigned char*>(io.ws + (size_t)blockIdx.x * io.ws_per) +
               (ws_adj * sizeof(R) + 7) / 8 * 8;
        dWl = reinterpret_cast<R*>(base + ((size_t)(5 + 2 * LBFGS_M) * NK + 2 * LBFGS_M) * sizeof(double));
        laml = dWl + NK;
    } else {
        base += ((size_t)NK * sizeof(R) + 15) / 16 * 16;
        red = reinterpret_cast<double*>(base);
        base += (size_t)(TP / 32) * K * sizeof(double);
        dWl = reinterpret_cast<R*>(base);
        base += ((size_t)NK * sizeof(R) + 15) / 16 * 16;
        laml = reinterpret_cast<R*>(base);
        base += ((size_t)NK * sizeof(R) + 15) / 16 * 16;
    }
    double* vx = reinterpret_cast<double*>(base);
    double* vg = vx + NK;
    double* vd = vg + NK;
    double* vxt = vd + NK;
    double* vgt = vxt + NK;
    double* hs = vgt + NK;                   // LBFGS_M x NK
    double* hy = hs + LBFGS_M * NK;          // LBFGS_M x NK
    double* hrho = hy + LBFGS_M * NK;        // LBFGS_M
    double* halpha = hrho + LBFGS_M;         // LBFGS_M

    const int p = blockIdx.x;
    const int t = threadIdx.x;
    R s0, c0, s1, c1;
    node_angle<R>(t * C - 1, A.n, s0, c0);
    node_angle<R>(t * C, A.n, s1, c1);
    const int ck = io.ck;
    R* start = io.ws + (size_t)p * io.ws_per;
    R* ckp = start + A.n;
    const int ncp = (Ns + ck - 1) / ck;
    R* seg = ckp + (size_t)ncp * A.n;
    R* lam_out = io.lam + (size_t)p * NK;
    R* dW_out = io.dW + (size_t)p * NK;
    int flags = 0, iters = 0, lb_iters = 0;

    // window state: start = m_start, dW = 0, lambda = initial guess (open loop) or 0
    {
        R v[C];
        load_field<R, C>(io.m_start + (size_t)p * A.n, v);
        store_field<R, C>(start, v);
    }
    for (int q = t; q < NK; q += TP) {
        dWl[q] = R(0);
        laml[q] = (io.mode == NUDGE_OPEN_LOOP) ? lam_out[q] : R(0);
    }
    __syncthreads();

    const int nstage = (io.mode == NUDGE_OPEN_LOOP) ? 1 : Ns;
    double Jlast = 0.0;
    for (int stage = 0; stage < nstage; ++stage) {
        const int n0 = (io.mode == NUDGE_OPEN_LOOP) ? 0 : stage;
        const int v0 = n0, v1 = (io.mode == NUDGE_OPEN_LOOP) ? Ns : n0 + 1;
        const int nv = (v1 - v0) * K;
        // a window of one segment keeps every state from the forward pass (the last
        // forward before each reverse sweep is the accepted point's)
        const bool one = ck >= Ns - n0;
        // x <- lambda of the variable steps
        for (int q = t; q < nv; q += TP) vx[q] = (double)laml[v0 * K + q];
        __syncthreads();
        auto set_lambda = [&](const double* x) {
            for (int q = t; q < nv; q += TP) laml[v0 * K + q] = (R)x[q];
            __syncthreads();
            if constexpr (NZ != SCH_NOISE_MATERN) stage_noise(A, noise, dWl, laml, Ns);
            __syncthreads();
        };
        Field<R, C> f;
        set_lambda(vx);
        double J = forward_ck<R, C, TP, S, NZ>(A, sh, noise, start, n0, Ns, ck, ckp, laml, io.y, s0, c0, f, iters,
                                               flags, dWl, one ? seg : nullptr);
        R gm[C];
        backward_ck<R, C, TP, S, double*, double*, NZ>(A, sh, noise, n0, Ns, ck, ckp, seg, laml, io.y, s0, c0, s1, c1,
                                                       f, v0, v1, red, vg, (double*)nullptr, gm, iters, flags, dWl,
                                                       one);
        __syncthreads();
        int hist = 0, head = 0;
        double gamma = 1.0;
        for (int it = 0; it < io.max_iter; ++it) {
            const double gmax = block_absmax<R, TP>(sh, vg, nv);
            if (!(gmax > io.gtol)) break;
            // two-loop recursion: vd = -H g
            for (int q = t; q < nv; q += TP) vd[q] = vg[q];
            __syncthreads();
            for (int i = 0; i < hist; ++i) {
                const int slot = (head - 1 - i + LBFGS_M) % LBFGS_M;
                const double a = hrho[slot] * block_dot<R, TP>(sh, hs + slot * NK, vd, nv);
                if (t == 0) halpha[slot] = a;
                for (int q = t; q < nv; q += TP) vd[q] -= a * hy[slot * NK + q];
                __syncthreads();
            }
            for (int q = t; q < nv; q += TP) vd[q] *= gamma;
            __syncthreads();
            for (int i = hist - 1; i >= 0; --i) {
                const int slot = (head - 1 - i + LBFGS_M) % LBFGS_M;
                const double b = hrho[slot] * block_dot<R, TP>(sh, hy + slot * NK, vd, nv);
                const double a = halpha[slot];
                for (int q = t; q < nv; q += TP) vd[q] += (a - b) * hs[slot * NK + q];
                __syncthreads();
            }
            for (int q = t; q < nv; q += TP) vd[q] = -vd[q];
            __syncthreads();
            double gd = block_dot<R, TP>(sh, vg, vd, nv);
            if (!(gd < 0.0)) {
                for (int q = t; q < nv; q += TP) vd[q] = -vg[q];
                __syncthreads();
                gd = -block_dot<R, TP>(sh, vg, vg, nv);
                hist = 0;
            }
            double step = 1.0;
            if (hist == 0) step = fmin(1.0, 1.0 / sqrt(-gd));
            bool ok = false;
            double Jt = 0.0;
            for (int ls = 0; ls < 30; ++ls) {
                for (int q = t; q < nv; q += TP) vxt[q] = vx[q] + step * vd[q];
                __syncthreads();
                set_lambda(vxt);
                Jt = forward_ck<R, C, TP, S, NZ>(A, sh, noise, start, n0, Ns, ck, ckp, laml, io.y, s0, c0, f, iters,
                                                 flags, dWl, one ? seg : nullptr);
                if (Jt <= J + 1e-4 * step * gd) {
                    ok = true;
                    break;
                }
                step *= 0.5;
            }
            if (!ok) {
                set_lambda(vx);
                break;
            }
            backward_ck<R, C, TP, S, double*, double*, NZ>(A, sh, noise, n0, Ns, ck, ckp, seg, laml, io.y, s0, c0, s1,
                                                           c1, f, v0, v1, red, vgt, (double*)nullptr, gm, iters, flags,
                                                           dWl, one);
            __syncthreads();
            // history update s = xt - x, y = gt - g
            for (int q = t; q < nv; q += TP) {
                hs[head * NK + q] = vxt[q] - vx[q];
                hy[head * NK + q] = vgt[q] - vg[q];
            }
            __syncthreads();
            const double sy = block_dot<R, TP>(sh, hs + head * NK, hy + head * NK, nv);
            const double yy = block_dot<R, TP>(sh, hy + head * NK, hy + head * NK, nv);
            if (sy > 1e-300 && yy > 0.0) {
                if (t == 0) hrho[head] = 1.0 / sy;
                gamma = sy / yy;
                head = (head + 1) % LBFGS_M;
                hist = min(hist + 1, LBFGS_M);
            }
            for (int q = t; q < nv; q += TP) {
                vx[q] = vxt[q];
                vg[q] = vgt[q];
            }
            J = Jt;
            lb_iters++;
            __syncthreads();
        }
        set_lambda(vx);
        Jlast = J;
        if (io.mode == NUDGE_SEQUENTIAL) {
            // reveal dW^n and advance the start state one step with (dW^n, lambda^n)
            const int nblk = (K + 3) >> 2;
            for (int q = t; q < nblk; q += TP) {
                R z[4];
                normal4<R>(io.seed, SCH_TAG_NUDGE, (uint64_t)q, (uint64_t)n0, (uint64_t)(io.particle0 + p), io.ctr, z);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (4 * q + e < K) dWl[n0 * K + 4 * q + e] = (R)sqrt(A.dt_d) * z[e];
            }
            __syncthreads();
            Field<R, C> h;
            if constexpr (NZ == SCH_NOISE_MATERN) {
                field_start<R, C, TP>(A, sh, start, h);
                matern_stage_step<R, C>(A, noise, dWl, laml, n0);
                step_any<S, R, C, TP, NZ>(A, sh, h, noise, s0, c0, iters, flags);
            } else {
                stage_noise(A, noise, dWl, laml, Ns);
                field_start<R, C, TP>(A, sh, start, h);
                step_any<S, R, C, TP>(A, sh, h, noise + n0 * K, s0, c0, iters, flags);
            }
            __syncthreads();
            store_field<R, C>(start, h.m);
            __syncthreads();
        }
    }
    if (io.mode == NUDGE_OPEN_LOOP) {
        const int nblk = (K + 3) >> 2;
        for (int q = t; q < Ns * nblk; q += TP) {
            const int s = q / nblk, b = q % nblk;
            R z[4];
            normal4<R>(io.seed, SCH_TAG_NUDGE, (uint64_t)b, (uint64_t)s, (uint64_t)(io.particle0 + p), io.ctr, z);
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (4 * b + e < K) dWl[s * K + 4 * b + e] = (R)sqrt(A.dt_d) * z[e];
        }
        __syncthreads();
    }
    for (int q = t; q < NK; q += TP) {
        lam_out[q] = laml[q];
        dW_out[q] = dWl[q];
    }
    if (t == 0) {
        io.J[p] = Jlast;
        if (io.iters) io.iters[p] = lb_iters;
        if (io.status) io.status[p] = flags;
    }
}

template <typename R, int C, int TP>
struct LaunchAdj {
    template <int S>
    static int adjoint(const ModelArgs<R>& A, const AdjointIO<R>& io, int N, cudaStream_t st) {
        const size_t sm = adj_smem_bytes<R, TP>(io.Ns, A.K);
        if (sm > 48 * 1024)
            cudaFuncSetAttribute(adjoint_kernel<R, C, TP, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        adjoint_kernel<R, C, TP, S><<<N, TP, sm, st>>>(A, io);
        return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
    }
    template <int S>
    static int nudge(const ModelArgs<R>& A, const NudgeIO<R>& io, int N, cudaStream_t st) {
        const size_t sm = nudge_smem_bytes<R, TP>(io.Ns, A.K);
        if (sm > 48 * 1024)
            cudaFuncSetAttribute(nudge_kernel<R, C, TP, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        nudge_kernel<R, C, TP, S><<<N, TP, sm, st>>>(A, io);
        return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
    }
    // the Matern noise: the solver scratch and one step's n cell weights
    template <int S>
    static int adjoint_matern(const ModelArgs<R>& A, const AdjointIO<R>& io, int N, cudaStream_t st) {
        const size_t sm = shm_base_bytes<R, TP>() + (size_t)A.n * sizeof(R);
        if (sm > 48 * 1024)
            cudaFuncSetAttribute(adjoint_kernel<R, C, TP, S, SCH_NOISE_MATERN>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        adjoint_kernel<R, C, TP, S, SCH_NOISE_MATERN><<<N, TP, sm, st>>>(A, io);
        return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
    }
    template <int S>
    static int nudge_matern(const ModelArgs<R>& A, const NudgeIO<R>& io, int N, cudaStream_t st) {
        const size_t sm = shm_base_bytes<R, TP>() + (size_t)A.n * sizeof(R);
        if (sm > 48 * 1024)
            cudaFuncSetAttribute(nudge_kernel<R, C, TP, S, SCH_NOISE_MATERN>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        nudge_kernel<R, C, TP, S, SCH_NOISE_MATERN><<<N, TP, sm, st>>>(A, io);
        return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
    }
    static size_t adj_smem(int Ns, int K) { return adj_smem_bytes<R, TP>(Ns, K); }
    static size_t nudge_smem(int Ns, int K) { return nudge_smem_bytes<R, TP>(Ns, K); }
};

}  // namespace sch
