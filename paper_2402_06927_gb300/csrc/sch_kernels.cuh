// Ensemble propagation of the viscous stochastic Camassa-Holm (SALT) equation
// on sm_103a: one CTA of TP threads per particle, the periodic field held in
// registers across all steps of an assimilation window (and across all PCN
// proposals of a jitter call).
//
// Discretisation (Sec. 2 of the paper): P1 elements on n = C * TP uniform
// periodic cells, Helmholtz relation (M + alpha^2 K) u = M m (Eq. sde1), and
// the implicit midpoint step (Eq. fde1)
//   M (m1 - m0) + mu dt K mbar + A(mbar, dv) = 0,
//   mbar = (m0 + m1)/2,  dv = dt (u0 + u1)/2 + dU,
// with the exact P1 advection operator
//   A(m, v)_i = 1/2 [ v_{i+1} (m_i + m_{i+1}) - v_{i-1} (m_{i-1} + m_i) ].
// Each step is solved by linearly implicit Picard iteration: with dv frozen
// at the last iterate, the cyclic tridiagonal system
//   (M + mu dt/2 K + 1/2 A_dv) m1 = (M - mu dt/2 K - 1/2 A_dv) m0
// is solved, then u1 = H^{-1} M m1, until max|m1 - m1_prev| <= tol max(1, max|m1|).
//
// Solver layout.  Thread t owns nodes [tC, tC + C).  A cyclic tridiagonal
// system is solved by a partition method: each thread eliminates the interior
// of its chunk with a forward and a backward sweep, which leaves a "first"
// row F_t (coupling E_{t-1}, F_t, E_t) and a "last" row E_t (coupling F_t,
// E_t, F_{t+1}).  Warp 0 eliminates the F rows, solves the resulting cyclic
// system in the E_t (each lane sweeps TP/32 consecutive rows, then a cyclic
// parallel cyclic reduction over the 32 lanes with shuffles), and publishes
// E_t and F_t in shared memory; every thread then back-substitutes its
// interior.  One Picard iteration therefore costs four CTA barriers: before
// and after each of the two reduced solves (the variable Picard matrix and
// the constant Helmholtz matrix).  Chunk-end neighbours come from the
// published interface values, and the convergence decision rides on the
// Helmholtz reduced solve.
#pragma once

#include "sch_internal.h"

namespace sch {

// --------------------------------------------------------------------------
// shared memory of one particle CTA
// --------------------------------------------------------------------------
template <typename R, int TP>
struct Shm {
    static constexpr int RR = TP / 32 > 1 ? TP / 32 : 1;
    R pa[TP], pc[TP], pd[TP], ae[TP], ge[TP], de[TP];   // reduced rows of the Picard matrix
    R hpd[TP], hde[TP];                                  // reduced rows of a constant matrix
    R E[TP], F[TP];                                      // interface values, Picard matrix
    R hE[TP], hF[TP];                                    // interface values, constant matrix
    R sw[3 * RR * 32];                                   // warp-0 lane sweeps
    R wred[2][32];                                       // per-warp convergence maxima
    double dsum[2][32];                                  // per-warp double sums
    int flag;
};

template <typename R, int TP>
__host__ __device__ constexpr size_t shm_base_bytes() {
    return (sizeof(Shm<R, TP>) + 15) / 16 * 16;
}

enum { FLAG_CONVERGED = 1, FLAG_NONFINITE = 2, FLAG_STOP = 4, FLAG_NOCONV = 8 };

// --------------------------------------------------------------------------
// cyclic PCR over the 32 lanes of a warp (one row per lane)
// --------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R shfl_pcr32(R A, R B, R Cc, R D) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 1; s < 16; s <<= 1) {
        const R rb = rcp(B);
        const int lo = (lane - s) & 31, hi = (lane + s) & 31;
        const R Am = __shfl_sync(FULL, A, lo), Cm = __shfl_sync(FULL, Cc, lo);
        const R Dm = __shfl_sync(FULL, D, lo), rbm = __shfl_sync(FULL, rb, lo);
        const R Ap = __shfl_sync(FULL, A, hi), Cp = __shfl_sync(FULL, Cc, hi);
        const R Dp = __shfl_sync(FULL, D, hi), rbp = __shfl_sync(FULL, rb, hi);
        const R k1 = A * rbm, k2 = Cc * rbp;
        const R nB = B - Cm * k1 - Ap * k2;
        D = D - Dm * k1 - Dp * k2;
        A = -Am * k1;
        Cc = -Cp * k2;
        B = nB;
    }
    // stride 16: both neighbours are lane ^ 16; close with a 2x2 solve
    const R e = A + Cc;
    const int j = lane ^ 16;
    const R ej = __shfl_sync(FULL, e, j), Bj = __shfl_sync(FULL, B, j), Dj = __shfl_sync(FULL, D, j);
    return (D * Bj - e * Dj) / (B * Bj - e * ej);
}

// --------------------------------------------------------------------------
// Warp 0: solve the cyclic system of TP interface rows
//   A_t E_{t-1} + B_t E_t + C_t E_{t+1} = D_t,    row(t, A, B, C, D)
// and store E_t.  Lane l owns rows [l RR, (l+1) RR).
// --------------------------------------------------------------------------
template <typename R, int TP, typename RowFn>
__device__ __forceinline__ void warp_cyclic_solve(RowFn row, R* E, R* sw) {
    constexpr int RR = TP / 32;
    const int lane = threadIdx.x & 31;
    const int t0 = lane * RR;
    if constexpr (RR == 1) {
        R A, B, Cc, D;
        row(t0, A, B, Cc, D);
        E[t0] = shfl_pcr32(A, B, Cc, D);
    } else {
        R* sal = sw;
        R* sga = sw + RR * 32;
        R* sdl = sw + 2 * RR * 32;
        R A0, B0, C0, D0;
        row(t0, A0, B0, C0, D0);
        R al = R(-1), ga = R(0), dl = R(0);
#pragma unroll
        for (int r = 1; r < RR; ++r) {
            R A, B, Cc, D;
            row(t0 + r, A, B, Cc, D);
            const R q = rcp(B - A * ga);
            ga = Cc * q;
            al = -A * al * q;
            dl = (D - A * dl) * q;
            sal[r * 32 + lane] = al;
            sga[r * 32 + lane] = ga;
            sdl[r * 32 + lane] = dl;
        }
        const R aeL = al, geL = ga, deL = dl;
        R dp = R(0), ap = R(0), gp = R(-1);
#pragma unroll
        for (int r = RR - 2; r >= 1; --r) {
            const R g = sga[r * 32 + lane];
            dp = sdl[r * 32 + lane] - g * dp;
            ap = sal[r * 32 + lane] - g * ap;
            gp = -g * gp;
            sal[r * 32 + lane] = ap;
            sga[r * 32 + lane] = gp;
            sdl[r * 32 + lane] = dp;
        }
        R BF, CF, DF;
        if (RR == 2) {
            BF = B0; CF = C0; DF = D0;
        } else {
            BF = B0 - C0 * ap; CF = -C0 * gp; DF = D0 - C0 * dp;
        }
        const R qi = rcp(BF);
        const R qa = A0 * qi, qc = CF * qi, qd = DF * qi;
        const int nx = (lane + 1) & 31;
        const R nqa = __shfl_sync(FULL, qa, nx), nqc = __shfl_sync(FULL, qc, nx), nqd = __shfl_sync(FULL, qd, nx);
        const R LA = -aeL * qa;
        const R LB = R(1) - aeL * qc - geL * nqa;
        const R LC = -geL * nqc;
        const R LD = deL - aeL * qd - geL * nqd;
        const R EL = shfl_pcr32(LA, LB, LC, LD);
        const R Ep = __shfl_sync(FULL, EL, (lane + 31) & 31);
        const R Ff = qd - qa * Ep - qc * EL;
        E[t0] = Ff;
        E[t0 + RR - 1] = EL;
#pragma unroll
        for (int r = 1; r < RR - 1; ++r)
            E[t0 + r] = sdl[r * 32 + lane] - sal[r * 32 + lane] * Ff - sga[r * 32 + lane] * EL;
    }
    __syncwarp();
}

// Warp 0: reduced solve of the Picard matrix, then F_t = pd_t - pa_t E_{t-1} - pc_t E_t.
template <typename R, int TP>
__device__ __forceinline__ void warp_reduce_var(Shm<R, TP>* sh) {
    auto row = [sh](int t, R& A, R& B, R& Cc, R& D) {
        const int tn = (t + 1) & (TP - 1);
        const R ae = sh->ae[t], ge = sh->ge[t];
        A = -ae * sh->pa[t];
        B = R(1) - ae * sh->pc[t] - ge * sh->pa[tn];
        Cc = -ge * sh->pc[tn];
        D = sh->de[t] - ae * sh->pd[t] - ge * sh->pd[tn];
    };
    warp_cyclic_solve<R, TP>(row, sh->E, sh->sw);
    constexpr int RR = Shm<R, TP>::RR;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < RR; ++r) {
        const int t = lane * RR + r;
        if (t < TP) sh->F[t] = sh->pd[t] - sh->pa[t] * sh->E[(t - 1) & (TP - 1)] - sh->pc[t] * sh->E[t];
    }
}

// cyclic PCR over 32 lanes for a constant reduced system: only D travels
template <typename R>
__device__ __forceinline__ R pcr32_const(R D, const RTab<R>& Q) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const int s = 1 << l;
        const R Dm = __shfl_sync(FULL, D, (lane - s) & 31);
        const R Dp = __shfl_sync(FULL, D, (lane + s) & 31);
        D = D - Q.k1[l] * Dm - Q.k2[l] * Dp;
    }
    const R Dj = __shfl_sync(FULL, D, lane ^ 16);
    return Q.f1 * D + Q.f2 * Dj;
}

// Warp 0, registers only: interface values of a tabulated constant matrix.
// Lane l holds the reduced-row inputs pd, de of rows t = l RR + r (RR = TP/32)
// and gets back E_t and F_t = pd_t - pa E_{t-1} - pc E_t.  Rows read
// D_t = de_t - ae pd_t - ge pd_{t+1} (A, B, C fixed); the next row's pd and the
// previous row's E cross lanes by shuffle.  T: any table with the reduced-row
// couplings ae, ge, pa, pc; Eprev_out, if given, receives E_{l RR - 1}.
template <typename R, int TP, typename Tab>
__device__ __forceinline__ void lane_solve_const(const Tab& T, const RTab<R>& Q, const R (&pd)[TP / 32],
                                                 const R (&de)[TP / 32], R (&E)[TP / 32], R (&F)[TP / 32],
                                                 R* Eprev_out = nullptr) {
    constexpr int RR = TP / 32;
    const int lane = threadIdx.x & 31;
    const R pd_next = __shfl_sync(FULL, pd[0], (lane + 1) & 31);
    R D[RR];
#pragma unroll
    for (int r = 0; r < RR; ++r) {
        const R pn = (r == RR - 1) ? pd_next : pd[(r + 1) % RR];
        D[r] = de[r] - T.ae * pd[r] - T.ge * pn;
    }
    if constexpr (RR == 1) {
        E[0] = pcr32_const(D[0], Q);
    } else {
        R dl[RR];
        dl[0] = R(0);
#pragma unroll
        for (int r = 1; r < RR; ++r) dl[r] = (D[r] - Q.A * dl[r - 1]) * Q.q[r];
        R dp[RR];
        dp[RR - 1] = R(0);
        dp[0] = R(0);
#pragma unroll
        for (int r = RR - 2; r >= 1; --r) dp[r] = dl[r] - Q.ga[r] * dp[r + 1];
        const R DF = (RR == 2) ? D[0] : D[0] - Q.Cc * dp[1];
        const R qd = DF * Q.iBF;
        const R nqd = __shfl_sync(FULL, qd, (lane + 1) & 31);
        const R LD = dl[RR - 1] - Q.aeL * qd - Q.geL * nqd;
        const R EL = pcr32_const(LD, Q);
        const R Ep = __shfl_sync(FULL, EL, (lane + 31) & 31);
        const R Ff = qd - Q.qa * Ep - Q.qc * EL;
        E[0] = Ff;
#pragma unroll
        for (int r = 1; r < RR - 1; ++r) E[r] = dp[r] - Q.alp[r] * Ff - Q.gap[r] * EL;
        E[RR - 1] = EL;
    }
    const R Eprev = __shfl_sync(FULL, E[RR - 1], (lane + 31) & 31);
#pragma unroll
    for (int r = 0; r < RR; ++r) {
        const R em1 = (r == 0) ? Eprev : E[(r + RR - 1) % RR];
        F[r] = pd[r] - T.pa * em1 - T.pc * E[r];
    }
    if (Eprev_out) *Eprev_out = Eprev;
}

// Warp 0: the same from shared-memory rows pd[t], de[t] into E[t], F[t].
template <typename R, int TP>
__device__ __forceinline__ void warp_solve_const(const CTab<R>& T, const RTab<R>& Q, const R* pd, const R* de,
                                                 R* E, R* F) {
    constexpr int RR = TP / 32;
    const int t0 = (threadIdx.x & 31) * RR;
    R p[RR], d[RR], e[RR], f[RR];
#pragma unroll
    for (int r = 0; r < RR; ++r) {
        p[r] = pd[t0 + r];
        d[r] = de[t0 + r];
    }
    lane_solve_const<R, TP>(T, Q, p, d, e, f);
#pragma unroll
    for (int r = 0; r < RR; ++r) {
        E[t0 + r] = e[r];
        F[t0 + r] = f[r];
    }
    __syncwarp();
}

// --------------------------------------------------------------------------
// constant matrix: local sweep (writes hpd/hde) and back substitution
// --------------------------------------------------------------------------
template <typename R, int C, int TP>
__device__ __forceinline__ void const_local(const CTab<R>& T, const R (&r)[C], R (&dp)[C], Shm<R, TP>* sh) {
    const R a = T.a;
    R de[C];
    de[0] = R(0);
#pragma unroll
    for (int i = 1; i < C; ++i) de[i] = (r[i] - a * de[i - 1]) * T.rden[i];
    dp[C - 1] = R(0);
#pragma unroll
    for (int i = C - 2; i >= 1; --i) dp[i] = de[i] - T.gam[i] * dp[i + 1];
    const R DF = (C == 2) ? r[0] : r[0] - a * dp[1];
    sh->hpd[threadIdx.x] = DF * T.iBF;
    sh->hde[threadIdx.x] = de[C - 1];
}

template <typename R, int C>
__device__ __forceinline__ void const_back(const CTab<R>& T, const R (&dp)[C], R F, R E, R (&x)[C]) {
    x[0] = F;
    x[C - 1] = E;
#pragma unroll
    for (int i = 1; i < C - 1; ++i) x[i] = dp[i] - T.alpp[i] * F - T.gamp[i] * E;
}

// Full solve of a tabulated constant matrix for right-hand side r: returns x
// and its chunk-end neighbours xp (= x_{tC-1}) and xn (= x_{tC+C}).
template <typename R, int C, int TP>
__device__ __forceinline__ void const_solve(const CTab<R>& T, const RTab<R>& Q, const R (&r)[C], R (&x)[C], R& xp,
                                            R& xn, Shm<R, TP>* sh) {
    R dp[C];
    const_local<R, C, TP>(T, r, dp, sh);
    __syncthreads();
    if (threadIdx.x < 32) warp_solve_const<R, TP>(T, Q, sh->hpd, sh->hde, sh->hE, sh->hF);
    __syncthreads();
    const int t = threadIdx.x;
    const R F = sh->hF[t], E = sh->hE[t];
    xp = sh->hE[(t - 1) & (TP - 1)];
    xn = sh->hF[(t + 1) & (TP - 1)];
    const_back<R, C>(T, dp, F, E, x);
}

// neighbours of a chunk (prev thread's last, next thread's first), through E/F
template <typename R, int C, int TP>
__device__ __forceinline__ void chunk_halo(const R (&v)[C], R& vp, R& vn, Shm<R, TP>* sh) {
    const int t = threadIdx.x;
    sh->E[t] = v[C - 1];
    sh->F[t] = v[0];
    __syncthreads();
    vp = sh->E[(t - 1) & (TP - 1)];
    vn = sh->F[(t + 1) & (TP - 1)];
    __syncthreads();
}

// M v for the P1 mass matrix, h/6 (v_{i-1} + 4 v_i + v_{i+1})
template <typename R, int C>
__device__ __forceinline__ void mass_apply(R h6, const R (&v)[C], R vp, R vn, R (&r)[C]) {
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const R lo = (i == 0) ? vp : v[i - 1];
        const R hi = (i == C - 1) ? vn : v[i + 1];
        r[i] = h6 * (lo + R(4) * v[i] + hi);
    }
}

// SALT increment dU/4 at the C + 2 nodes i0 - 1 .. i0 + C of this thread's
// chunk, from the step's K weights wq_k = a_j/4 (dW_k + lambda_k dt):
// dU_i / 4 = sum_j wq_{2j-2} sin(j theta_i) + wq_{2j-1} cos(j theta_i).
// (sin, cos)(j theta_{i0-1}) follow a Chebyshev recurrence over j; along the
// chunk each harmonic is rotated by its tabulated angle j 2 pi / n.  Each weight
// is read once per step.
template <typename R, int C>
__device__ __forceinline__ void noise_nodes(const ModelArgs<R>& A, const R* wq, R s0, R c0, R (&nq)[C + 2]) {
#pragma unroll
    for (int q = 0; q < C + 2; ++q) nq[q] = R(0);
    const R twoc = R(2) * c0;
    R sj = s0, cj = c0, sjm = R(0), cjm = R(1);
    for (int j = 0; j < A.K2; ++j) {
        const R a = wq[2 * j], b = wq[2 * j + 1];
        const R rc = A.rot_c[j], rs = A.rot_s[j];
        R sn = sj, cs = cj;
#pragma unroll
        for (int q = 0; q < C + 2; ++q) {
            nq[q] += a * sn + b * cs;
            const R s2 = sn * rc + cs * rs;
            cs = cs * rc - sn * rs;
            sn = s2;
        }
        const R sn2 = twoc * sj - sjm, cn2 = twoc * cj - cjm;
        sjm = sj;
        cjm = cj;
        sj = sn2;
        cj = cn2;
    }
}

// sin and cos of the angle 2 pi i / n of node i (taken mod n)
template <typename R>
__device__ __forceinline__ void node_angle(int node, int n, R& s, R& c) {
    const int i = (node + n) % n;
    sincospi(R(2) * R(i) / R(n), &s, &c);
}

// Matern SALT increment dU/4 at the C + 2 nodes i0 - 1 .. i0 + C (Eq. noise_solve2):
// wq holds the step's n cell weights eta sqrt(h)/8 (dW_c + lambda_c dt), so the
// load eta (dW_h, phi_i) / 4 is wq_{i-1} + wq_i; then mk solves with the
// tabulated G = M + kappa^-2 K, each later one loaded with M U_{j-1}.
template <typename R, int C, int TP>
__device__ __forceinline__ void matern_nodes(const ModelArgs<R>& A, Shm<R, TP>* sh, const R* wq, R (&nq)[C + 2]) {
    const int i0 = threadIdx.x * C;
    R r[C], U[C], Up, Un;
    r[0] = wq[i0 == 0 ? A.n - 1 : i0 - 1] + wq[i0];
#pragma unroll
    for (int i = 1; i < C; ++i) r[i] = wq[i0 + i - 1] + wq[i0 + i];
    const_solve<R, C, TP>(A.matern, A.rmatern, r, U, Up, Un, sh);
    for (int j = 1; j < A.mk; ++j) {
        mass_apply<R, C>(A.h6, U, Up, Un, r);
        const_solve<R, C, TP>(A.matern, A.rmatern, r, U, Up, Un, sh);
    }
    nq[0] = Up;
#pragma unroll
    for (int i = 0; i < C; ++i) nq[i + 1] = U[i];
    nq[C + 1] = Un;
}

// the step's noise at the chunk's nodes and its two neighbours, for noise model NZ
template <int NZ, typename R, int C, int TP>
__device__ __forceinline__ void noise_any(const ModelArgs<R>& A, Shm<R, TP>* sh, const R* wq, R s0, R c0,
                                          R (&nq)[C + 2]) {
    if constexpr (NZ == SCH_NOISE_MATERN)
        matern_nodes<R, C, TP>(A, sh, wq, nq);
    else
        noise_nodes<R, C>(A, wq, s0, c0, nq);
}

// --------------------------------------------------------------------------
// the per-thread state carried through a window
// --------------------------------------------------------------------------
template <typename R, int C>
struct Field {
    R m[C], u[C];
    R mp, mn, up, un;   // chunk-end neighbours of m and u
};

// --------------------------------------------------------------------------
// One implicit-midpoint step (Eq. fde1) for this thread's chunk.
// wq: the K noise weights of the step, scaled by a_j / 4.
// --------------------------------------------------------------------------
template <typename R, int C, int TP, int NZ = SCH_NOISE_MODES>
__device__ __forceinline__ void sch_step(const ModelArgs<R>& A, Shm<R, TP>* sh, Field<R, C>& f, const R* wq,
                                         R s0, R c0, int& iters, int& flags) {
    const int t = threadIdx.x;
    // W0 = dt/8 u0 + dU/4, at the chunk and its two neighbour nodes
    R nq[C + 2];
    noise_any<NZ, R, C, TP>(A, sh, wq, s0, c0, nq);
    R W0[C];
#pragma unroll
    for (int i = 0; i < C; ++i) W0[i] = A.dt8 * f.u[i] + nq[i + 1];
    const R W0p = A.dt8 * f.up + nq[0];
    const R W0n = A.dt8 * f.un + nq[C + 1];
    // from m0: S_i = m_i + m_{i+1}, D0_i = c0p (m_{i-1} + m_{i+1}) + b0p m_i
    R Ssum[C], D0[C];
    const R Sprev = f.mp + f.m[0];
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const R lo = (i == 0) ? f.mp : f.m[i - 1];
        const R hi = (i == C - 1) ? f.mn : f.m[i + 1];
        Ssum[i] = f.m[i] + hi;
        D0[i] = A.c0p * (lo + hi) + A.b0p * f.m[i];
    }
    // iterates (m, u) and the u neighbours
    R mi[C], ui[C];
    R uip = f.up, uin = f.un, mip = f.mp, min_ = f.mn;
#pragma unroll
    for (int i = 0; i < C; ++i) { mi[i] = f.m[i]; ui[i] = f.u[i]; }

    for (int it = 1; it <= A.max_iter; ++it) {
        // w = dv / 4 at the current iterate
        R w[C];
#pragma unroll
        for (int i = 0; i < C; ++i) w[i] = W0[i] + A.dt8 * ui[i];
        const R wp = W0p + A.dt8 * uip;
        const R wn = W0n + A.dt8 * uin;
        // rows: a_i = c0 - w_{i-1}, c_i = c0 + w_{i+1}, b_i = b0 + w_{i+1} - w_{i-1},
        //       d_i = D0_i + w_{i-1} S_{i-1} - w_{i+1} S_i ; forward sweep of rows 1..C-1
        R al[C], ga[C], de[C];
        const R a0 = A.c0 - wp;
        const R wr0 = (C > 1) ? w[1] : wn;
        const R c0 = A.c0 + wr0;
        const R b0 = A.b0 + wr0 - wp;
        const R d0 = D0[0] + wp * Sprev - wr0 * Ssum[0];
        al[0] = R(-1);
        ga[0] = R(0);
        de[0] = R(0);
#pragma unroll
        for (int i = 1; i < C; ++i) {
            const R wl = w[i - 1];
            const R wr = (i == C - 1) ? wn : w[i + 1];
            const R ai = A.c0 - wl;
            const R ci = A.c0 + wr;
            const R bi = A.b0 + wr - wl;
            const R di = D0[i] + wl * Ssum[i - 1] - wr * Ssum[i];
            const R q = rcp(bi - ai * ga[i - 1]);
            ga[i] = ci * q;
            al[i] = -ai * al[i - 1] * q;
            de[i] = (di - ai * de[i - 1]) * q;
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
            BF = b0; CF = c0; DF = d0;
        } else {
            BF = b0 - c0 * al[1];
            CF = -c0 * ga[1];
            DF = d0 - c0 * de[1];
        }
        const R qF = rcp(BF);
        sh->pa[t] = a0 * qF;
        sh->pc[t] = CF * qF;
        sh->pd[t] = DF * qF;
        __syncthreads();                                             // B1
        if (t < 32) warp_reduce_var<R, TP>(sh);
        __syncthreads();                                             // B2
        const R E = sh->E[t], F = sh->F[t];
        const R Ep = sh->E[(t - 1) & (TP - 1)], Fn = sh->F[(t + 1) & (TP - 1)];
        R mnew[C];
        mnew[0] = F;
        mnew[C - 1] = E;
#pragma unroll
        for (int i = 1; i < C - 1; ++i) mnew[i] = de[i] - al[i] * F - ga[i] * E;
        // convergence maxima of this warp
        R dmax = R(0), mmax = R(0);
#pragma unroll
        for (int i = 0; i < C; ++i) {
            R dd = rabs(mnew[i] - mi[i]);
            if (!(dd == dd)) dd = R(INFINITY);
            dmax = fmax(dmax, dd);
            mmax = fmax(mmax, rabs(mnew[i]));
        }
        dmax = warp_max(dmax);
        mmax = warp_max(mmax);
        if ((t & 31) == 0) {
            sh->wred[0][t >> 5] = dmax;
            sh->wred[1][t >> 5] = mmax;
        }
        // Helmholtz for the new iterate: r = M m, local sweep
        R r[C], dpH[C];
        mass_apply<R, C>(A.h6, mnew, Ep, Fn, r);
        const_local<R, C, TP>(A.hel, r, dpH, sh);
        __syncthreads();                                             // B3
        if (t < 32) {
            warp_solve_const<R, TP>(A.hel, A.rhel, sh->hpd, sh->hde, sh->hE, sh->hF);
            constexpr int NW = TP / 32;
            R dm = (t < NW) ? sh->wred[0][t] : R(0);
            R mm = (t < NW) ? sh->wred[1][t] : R(0);
            dm = warp_max(dm);
            mm = warp_max(mm);
            if (t == 0) {
                int fl = 0;
                if (!(dm < R(INFINITY)) || !(mm < R(INFINITY))) fl = FLAG_NONFINITE;
                else if (dm <= A.tol * fmax(R(1), mm)) fl = FLAG_CONVERGED;
                sh->flag = fl;
            }
        }
        __syncthreads();                                             // B4
        const R hF = sh->hF[t], hE = sh->hE[t];
        uip = sh->hE[(t - 1) & (TP - 1)];
        uin = sh->hF[(t + 1) & (TP - 1)];
        const_back<R, C>(A.hel, dpH, hF, hE, ui);
#pragma unroll
        for (int i = 0; i < C; ++i) mi[i] = mnew[i];
        mip = Ep;
        min_ = Fn;
        iters++;
        const int fl = sh->flag;
        if (fl & FLAG_NONFINITE) {
            flags |= SCH_DEV_NONFINITE;
            break;
        }
        if (fl & FLAG_CONVERGED) break;
        if (it == A.max_iter) flags |= SCH_DEV_NOCONVERGE;
    }
#pragma unroll
    for (int i = 0; i < C; ++i) { f.m[i] = mi[i]; f.u[i] = ui[i]; }
    f.mp = mip;
    f.mn = min_;
    f.up = uip;
    f.un = uin;
}

// Stop test of the explicit-advection Picard iteration after a step of size dm
// (max-norm of the change of the iterate) against lim = tol max(1, max|m|).  It
// stops when dm <= lim.  In FP32 it also stops when the contraction seen over the
// last two steps (dm_prev is infinite before the second), rho = dm / dm_prev < 1/2,
// puts the error of the current iterate,
// at most about rho dm / (1 - rho), below lim: that saves the iteration whose only
// purpose would be to confirm it (the iteration contracts by about 0.05 per
// iteration, so the plain test stops about one iteration past the tolerance, with
// the error already near float rounding).  FP64 keeps the plain test.
template <typename R>
__device__ __forceinline__ bool ea_converged(R dm, R dm_prev, R lim) {
    if (dm <= lim) return true;
    if constexpr (sizeof(R) == 4) {
        // rho < 1/2 and rho dm <= lim (1 - rho), multiplied through by dm_prev > 0
        return dm_prev < R(INFINITY) && R(2) * dm < dm_prev && dm * dm <= lim * (dm_prev - dm);
    }
    return false;
}

// --------------------------------------------------------------------------
// One implicit-midpoint step by explicit-advection Picard iteration:
//   (M + mu dt/2 K) m^{p+1} = (M - mu dt/2 K) m0 - A(mbar^p, dv^p),
//   u^{p+1} = H^{-1} M m^{p+1}.
// Both matrices are constant, so warp 0 can build the Helmholtz interface rows
// from the Picard interface values with host-tabulated functionals and solve
// both reduced systems between one pair of barriers.  The convergence test of
// iterate p is decided at the first barrier of iteration p + 1 (whose local
// work is then discarded), so an iteration costs two barriers.
// --------------------------------------------------------------------------
template <typename R, int C, int TP, int NZ = SCH_NOISE_MODES>
__device__ __forceinline__ void sch_step_ea(const ModelArgs<R>& A, Shm<R, TP>* sh, Field<R, C>& f, const R* wq,
                                            R s0, R c0, int& iters, int& flags) {
    constexpr int RR = TP / 32;
    const int t = threadIdx.x;
    R nq[C + 2];
    noise_any<NZ, R, C, TP>(A, sh, wq, s0, c0, nq);
    // W0 = dt/8 u0 + dU/4, so that dv/4 = W0 + dt/8 u at an iterate
    R W0[C];
#pragma unroll
    for (int i = 0; i < C; ++i) W0[i] = A.dt8 * f.u[i] + nq[i + 1];
    const R W0p = A.dt8 * f.up + nq[0];
    const R W0n = A.dt8 * f.un + nq[C + 1];
    // R0 = (M - mu dt/2 K) m0
    R R0[C];
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const R lo = (i == 0) ? f.mp : f.m[i - 1];
        const R hi = (i == C - 1) ? f.mn : f.m[i + 1];
        R0[i] = A.c0p * (lo + hi) + A.b0p * f.m[i];
    }
    R mi[C], ui[C];
#pragma unroll
    for (int i = 0; i < C; ++i) { mi[i] = f.m[i]; ui[i] = f.u[i]; }
    R mip = f.mp, min_ = f.mn, uip = f.up, uin = f.un;
    const R m0p = f.mp, m0n = f.mn;
    R dm_prev = R(INFINITY);   // warp 0: the step size of the previous test

    for (int it = 1;; ++it) {
        // local phase: right-hand side and chunk sweep of M + mu dt/2 K
        R rhs[C];
        {
            R w[C], mb[C];
#pragma unroll
            for (int i = 0; i < C; ++i) {
                w[i] = W0[i] + A.dt8 * ui[i];
                mb[i] = R(0.5) * (f.m[i] + mi[i]);
            }
            const R wp = W0p + A.dt8 * uip, wn = W0n + A.dt8 * uin;
            const R mbp = R(0.5) * (m0p + mip), mbn = R(0.5) * (m0n + min_);
#pragma unroll
            for (int i = 0; i < C; ++i) {
                const R wl = (i == 0) ? wp : w[i - 1];
                const R wr = (i == C - 1) ? wn : w[i + 1];
                const R ml = (i == 0) ? mbp : mb[i - 1];
                const R mr = (i == C - 1) ? mbn : mb[i + 1];
                // A(mbar, dv)_i = 1/2 [dv_{i+1} (mbar_i + mbar_{i+1}) - dv_{i-1} (mbar_{i-1} + mbar_i)]
                rhs[i] = R0[i] - R(2) * (wr * (mb[i] + mr) - wl * (ml + mb[i]));
            }
        }
        R dp[C];
        R de_last, DF;
        {
            R de[C];
            de[0] = R(0);
#pragma unroll
            for (int i = 1; i < C; ++i) de[i] = (rhs[i] - A.pic.a * de[i - 1]) * A.pic.rden[i];
            dp[0] = R(0);
            dp[C - 1] = R(0);
#pragma unroll
            for (int i = C - 2; i >= 1; --i) dp[i] = de[i] - A.pic.gam[i] * dp[i + 1];
            de_last = de[C - 1];
            DF = (C == 2) ? rhs[0] : rhs[0] - A.pic.a * dp[1];
        }
        R hpl = R(0), hdl = R(0);
#pragma unroll
        for (int i = 1; i < C - 1; ++i) {
            hpl += A.hb.apd[i] * dp[i];
            hdl += A.hb.ade[i] * dp[i];
        }
        sh->pd[t] = DF * A.pic.iBF;
        sh->de[t] = de_last;
        sh->hpd[t] = hpl;
        sh->hde[t] = hdl;
        __syncthreads();                                             // B1
        if (t < 32) {
            int fl = 0;
            if (it > 1) {
                constexpr int NW = TP / 32;
                R dm = (t < NW) ? sh->wred[0][t] : R(0);
                R mm = (t < NW) ? sh->wred[1][t] : R(0);
                dm = warp_max(dm);
                mm = warp_max(mm);
                if (!(dm < R(INFINITY)) || !(mm < R(INFINITY))) fl = FLAG_STOP | FLAG_NONFINITE;
                else if (ea_converged(dm, dm_prev, A.tol * fmax(R(1), mm))) fl = FLAG_STOP | FLAG_CONVERGED;
                else if (it > A.max_iter) fl = FLAG_STOP | FLAG_NOCONV;
                dm_prev = dm;
            }
            if (!(fl & FLAG_STOP)) {
                R pdr[RR], der[RR], hpr[RR], hdr[RR], Er[RR], Fr[RR];
#pragma unroll
                for (int r = 0; r < RR; ++r) {
                    const int q = t * RR + r;
                    pdr[r] = sh->pd[q];
                    der[r] = sh->de[q];
                    hpr[r] = sh->hpd[q];
                    hdr[r] = sh->hde[q];
                }
                lane_solve_const<R, TP>(A.pic, A.rpic, pdr, der, Er, Fr);
                // Helmholtz rows from the Picard interface values
                const R Ep = __shfl_sync(FULL, Er[RR - 1], (t + 31) & 31);
                const R Fn = __shfl_sync(FULL, Fr[0], (t + 1) & 31);
#pragma unroll
                for (int r = 0; r < RR; ++r) {
                    const R em1 = (r == 0) ? Ep : Er[(r + RR - 1) % RR];
                    const R fp1 = (r == RR - 1) ? Fn : Fr[(r + 1) % RR];
                    hpr[r] += A.hb.cpF * Fr[r] + A.hb.cpE * Er[r] + A.hb.cpEp * em1 + A.hb.cpFn * fp1;
                    hdr[r] += A.hb.cdF * Fr[r] + A.hb.cdE * Er[r] + A.hb.cdEp * em1 + A.hb.cdFn * fp1;
                }
                R hEr[RR], hFr[RR];
                lane_solve_const<R, TP>(A.hel, A.rhel, hpr, hdr, hEr, hFr);
#pragma unroll
                for (int r = 0; r < RR; ++r) {
                    const int q = t * RR + r;
                    sh->E[q] = Er[r];
                    sh->F[q] = Fr[r];
                    sh->hE[q] = hEr[r];
                    sh->hF[q] = hFr[r];
                }
            }
            if (t == 0) sh->flag = fl;
        }
        __syncthreads();                                             // B2
        const int fl = sh->flag;
        if (fl & FLAG_STOP) {
            if (fl & FLAG_NONFINITE) flags |= SCH_DEV_NONFINITE;
            if (fl & FLAG_NOCONV) flags |= SCH_DEV_NOCONVERGE;
            break;
        }
        // back phase: the new iterate (m, u) of this chunk
        const R E = sh->E[t], F = sh->F[t];
        const R Ep = sh->E[(t - 1) & (TP - 1)], Fn = sh->F[(t + 1) & (TP - 1)];
        R mnew[C];
        mnew[0] = F;
        mnew[C - 1] = E;
#pragma unroll
        for (int i = 1; i < C - 1; ++i) mnew[i] = dp[i] - A.pic.alpp[i] * F - A.pic.gamp[i] * E;
        R r[C];
        mass_apply<R, C>(A.h6, mnew, Ep, Fn, r);
        R hd[C];
        hd[0] = R(0);
#pragma unroll
        for (int i = 1; i < C; ++i) hd[i] = (r[i] - A.hel.a * hd[i - 1]) * A.hel.rden[i];
        R hdp[C];
        hdp[C - 1] = R(0);
#pragma unroll
        for (int i = C - 2; i >= 1; --i) hdp[i] = hd[i] - A.hel.gam[i] * hdp[i + 1];
        const R hF = sh->hF[t], hE = sh->hE[t];
        R dmax = R(0), mmax = R(0);
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const R un = (i == 0) ? hF : (i == C - 1 ? hE : hdp[i] - A.hel.alpp[i] * hF - A.hel.gamp[i] * hE);
            R dd = rabs(mnew[i] - mi[i]);
            if (!(dd == dd)) dd = R(INFINITY);
            dmax = fmax(dmax, dd);
            mmax = fmax(mmax, rabs(mnew[i]));
            mi[i] = mnew[i];
            ui[i] = un;
        }
        dmax = warp_max(dmax);
        mmax = warp_max(mmax);
        if ((t & 31) == 0) {
            sh->wred[0][t >> 5] = dmax;
            sh->wred[1][t >> 5] = mmax;
        }
        mip = Ep;
        min_ = Fn;
        uip = sh->hE[(t - 1) & (TP - 1)];
        uin = sh->hF[(t + 1) & (TP - 1)];
        iters++;
    }
#pragma unroll
    for (int i = 0; i < C; ++i) { f.m[i] = mi[i]; f.u[i] = ui[i]; }
    f.mp = mip;
    f.mn = min_;
    f.up = uip;
    f.un = uin;
}

template <int S, typename R, int C, int TP, int NZ = SCH_NOISE_MODES>
__device__ __forceinline__ void step_any(const ModelArgs<R>& A, Shm<R, TP>* sh, Field<R, C>& f, const R* wq, R s0,
                                         R c0, int& iters, int& flags) {
    if constexpr (S == SCH_SOLVER_EA)
        sch_step_ea<R, C, TP, NZ>(A, sh, f, wq, s0, c0, iters, flags);
    else
        sch_step<R, C, TP, NZ>(A, sh, f, wq, s0, c0, iters, flags);
}

// load m of a particle, exchange its chunk ends and solve for u
template <typename R, int C, int TP>
__device__ __forceinline__ void field_start(const ModelArgs<R>& A, Shm<R, TP>* sh, const R* m_src, Field<R, C>& f) {
    const int i0 = threadIdx.x * C;
#pragma unroll
    for (int i = 0; i < C; ++i) f.m[i] = m_src[i0 + i];
    chunk_halo<R, C, TP>(f.m, f.mp, f.mn, sh);
    R r[C];
    mass_apply<R, C>(A.h6, f.m, f.mp, f.mn, r);
    const_solve<R, C, TP>(A.hel, A.rhel, r, f.u, f.up, f.un, sh);
}

// the noise weights a_j/4 (dW + lambda dt) of a window, staged in smem
template <typename R>
__device__ __forceinline__ void stage_noise(const ModelArgs<R>& A, R* dst, const R* dW, const R* lam, int Ns) {
    const int tot = Ns * A.K;
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
        const int k = q % A.K;
        R v = dW[q];
        if (lam) v += lam[q] * A.dt;
        dst[q] = A.amp4[k >> 1] * v;
    }
}

template <typename R, int C>
__device__ __forceinline__ double chunk_misfit(const ModelArgs<R>& A, const R (&u)[C], const R* y) {
    const int i0 = threadIdx.x * C;
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const int node = i0 + i;
        if (node % A.stride == 0) {
            const R yj = y[node / A.stride];
            if (yj == yj) {   // NaN: not observed
                const R r = (u[i] - yj) * A.sigma_inv;
                acc += (double)r * (double)r;
            }
        }
    }
    return acc;
}

template <typename R>
__device__ __forceinline__ double window_girsanov(const ModelArgs<R>& A, const R* dW, const R* lam, int Ns) {
    double acc = 0.0;
    if (lam) {
        const int tot = Ns * A.K;
        for (int q = threadIdx.x; q < tot; q += blockDim.x) {
            const double l = lam[q], w = dW[q];
            acc += l * w + 0.5 * l * l * A.dt_d;
        }
    }
    return acc;
}

// sums of two doubles over the CTA; valid in thread 0
template <typename R, int TP>
__device__ __forceinline__ void block_sum2(Shm<R, TP>* sh, double& a, double& b) {
    a = warp_sum(a);
    b = warp_sum(b);
    const int t = threadIdx.x;
    if ((t & 31) == 0) {
        sh->dsum[0][t >> 5] = a;
        sh->dsum[1][t >> 5] = b;
    }
    __syncthreads();
    if (t == 0) {
        double sa = 0.0, sb = 0.0;
        for (int w = 0; w < TP / 32; ++w) {
            sa += sh->dsum[0][w];
            sb += sh->dsum[1][w];
        }
        a = sa;
        b = sb;
    }
    __syncthreads();
}

// --------------------------------------------------------------------------
// kernels
// --------------------------------------------------------------------------
// Minimum resident CTAs per SM requested from the compiler.  FP32 with 128
// threads per particle (n = 1024) asks for 7, so that 7 x 152 SMs hold a
// 1024-particle ensemble in one wave (72 registers, a few spilled); otherwise
// the register file allows up to 128 registers per thread.
template <typename R, int TP>
struct Occ {
    static constexpr int minb = (sizeof(R) == 4 && TP == 128)
                                    ? 7
                                    : (TP <= 32 ? 16 : (TP <= 64 ? 8 : (TP <= 128 ? 4 : (TP <= 256 ? 2 : 1))));
};

template <typename R, int C, int TP, int S>
__global__ void __launch_bounds__(TP, Occ<R, TP>::minb) window_kernel(ModelArgs<R> A, WindowIO<R> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shm<R, TP>* sh = reinterpret_cast<Shm<R, TP>*>(smem_raw);
    R* noise = reinterpret_cast<R*>(smem_raw + shm_base_bytes<R, TP>());
    const int p = blockIdx.x;
    const size_t NK = (size_t)io.Ns * A.K;
    stage_noise(A, noise, io.dW + p * NK, io.lam ? io.lam + p * NK : nullptr, io.Ns);
    R s0, c0;
    node_angle<R>((int)threadIdx.x * C - 1, A.n, s0, c0);
    Field<R, C> f;
    field_start<R, C, TP>(A, sh, io.m_in + (size_t)p * A.n, f);   // its barriers publish the noise
    int iters = 0, flags = 0;
    for (int s = 0; s < io.Ns; ++s) step_any<S, R, C, TP>(A, sh, f, noise + s * A.K, s0, c0, iters, flags);
    const int i0 = threadIdx.x * C;
#pragma unroll
    for (int i = 0; i < C; ++i) {
        io.m_out[(size_t)p * A.n + i0 + i] = f.m[i];
        io.u_out[(size_t)p * A.n + i0 + i] = f.u[i];
    }
    if (io.y) {
        double mis = chunk_misfit<R, C>(A, f.u, io.y);
        double gl = window_girsanov(A, io.dW + p * NK, io.lam ? io.lam + p * NK : nullptr, io.Ns);
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

// PCN jittering: n_iter proposals of the window noise, each run through the
// whole window from m_start and accepted with probability min(1, exp(w0 - w1)).
template <typename R, int C, int TP, int S>
__global__ void __launch_bounds__(TP, Occ<R, TP>::minb) jitter_kernel(ModelArgs<R> A, JitterIO<R> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shm<R, TP>* sh = reinterpret_cast<Shm<R, TP>*>(smem_raw);
    // a device-gated stage reads its temperature, and does nothing when inactive
    if (io.tstate && io.tstate[4] == 0.0) return;
    const double theta = io.tstate ? io.tstate[2] : io.theta;
    const int p = blockIdx.x;
    const int Ns = io.Ns, K = A.K, NK = Ns * K;
    R* noise = reinterpret_cast<R*>(smem_raw + shm_base_bytes<R, TP>());
    R* cur = noise + NK;
    R* prop = noise + 2 * NK;
    __shared__ double sh_state[2];
    __shared__ int sh_acc;
    R* dW = io.dW + (size_t)p * NK;
    const R* lam = io.lam ? io.lam + (size_t)p * NK : nullptr;
    for (int q = threadIdx.x; q < NK; q += TP) cur[q] = dW[q];
    if (threadIdx.x == 0) {
        sh_state[0] = io.nll[p];
        sh_state[1] = io.logG ? io.logG[p] : 0.0;
    }
    R s0, c0;
    node_angle<R>((int)threadIdx.x * C - 1, A.n, s0, c0);
    const R sq = io.sq1mr2 * (R)sqrt(A.dt_d);
    const int nblk = (K + 3) >> 2;
    const int i0 = threadIdx.x * C;
    int iters = 0, flags = 0, n_acc = 0, changed = 0;
    __syncthreads();
    for (int j = 0; j < io.n_iter; ++j) {
        const uint64_t ctr = io.ctr + (uint64_t)j;
        // proposal dW' = rho dW + sqrt(1 - rho^2) sqrt(dt) z
        for (int q = threadIdx.x; q < Ns * nblk; q += TP) {
            const int s = q / nblk, b = q % nblk;
            R z[4];
            normal4<R>(io.seed, SCH_TAG_PCN, (uint64_t)b, (uint64_t)s, (uint64_t)(io.particle0 + p), ctr, z);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 4 * b + e;
                if (k < K) prop[s * K + k] = io.rho * cur[s * K + k] + sq * z[e];
            }
        }
        __syncthreads();
        stage_noise(A, noise, prop, lam, Ns);
        Field<R, C> f;
        field_start<R, C, TP>(A, sh, io.m_start + (size_t)p * A.n, f);   // barriers publish the noise
        int fl = 0;
        for (int s = 0; s < Ns; ++s) step_any<S, R, C, TP>(A, sh, f, noise + s * K, s0, c0, iters, fl);
        double mis = chunk_misfit<R, C>(A, f.u, io.y);
        double gl = window_girsanov(A, prop, lam, Ns);
        block_sum2<R, TP>(sh, mis, gl);
        if (threadIdx.x == 0) {
            const double nll1 = 0.5 * mis, lg1 = -gl;
            const double w0 = theta * (sh_state[0] - sh_state[1]);
            const double w1 = theta * (nll1 - lg1);
            const double logU = log(uniform_open0(io.seed, SCH_TAG_PCN_ACCEPT, (uint64_t)(io.particle0 + p), ctr));
            const int acc = (fl == 0) && (logU < w0 - w1);
            sh_acc = acc;
            if (acc) {
                sh_state[0] = nll1;
                sh_state[1] = lg1;
            }
        }
        __syncthreads();
        if (sh_acc) {
            for (int q = threadIdx.x; q < NK; q += TP) cur[q] = prop[q];
#pragma unroll
            for (int i = 0; i < C; ++i) {
                io.m_end[(size_t)p * A.n + i0 + i] = f.m[i];
                io.u_end[(size_t)p * A.n + i0 + i] = f.u[i];
            }
            n_acc++;
            changed = 1;
        }
        flags |= fl;
        __syncthreads();
    }
    if (changed)
        for (int q = threadIdx.x; q < NK; q += TP) dW[q] = cur[q];
    if (threadIdx.x == 0) {
        io.nll[p] = sh_state[0];
        if (io.logG) io.logG[p] = sh_state[1];
        if (io.accepts) io.accepts[p] = n_acc;
        if (io.iters) io.iters[p] = iters;
        if (io.status) io.status[p] = flags;
    }
}

// Helmholtz utilities: mode 0: u = H^{-1} M m ; mode 1: m = M^{-1} H u
template <typename R, int C, int TP>
__global__ void __launch_bounds__(TP, Occ<R, TP>::minb) helm_kernel(ModelArgs<R> A, const R* in, R* out, int mode) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shm<R, TP>* sh = reinterpret_cast<Shm<R, TP>*>(smem_raw);
    const int p = blockIdx.x;
    const int i0 = threadIdx.x * C;
    R v[C], x[C], vp, vn, xp, xn, r[C];
#pragma unroll
    for (int i = 0; i < C; ++i) v[i] = in[(size_t)p * A.n + i0 + i];
    chunk_halo<R, C, TP>(v, vp, vn, sh);
    if (mode == 0) {
        mass_apply<R, C>(A.h6, v, vp, vn, r);
        const_solve<R, C, TP>(A.hel, A.rhel, r, x, xp, xn, sh);
    } else {
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const R lo = (i == 0) ? vp : v[i - 1];
            const R hi = (i == C - 1) ? vn : v[i + 1];
            r[i] = A.hel_a * (lo + hi) + A.hel_b * v[i];
        }
        const_solve<R, C, TP>(A.mass, A.rmass, r, x, xp, xn, sh);
    }
#pragma unroll
    for (int i = 0; i < C; ++i) out[(size_t)p * A.n + i0 + i] = x[i];
}

// Prior ensemble, S the P1 solve of (U, v) + (U_x, v_x) = (f, v), then m = M^{-1} H u:
//   mode 0: u = u_truth + scale (a_p S^3 W_p + b_p);
//   mode 1: u = a_p^2 S^3 |W_p| + b_p^2 (the Exp 1 ensemble of Eq. init_solve).
// Member p uses Philox counter particle0 + p.
template <typename R, int C, int TP>
__global__ void __launch_bounds__(TP, Occ<R, TP>::minb) prior_kernel(ModelArgs<R> A, const R* u_truth, uint64_t seed,
                                                                 R scale, R* m_out, R* u_out, int mode,
                                                                 int particle0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shm<R, TP>* sh = reinterpret_cast<Shm<R, TP>*>(smem_raw);
    const int p = blockIdx.x;
    const int i0 = threadIdx.x * C;
    const R h = A.h;
    R cell[C];
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const int e = i0 + i;
        R z[4];
        normal4<R>(seed, SCH_TAG_INIT, (uint64_t)(e >> 2), 0, (uint64_t)(particle0 + p), 0, z);
        cell[i] = (R)sqrt((double)h) * z[e & 3];
        if (mode == 1) cell[i] = fabs(cell[i]);
    }
    R ab[2];
    {
        const int k0 = A.n;
        R z[4], z2[4];
        normal4<R>(seed, SCH_TAG_INIT, (uint64_t)(k0 >> 2), 0, (uint64_t)(particle0 + p), 0, z);
        normal4<R>(seed, SCH_TAG_INIT, (uint64_t)((k0 + 1) >> 2), 0, (uint64_t)(particle0 + p), 0, z2);
        ab[0] = z[k0 & 3];
        ab[1] = z2[(k0 + 1) & 3];
    }
    // rhs (W, phi_i) = h/2 (W_{i-1} + W_i)
    R cp, cn, r[C], U[C], Up, Un;
    chunk_halo<R, C, TP>(cell, cp, cn, sh);
#pragma unroll
    for (int i = 0; i < C; ++i) r[i] = R(0.5) * h * (((i == 0) ? cp : cell[i - 1]) + cell[i]);
    const_solve<R, C, TP>(A.smooth, A.rsmooth, r, U, Up, Un, sh);
    for (int rep = 0; rep < 2; ++rep) {
        mass_apply<R, C>(A.h6, U, Up, Un, r);
        R V[C];
        const_solve<R, C, TP>(A.smooth, A.rsmooth, r, V, Up, Un, sh);
#pragma unroll
        for (int i = 0; i < C; ++i) U[i] = V[i];
    }
    R u[C], up, un;
#pragma unroll
    for (int i = 0; i < C; ++i)
        u[i] = (mode == 1) ? ab[0] * ab[0] * U[i] + ab[1] * ab[1] : u_truth[i0 + i] + scale * (ab[0] * U[i] + ab[1]);
    chunk_halo<R, C, TP>(u, up, un, sh);
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const R lo = (i == 0) ? up : u[i - 1];
        const R hi = (i == C - 1) ? un : u[i + 1];
        r[i] = A.hel_a * (lo + hi) + A.hel_b * u[i];
    }
    R m[C], mp, mn;
    const_solve<R, C, TP>(A.mass, A.rmass, r, m, mp, mn, sh);
#pragma unroll
    for (int i = 0; i < C; ++i) {
        m_out[(size_t)p * A.n + i0 + i] = m[i];
        u_out[(size_t)p * A.n + i0 + i] = u[i];
    }
}

// --------------------------------------------------------------------------
// launchers for one (R, C, TP)
// --------------------------------------------------------------------------
template <typename R, int C, int TP>
struct Launch {
    static size_t smem(int Ns, int K, int bufs) { return shm_base_bytes<R, TP>() + (size_t)bufs * Ns * K * sizeof(R); }

    template <typename Kern>
    static void prep(Kern k, size_t sm) {
        if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    }

    template <int S>
    static int window(const ModelArgs<R>& A, const WindowIO<R>& io, int N, cudaStream_t st) {
        const size_t sm = smem(io.Ns, A.K, 1);
        prep(window_kernel<R, C, TP, S>, sm);
        window_kernel<R, C, TP, S><<<N, TP, sm, st>>>(A, io);
        return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
    }
    template <int S>
    static int jitter(const ModelArgs<R>& A, const JitterIO<R>& io, int N, cudaStream_t st) {
        const size_t sm = smem(io.Ns, A.K, 3);
        prep(jitter_kernel<R, C, TP, S>, sm);
        jitter_kernel<R, C, TP, S><<<N, TP, sm, st>>>(A, io);
        return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
    }
    static int helm(const ModelArgs<R>& A, const R* in, R* out, int mode, int N, cudaStream_t st) {
        const size_t sm = smem(0, A.K, 0);
        prep(helm_kernel<R, C, TP>, sm);
        helm_kernel<R, C, TP><<<N, TP, sm, st>>>(A, in, out, mode);
        return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
    }
    static int prior(const ModelArgs<R>& A, const R* ut, uint64_t seed, R scale, R* m, R* u, int N,
                     cudaStream_t st, int mode, int particle0) {
        const size_t sm = smem(0, A.K, 0);
        prep(prior_kernel<R, C, TP>, sm);
        prior_kernel<R, C, TP><<<N, TP, sm, st>>>(A, ut, seed, scale, m, u, mode, particle0);
        return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
    }
};

}  // namespace sch
