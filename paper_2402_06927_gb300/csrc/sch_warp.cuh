// Warp-per-particle propagation for float fields (explicit-advection Picard
// solver of the implicit midpoint step, Eq. fde1), n = 64 P CS nodes.
//
// One warp carries one particle and needs no CTA barrier.  Lane l owns the
// LN = 2 P CS consecutive nodes [LN l, LN (l + 1)) as S = 2P sub-chunks of CS
// nodes, s = 0 .. S-1 in node order.  Stream p (p < P) keeps node i of
// sub-chunk p and node i of sub-chunk p + P in one float2, so stencil work on
// a stream runs on two sub-chunks at once, and a stream's chunk-end neighbours
// are whole pairs of the adjacent streams (only the lane's first and last
// nodes cross lanes).  The sub-chunk sweeps run as 2P interleaved scalar
// recurrences.  The 32 S sub-chunks of a particle leave a cyclic reduced
// system of 32 S interface rows (S per lane, rows S l + s), solved by every
// lane at once: an S-row lane partition and a cyclic PCR across the 32 lanes
// with shuffles.
//
// One Picard iteration (the step's right-hand sides R0 = (M - mu dt/2 K) m0 and
// W0 = dt/8 u0 + dU/4 fixed):
//   w = W0 + dt/8 u_it              (= dv/4 at the iterate)
//   mb2 = m0 + m_it                 (= 2 mbar)
//   rhs_i = R0_i + w_{i-1} (mb2_{i-1} + mb2_i) - w_{i+1} (mb2_i + mb2_{i+1})
//         = R0_i - A(mbar, dv)_i    (the P1 advection operator)
//   (M + mu dt/2 K) m_new = rhs            partitioned solve, reduced rows
//   (6/h)(M + alpha^2 K) u_new = m_{i-1} + 4 m_i + m_{i+1}    likewise
// followed by the stop test on the whole particle (two warp reductions):
// max|m_new - m_it| <= tol max(1, max|m_new|), or the contraction estimate of
// ea_converged.
#pragma once

#include "sch_kernels.cuh"

namespace sch {

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2b(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)));
    return *reinterpret_cast<float2*>(&r);
}

// max(a, b, c), NaN if any input is NaN
__device__ __forceinline__ float fmax3_nan(float a, float b, float c) {
    float r;
    asm("max.NaN.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// maximum over the warp, NaN if any lane holds NaN
__device__ __forceinline__ float warp_max_nan(float v) {
    float r;
    asm volatile("redux.sync.max.NaN.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

// The lane's outer chunk-end neighbours of a paired field: lo, left of pair 0
// of stream 0 = (previous lane's last node, last node of sub-chunk P-1), and
// hi, right of the last pair of stream P-1 = (first node of sub-chunk P, next
// lane's first node).  Every other stream boundary is an adjacent stream's pair.
template <int CS, int P>
__device__ __forceinline__ void whalo(const float2 (&v)[P][CS], float2& lo, float2& hi) {
    const int lane = threadIdx.x & 31;
    lo = make_float2(__shfl_sync(FULL, v[P - 1][CS - 1].y, (lane + 31) & 31), v[P - 1][CS - 1].x);
    hi = make_float2(v[0][0].y, __shfl_sync(FULL, v[0][0].x, (lane + 1) & 31));
}

// stencil neighbours of pair i of stream p
template <int CS, int P>
__device__ __forceinline__ float2 wleft(const float2 (&v)[P][CS], int p, int i, float2 lo) {
    return (i > 0) ? v[p][i - 1] : ((p == 0) ? lo : v[p - 1][CS - 1]);
}
template <int CS, int P>
__device__ __forceinline__ float2 wright(const float2 (&v)[P][CS], int p, int i, float2 hi) {
    return (i < CS - 1) ? v[p][i + 1] : ((p == P - 1) ? hi : v[p + 1][0]);
}

// Forward and backward sweep of every sub-chunk.  x holds the right-hand side
// on entry and the interior particular solution dp_1 .. dp_{CS-2} on exit (x[.][0]
// keeps rhs_0); pd = (rhs_0 - a dp_1) / BF and de = the last forward value,
// the two reduced-row inputs of each sub-chunk.  The 2P recurrences are
// interleaved; their coefficients come from the parameter bank.
template <int CS, int P>
__device__ __forceinline__ void wsweep(const WTab& T, float2 (&x)[P][CS], float2 (&pd)[P], float2 (&de)[P]) {
    float dx[P], dy[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        dx[p] = T.rden[1] * x[p][1].x;
        dy[p] = T.rden[1] * x[p][1].y;
        x[p][1] = make_float2(dx[p], dy[p]);
    }
#pragma unroll
    for (int i = 2; i < CS; ++i) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            dx[p] = fmaf(T.nar[i], dx[p], T.rden[i] * x[p][i].x);
            dy[p] = fmaf(T.nar[i], dy[p], T.rden[i] * x[p][i].y);
            x[p][i] = make_float2(dx[p], dy[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        de[p] = make_float2(dx[p], dy[p]);
        dx[p] = x[p][CS - 2].x;
        dy[p] = x[p][CS - 2].y;
    }
#pragma unroll
    for (int i = CS - 3; i >= 1; --i) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            dx[p] = fmaf(T.ngam[i], dx[p], x[p][i].x);
            dy[p] = fmaf(T.ngam[i], dy[p], x[p][i].y);
            x[p][i] = make_float2(dx[p], dy[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
        pd[p] = make_float2(T.iBF * fmaf(T.na, x[p][1].x, x[p][0].x), T.iBF * fmaf(T.na, x[p][1].y, x[p][0].y));
}

// How a kernel solves a table's reduced system: by its diag flag at run time, or
// specialised at launch to the diagonal solve or the PCR (the loop then holds one
// of the two, which keeps it within the instruction cache)
constexpr int RED_RUNTIME = 0, RED_DIAG = 1, RED_PCR = 2;

// The cyclic reduced system E_t (t = S l + s) of a constant matrix,
// D_t = de_t - ae pd_t - ge pd_{t+1}.  Returns the pairs E[p] = (E of sub-chunk
// p, of p + P) and F[p] likewise (the last and first values of the sub-chunks),
// and the lane's outer neighbours Ep = E_{S l - 1}, Fn = F_{S (l + 1)}.  A system
// flagged diagonal (T.diag) is solved as E_t = D_t / B; otherwise an S-row lane
// partition feeds a cyclic PCR over the lanes.  RM: one of RED_*.
template <int P, int RM = RED_RUNTIME>
__device__ __forceinline__ void wreduced(const WTab& T, const RTab<float>& Q, const float2 (&pd)[P],
                                         const float2 (&de)[P], float2 (&E)[P], float2 (&F)[P], float& Ep,
                                         float& Fn) {
    constexpr int S = 2 * P;
    const int lane = threadIdx.x & 31;
    float pr[S], dr[S], Er[S], Fr[S];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        pr[p] = pd[p].x;
        pr[p + P] = pd[p].y;
        dr[p] = de[p].x;
        dr[p + P] = de[p].y;
    }
    const bool diag = (RM == RED_DIAG) || (RM == RED_RUNTIME && T.diag);
    if (diag) {
        const float pdn = __shfl_sync(FULL, pr[0], (lane + 1) & 31);
#pragma unroll
        for (int r = 0; r < S; ++r)
            Er[r] = (dr[r] - T.ae * pr[r] - T.ge * ((r == S - 1) ? pdn : pr[r + 1])) * T.iB;
        Ep = __shfl_sync(FULL, Er[S - 1], (lane + 31) & 31);
#pragma unroll
        for (int r = 0; r < S; ++r) Fr[r] = pr[r] - T.pa * ((r == 0) ? Ep : Er[r - 1]) - T.pc * Er[r];
    } else {
        lane_solve_const<float, 32 * S>(T, Q, pr, dr, Er, Fr, &Ep);
    }
    Fn = __shfl_sync(FULL, Fr[0], (lane + 1) & 31);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        E[p] = make_float2(Er[p], Er[p + P]);
        F[p] = make_float2(Fr[p], Fr[p + P]);
    }
}

// back substitution: x_i = dp_i - alpp_i F - gamp_i E, x_0 = F, x_{CS-1} = E
template <int CS, int P>
__device__ __forceinline__ void wback(const WTab& T, const float2 (&dp)[P][CS], const float2 (&F)[P],
                                      const float2 (&E)[P], float2 (&x)[P][CS]) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
        x[p][0] = F[p];
        x[p][CS - 1] = E[p];
#pragma unroll
        for (int i = 1; i < CS - 1; ++i)
            x[p][i] = make_float2(fmaf(T.nalpp[i], F[p].x, fmaf(T.ngamp[i], E[p].x, dp[p][i].x)),
                                  fmaf(T.nalpp[i], F[p].y, fmaf(T.ngamp[i], E[p].y, dp[p][i].y)));
    }
}

// the lane's outer chunk-end neighbours of a field just solved for, from its
// reduced solve (see whalo)
template <int P>
__device__ __forceinline__ void wsolved_halo(const float2 (&E)[P], const float2 (&F)[P], float Ep, float Fn,
                                             float2& lo, float2& hi) {
    lo = make_float2(Ep, E[P - 1].x);
    hi = make_float2(F[0].y, Fn);
}

// u = H^{-1} M m for this lane's nodes
template <int CS, int P, int HM = RED_RUNTIME>
__device__ __forceinline__ void wu_from_m(const WArgs& W, const float2 (&m)[P][CS], float2 (&u)[P][CS]) {
    float2 lo, hi, x[P][CS];
    whalo<CS, P>(m, lo, hi);
    const float2 four = f2b(4.f);
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
        for (int i = 0; i < CS; ++i)
            x[p][i] = f2fma(four, m[p][i], f2add(wleft<CS, P>(m, p, i, lo), wright<CS, P>(m, p, i, hi)));
    float2 pd[P], de[P], E[P], F[P];
    float Ep, Fn;
    wsweep<CS, P>(W.hel, x, pd, de);
    wreduced<P, HM>(W.hel, W.rhel, pd, de, E, F, Ep, Fn);
    wback<CS, P>(W.hel, x, F, E, u);
}

// SALT increment dU/4 at this lane's nodes from the step's K weights
// wq_k = a_j/4 (dW_k + lambda_k dt): dU_i/4 = sum_j wq_{2j-2} sin(j theta_i) +
// wq_{2j-1} cos(j theta_i).  The lane's 2H nodes (H = P CS) sit at theta_c -+ d_m,
// d_m = (m + 1/2) 2 pi / n, m < H, about its centre theta_c; by the angle-sum rules
//   dU/4 (theta_c +- d) = E(d) +- O(d),  E(d) = sum_j v_j cos(j d),  O(d) = sum_j q_j sin(j d),
//   v_j = wq_{2j-2} sin(j theta_c) + wq_{2j-1} cos(j theta_c),  q_j = wq_{2j-2} cos(j theta_c)
//         - wq_{2j-1} sin(j theta_c),
// so a harmonic costs the lane two FMAs for each pair of mirrored nodes (tabulated
// cos(j d), sin(j d): WArgs nco, nsi) plus the rotation of (sin, cos)(j theta_c) to j + 1.
// (The warp-group kernels can instead sum the harmonics through polynomials of the
// offsets: gnoise in sch_group.cuh.)
// EP[q] = (E(d_{H-1-q}), E(d_q)), OP likewise, q < H/2.  sc, cc: sin and cos of theta_c.
template <int CS, int P>
__device__ __forceinline__ void wnoise_tab(const ModelArgs<float>& A, const WArgs& Wa, const float* wq, float sc,
                                           float cc, float2 (&EP)[P * CS / 2], float2 (&OP)[P * CS / 2]) {
    constexpr int H = P * CS, Q = H / 2;
    static_assert(H % 2 == 0 && Q <= WNQ_MAX, "a lane half of an even number of nodes within the tables");
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        EP[q] = f2b(0.f);
        OP[q] = f2b(0.f);
    }
    float sj = sc, cj = cc;
#pragma unroll 2
    for (int j = 0; j < A.K2; ++j) {
        const float2 ab = *reinterpret_cast<const float2*>(wq + 2 * j);
        const float2 v = f2b(fmaf(ab.x, sj, ab.y * cj));
        const float2 qv = f2b(fmaf(ab.x, cj, -(ab.y * sj)));
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            EP[q] = f2fma(v, Wa.nco[j][q], EP[q]);
            OP[q] = f2fma(qv, Wa.nsi[j][q], OP[q]);
        }
        const float sn = fmaf(sj, cc, cj * sc);
        cj = fmaf(cj, cc, -(sj * sc));
        sj = sn;
    }
}

// dU/4 at the lane's 2H nodes from the even and odd parts: pair (p, i), k = p CS + i:
// node k of the lane's first half is theta_c - d_{H-1-k}, node H + k of its second half
// theta_c + d_k
template <int CS, int P>
__device__ __forceinline__ void wnoise_finish(const float2 (&EP)[P * CS / 2], const float2 (&OP)[P * CS / 2],
                                              float2 (&nq)[P][CS]) {
    constexpr int H = P * CS, Q = H / 2;
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
        for (int i = 0; i < CS; ++i) {
            const int k = p * CS + i;
            if (k < Q) {
                nq[p][i] = make_float2(EP[k].x - OP[k].x, EP[k].y + OP[k].y);
            } else {
                const int q = H - 1 - k;
                nq[p][i] = make_float2(EP[q].y - OP[q].y, EP[q].x + OP[q].x);
            }
        }
}

template <int CS, int P>
__device__ __forceinline__ void wnoise(const ModelArgs<float>& A, const WArgs& Wa, const float* wq, float sc,
                                       float cc, float2 (&nq)[P][CS]) {
    float2 EP[P * CS / 2], OP[P * CS / 2];
    wnoise_tab<CS, P>(A, Wa, wq, sc, cc, EP, OP);
    wnoise_finish<CS, P>(EP, OP, nq);
}

// One implicit-midpoint step of this warp's particle: (m, u) in/out, W0 holding the
// step's dU/4 at the lane's nodes on entry.
// R0sm: this warp's [P][CS][32] float2 scratch for R0 = (M - mu dt/2 K) m0.
// PM, HM: how the Picard and Helmholtz reduced systems are solved (RED_*).
template <int CS, int P, int PM = RED_RUNTIME, int HM = RED_RUNTIME>
__device__ __forceinline__ void wstep_core(const ModelArgs<float>& A, const WArgs& W, float2 (&m)[P][CS],
                                           float2 (&u)[P][CS], float2* R0sm, float2 (&W0)[P][CS], int& iters,
                                           int& flags) {
    const int lane = threadIdx.x & 31;
    // W0 = dt/8 u0 + dU/4 (registers) and R0 (shared memory), fixed for the step
    {
        const float2 dt8 = f2b(A.dt8);
        float2 lo, hi;
        whalo<CS, P>(m, lo, hi);
        const float2 c0p = f2b(A.c0p), b0p = f2b(A.b0p);
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int i = 0; i < CS; ++i) {
                W0[p][i] = f2fma(dt8, u[p][i], W0[p][i]);
                R0sm[(p * CS + i) * 32 + lane] =
                    f2fma(c0p, f2add(wleft<CS, P>(m, p, i, lo), wright<CS, P>(m, p, i, hi)), f2mul(b0p, m[p][i]));
            }
    }
    float2 mi[P][CS];
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
        for (int i = 0; i < CS; ++i) mi[p][i] = m[p][i];
    const float2 dt8 = f2b(A.dt8);
    float dm_prev = INFINITY;
    for (int it = 1;; ++it) {
        // rhs_i = R0_i + w_{i-1} g_{i-1} - w_{i+1} g_i,  w = W0 + dt/8 u_it,  g_i = mb2_i + mb2_{i+1}
        float2 x[P][CS];
        {
            float2 w[P][CS], mb[P][CS];
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int i = 0; i < CS; ++i) {
                    w[p][i] = f2fma(dt8, u[p][i], W0[p][i]);
                    mb[p][i] = f2add(m[p][i], mi[p][i]);
                }
            float2 wl, wr, ml, mr;
            whalo<CS, P>(w, wl, wr);
            whalo<CS, P>(mb, ml, mr);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                float2 gp = f2add(wleft<CS, P>(mb, p, 0, ml), mb[p][0]);
#pragma unroll
                for (int i = 0; i < CS; ++i) {
                    const float2 g = f2add(mb[p][i], wright<CS, P>(mb, p, i, mr));
                    x[p][i] = f2sub(f2fma(wleft<CS, P>(w, p, i, wl), gp, R0sm[(p * CS + i) * 32 + lane]),
                                    f2mul(wright<CS, P>(w, p, i, wr), g));
                    gp = g;
                }
            }
        }
        // (M + mu dt/2 K) m_new = rhs
        float2 pd[P], de[P], E[P], F[P];
        float Ep, Fn;
        wsweep<CS, P>(W.pic, x, pd, de);
        wreduced<P, PM>(W.pic, W.rpic, pd, de, E, F, Ep, Fn);
        float2 mn[P][CS];
        wback<CS, P>(W.pic, x, F, E, mn);
        float dmax = 0.f, mmax = 0.f;
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int i = 0; i < CS; ++i) {
                const float2 d = f2sub(mn[p][i], mi[p][i]);
                dmax = fmax3_nan(dmax, fabsf(d.x), fabsf(d.y));
                mmax = fmaxf(mmax, fmaxf(fabsf(mn[p][i].x), fabsf(mn[p][i].y)));
                mi[p][i] = mn[p][i];
            }
        // u_new = H^{-1} M m_new, the mass product's chunk ends from the reduced solve
        {
            float2 lo, hi;
            wsolved_halo<P>(E, F, Ep, Fn, lo, hi);
            const float2 four = f2b(4.f);
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int i = 0; i < CS; ++i)
                    x[p][i] = f2fma(four, mn[p][i], f2add(wleft<CS, P>(mn, p, i, lo), wright<CS, P>(mn, p, i, hi)));
            float2 hpd[P], hde[P], hE[P], hF[P];
            float hEp, hFn;
            wsweep<CS, P>(W.hel, x, hpd, hde);
            wreduced<P, HM>(W.hel, W.rhel, hpd, hde, hE, hF, hEp, hFn);
            wback<CS, P>(W.hel, x, hF, hE, u);
        }
        iters++;
        const float dm = warp_max_nan(dmax);
        const float mm = warp_max_nan(mmax);
        if (!(dm < INFINITY) || !(mm < INFINITY)) {
            flags |= SCH_DEV_NONFINITE;
            break;
        }
        if (ea_converged(dm, dm_prev, A.tol * fmaxf(1.f, mm))) break;
        dm_prev = dm;
        if (it >= A.max_iter) {
            flags |= SCH_DEV_NOCONVERGE;
            break;
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
        for (int i = 0; i < CS; ++i) m[p][i] = mi[p][i];
}

// One step with the mode-expansion noise of the step's K weights wq.
template <int CS, int P, int PM, int HM>
__device__ __forceinline__ void wstep(const ModelArgs<float>& A, const WArgs& W, float2 (&m)[P][CS],
                                      float2 (&u)[P][CS], float2* R0sm, const float* wq, float sc, float cc,
                                      int& iters, int& flags) {
    float2 W0[P][CS];
    wnoise<CS, P>(A, W, wq, sc, cc, W0);
    wstep_core<CS, P, PM, HM>(A, W, m, u, R0sm, W0, iters, flags);
}

// this thread's LN = 2 P CS nodes of a particle row <-> the paired registers:
// sub-chunk s < P is stream s's .x, sub-chunk s >= P is stream s - P's .y.  Thread t
// of the CTA owns nodes [LN t, LN (t + 1)): lane t of a one-warp CTA, or lane t % 32
// of warp t / 32 when several warps carry the particle (sch_group.cuh).
template <int CS, int P>
__device__ __forceinline__ void wload(const float* row, float2 (&v)[P][CS]) {
    const float4* q4 = reinterpret_cast<const float4*>(row + threadIdx.x * 2 * P * CS);
#pragma unroll
    for (int s = 0; s < 2 * P; ++s)
#pragma unroll
        for (int q = 0; q < CS / 4; ++q) {
            const float4 a = q4[s * (CS / 4) + q];
            const float e[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (s < P) v[s][4 * q + k].x = e[k];
                else v[s - P][4 * q + k].y = e[k];
            }
        }
}

template <int CS, int P>
__device__ __forceinline__ void wstore(float* row, const float2 (&v)[P][CS]) {
    float4* q4 = reinterpret_cast<float4*>(row + threadIdx.x * 2 * P * CS);
#pragma unroll
    for (int s = 0; s < 2 * P; ++s)
#pragma unroll
        for (int q = 0; q < CS / 4; ++q) {
            float e[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) e[k] = (s < P) ? v[s][4 * q + k].x : v[s - P][4 * q + k].y;
            q4[s * (CS / 4) + q] = make_float4(e[0], e[1], e[2], e[3]);
        }
}

// observation misfit sum_j ((u(x_j) - y_j) / sigma)^2 over this thread's observed
// nodes (y_j not NaN); node mod stride and the observation index advance node by node
template <int CS, int P>
__device__ __forceinline__ double wmisfit(const ModelArgs<float>& A, const float2 (&u)[P][CS], const float* y) {
    const int base = threadIdx.x * 2 * P * CS;
    double acc = 0.0;
    int rem = base % A.stride;
    int j = base / A.stride + (rem != 0);
#pragma unroll
    for (int s = 0; s < 2 * P; ++s) {
#pragma unroll
        for (int i = 0; i < CS; ++i) {
            if (rem == 0) {
                const float yj = y[j];
                if (yj == yj) {   // NaN: not observed
                    const float r = (((s < P) ? u[s][i].x : u[s - P][i].y) - yj) * A.sigma_inv;
                    acc += (double)r * (double)r;
                }
                ++j;
            }
            rem = (rem + 1 == A.stride) ? 0 : rem + 1;
        }
    }
    return acc;
}

// sin and cos of the angle of this thread's lane centre, halfway between its nodes
// H - 1 and H (H = P CS): 2 pi (LN t + H - 1/2) / n for thread t, LN = 2H
template <int CS, int P>
__device__ __forceinline__ void wcentre(int n, float& sc, float& cc) {
    constexpr int LN = 2 * P * CS;
    double s, c;
    sincospi((double)(2 * LN * (int)threadIdx.x + LN - 1) / (double)n, &s, &c);
    sc = (float)s;
    cc = (float)c;
}

template <int CS, int P>
__host__ __device__ constexpr size_t wsmem_base() {
    return (size_t)P * CS * 32 * sizeof(float2);
}

// Occupancy: 8 one-warp CTAs per SM (255 registers a thread)
constexpr int WMINB = 8;

template <int CS, int P, int PM, int HM>
__global__ void __launch_bounds__(32, WMINB) wwindow_kernel(ModelArgs<float> A, WArgs W, WindowIO<float> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* R0sm = reinterpret_cast<float2*>(smem_raw);
    float* noise = reinterpret_cast<float*>(smem_raw + wsmem_base<CS, P>());
    const int p = blockIdx.x;
    const size_t NK = (size_t)io.Ns * A.K;
    stage_noise(A, noise, io.dW + p * NK, io.lam ? io.lam + p * NK : nullptr, io.Ns);
    float sc, cc;
    wcentre<CS, P>(A.n, sc, cc);
    float2 m[P][CS], u[P][CS];
    wload<CS, P>(io.m_in + (size_t)p * A.n, m);
    wu_from_m<CS, P, HM>(W, m, u);
    __syncwarp();
    int iters = 0, flags = 0;
    for (int s = 0; s < io.Ns; ++s) wstep<CS, P, PM, HM>(A, W, m, u, R0sm, noise + s * A.K, sc, cc, iters, flags);
    wstore<CS, P>(io.m_out + (size_t)p * A.n, m);
    wstore<CS, P>(io.u_out + (size_t)p * A.n, u);
    if (io.y) {
        double mis = warp_sum(wmisfit<CS, P>(A, u, io.y));
        double gl = warp_sum(window_girsanov(A, io.dW + p * NK, io.lam ? io.lam + p * NK : nullptr, io.Ns));
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

// PCN jittering (Sec. 3.1.2): n_iter proposals dW' = rho dW + sqrt(1 - rho^2)
// sqrt(dt) z of the window noise, each run through the window from m_start
// and accepted with probability min(1, exp(w0 - w1)), w = theta (NLL - log G).
template <int CS, int P, int PM, int HM>
__global__ void __launch_bounds__(32, WMINB) wjitter_kernel(ModelArgs<float> A, WArgs W, JitterIO<float> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* R0sm = reinterpret_cast<float2*>(smem_raw);
    // a device-gated stage reads its temperature, and does nothing when inactive
    if (io.tstate && io.tstate[4] == 0.0) return;
    const double theta = io.tstate ? io.tstate[2] : io.theta;
    const int p = blockIdx.x;
    const int lane = threadIdx.x;
    const int Ns = io.Ns, K = A.K, NK = Ns * K;
    float* noise = reinterpret_cast<float*>(smem_raw + wsmem_base<CS, P>());
    float* cur = noise + NK;
    float* prop = noise + 2 * NK;
    float* dW = io.dW + (size_t)p * NK;
    const float* lam = io.lam ? io.lam + (size_t)p * NK : nullptr;
    for (int q = lane; q < NK; q += 32) cur[q] = dW[q];
    double nll0 = io.nll[p], lg0 = io.logG ? io.logG[p] : 0.0;
    float sc, cc;
    wcentre<CS, P>(A.n, sc, cc);
    const float sq = io.sq1mr2 * (float)sqrt(A.dt_d);
    const int nblk = (K + 3) >> 2;
    int iters = 0, flags = 0, n_acc = 0, changed = 0;
    __syncwarp();
    for (int j = 0; j < io.n_iter; ++j) {
        const uint64_t ctr = io.ctr + (uint64_t)j;
        for (int q = lane; q < Ns * nblk; q += 32) {
            const int s = q / nblk, b = q % nblk;
            float z[4];
            normal4<float>(io.seed, SCH_TAG_PCN, (uint64_t)b, (uint64_t)s, (uint64_t)(io.particle0 + p), ctr, z);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 4 * b + e;
                if (k < K) prop[s * K + k] = io.rho * cur[s * K + k] + sq * z[e];
            }
        }
        __syncwarp();
        stage_noise(A, noise, prop, lam, Ns);
        float2 m[P][CS], u[P][CS];
        wload<CS, P>(io.m_start + (size_t)p * A.n, m);
        wu_from_m<CS, P, HM>(W, m, u);
        __syncwarp();
        int fl = 0;
        for (int s = 0; s < Ns; ++s) wstep<CS, P, PM, HM>(A, W, m, u, R0sm, noise + s * K, sc, cc, iters, fl);
        const double mis = warp_sum(wmisfit<CS, P>(A, u, io.y));
        const double gl = warp_sum(window_girsanov(A, prop, lam, Ns));
        const double nll1 = 0.5 * mis, lg1 = -gl;
        int acc = 0;
        if (lane == 0) {
            const double w0 = theta * (nll0 - lg0);
            const double w1 = theta * (nll1 - lg1);
            const double logU = log(uniform_open0(io.seed, SCH_TAG_PCN_ACCEPT, (uint64_t)(io.particle0 + p), ctr));
            acc = (fl == 0) && (logU < w0 - w1);
        }
        acc = __shfl_sync(FULL, acc, 0);
        if (acc) {
            nll0 = nll1;
            lg0 = lg1;
            for (int q = lane; q < NK; q += 32) cur[q] = prop[q];
            wstore<CS, P>(io.m_end + (size_t)p * A.n, m);
            wstore<CS, P>(io.u_end + (size_t)p * A.n, u);
            n_acc++;
            changed = 1;
        }
        flags |= fl;
        __syncwarp();
    }
    if (changed)
        for (int q = lane; q < NK; q += 32) dW[q] = cur[q];
    if (lane == 0) {
        io.nll[p] = nll0;
        if (io.logG) io.logG[p] = lg0;
        if (io.accepts) io.accepts[p] = n_acc;
        if (io.iters) io.iters[p] = iters;
        if (io.status) io.status[p] = flags;
    }
}

}  // namespace sch
