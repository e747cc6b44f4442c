// Warp-per-particle propagation for float fields (explicit-advection Picard
// solver of the implicit midpoint step, Eq. fde1), n = 64 CS nodes, CS <= 16.
//
// One warp carries one particle and needs no CTA barrier.  Lane l owns the
// 2 CS consecutive nodes [2 CS l, 2 CS (l + 1)) as two sub-chunks X (first CS
// nodes) and Y (last CS), and keeps node i of X and node i of Y in one float2.
// Every stencil operation and every chunk sweep then runs on both sub-chunks at
// once with the packed f32x2 instructions (fma.rn.f32x2 and friends).  The
// 64 sub-chunks of a particle leave a cyclic reduced system of 64 interface
// rows (two per lane, rows 2l and 2l + 1), solved by every lane at once: a
// two-row lane sweep and a cyclic PCR across the 32 lanes with shuffles.
//
// One Picard iteration (the step's right-hand sides R0 = (M - mu dt/2 K) m0 and
// W0 = dt/8 u0 + dU/4 fixed):
//   w = W0 + dt/8 u_it              (= dv/4 at the iterate)
//   mb2 = m0 + m_it                 (= 2 mbar)
//   rhs_i = R0_i + w_{i-1} (mb2_{i-1} + mb2_i) - w_{i+1} (mb2_i + mb2_{i+1})
//         = R0_i - A(mbar, dv)_i    (the P1 advection operator)
//   (M + mu dt/2 K) m_new = rhs            partitioned solve, reduced rows
//   (6/h)(M + alpha^2 K) u_new = m_{i-1} + 4 m_i + m_{i+1}    likewise
// followed by the stop test max|m_new - m_it| <= tol max(1, max|m_new|) on
// the whole particle (two warp reductions).
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

// chunk-end neighbours of a paired field: lo = (x_{-1}, y_{-1}) of pair 0 and
// hi = (x_CS, y_CS) of pair CS - 1, i.e. (previous lane's last Y node, own
// last X node) and (own first Y node, next lane's first X node)
template <int CS>
__device__ __forceinline__ void whalo(const float2 (&v)[CS], float2& lo, float2& hi) {
    const int lane = threadIdx.x & 31;
    lo = make_float2(__shfl_sync(FULL, v[CS - 1].y, (lane + 31) & 31), v[CS - 1].x);
    hi = make_float2(v[0].y, __shfl_sync(FULL, v[0].x, (lane + 1) & 31));
}

// Forward and backward sweep of both sub-chunks.  x holds the right-hand side
// on entry and the interior particular solution dp_1 .. dp_{CS-2} on exit (x[0]
// keeps rhs_0); pd = (rhs_0 - a dp_1) / BF and de = the last forward value,
// the two reduced-row inputs of each sub-chunk.  The X and Y halves run as two
// independent scalar recurrences whose coefficients come from the parameter bank.
template <int CS>
__device__ __forceinline__ void wsweep(const WTab& T, float2 (&x)[CS], float2& pd, float2& de) {
    float dx = T.rden[1] * x[1].x, dy = T.rden[1] * x[1].y;
    x[1] = make_float2(dx, dy);
#pragma unroll
    for (int i = 2; i < CS; ++i) {
        dx = fmaf(T.nar[i], dx, T.rden[i] * x[i].x);
        dy = fmaf(T.nar[i], dy, T.rden[i] * x[i].y);
        x[i] = make_float2(dx, dy);
    }
    de = make_float2(dx, dy);
    float px = x[CS - 2].x, py = x[CS - 2].y;
#pragma unroll
    for (int i = CS - 3; i >= 1; --i) {
        px = fmaf(T.ngam[i], px, x[i].x);
        py = fmaf(T.ngam[i], py, x[i].y);
        x[i] = make_float2(px, py);
    }
    pd = make_float2(T.iBF * fmaf(T.na, x[1].x, x[0].x), T.iBF * fmaf(T.na, x[1].y, x[0].y));
}

// The 64-row reduced cyclic system E_t of a constant matrix.  Row t of lane l:
// t = 2l (sub-chunk X) and 2l + 1 (Y), D_t = de_t - ae pd_t - ge pd_{t+1}.
// Returns E = (E_2l, E_2l+1) and F = (F_2l, F_2l+1), the last and first values
// of the two sub-chunks, and the neighbours Ep = E_{2l-1} (previous lane's Y
// last value) and Fn = F_{2l+2}.  A system flagged diagonal (T.diag) is solved
// as E_t = D_t / B; otherwise a two-row lane partition feeds a cyclic PCR over
// the lanes' last rows.
__device__ __forceinline__ void wreduced(const WTab& T, const RTab<float>& Q, float2 pd, float2 de, float2& E,
                                         float2& F, float& Ep, float& Fn) {
    const int lane = threadIdx.x & 31;
    const float pdn = __shfl_sync(FULL, pd.x, (lane + 1) & 31);
    const float D0 = de.x - T.ae * pd.x - T.ge * pd.y;
    const float D1 = de.y - T.ae * pd.y - T.ge * pdn;
    if (T.diag) {
        E = make_float2(D0 * T.iB, D1 * T.iB);
        Ep = __shfl_sync(FULL, E.y, (lane + 31) & 31);
    } else {
        const float qd = D0 * Q.iBF;
        const float nqd = __shfl_sync(FULL, qd, (lane + 1) & 31);
        const float LD = D1 * Q.q[1] - Q.aeL * qd - Q.geL * nqd;
        const float EL = pcr32_const(LD, Q);
        Ep = __shfl_sync(FULL, EL, (lane + 31) & 31);
        E = make_float2(qd - Q.qa * Ep - Q.qc * EL, EL);
    }
    F = make_float2(pd.x - T.pa * Ep - T.pc * E.x, pd.y - T.pa * E.x - T.pc * E.y);
    Fn = __shfl_sync(FULL, F.x, (lane + 1) & 31);
}

// back substitution: x_i = dp_i - alpp_i F - gamp_i E, x_0 = F, x_{CS-1} = E
template <int CS>
__device__ __forceinline__ void wback(const WTab& T, const float2 (&dp)[CS], float2 F, float2 E, float2 (&x)[CS]) {
    x[0] = F;
    x[CS - 1] = E;
#pragma unroll
    for (int i = 1; i < CS - 1; ++i)
        x[i] = make_float2(fmaf(T.nalpp[i], F.x, fmaf(T.ngamp[i], E.x, dp[i].x)),
                           fmaf(T.nalpp[i], F.y, fmaf(T.ngamp[i], E.y, dp[i].y)));
}

// u = H^{-1} M m for this lane's nodes
template <int CS>
__device__ __forceinline__ void wu_from_m(const WArgs& W, const float2 (&m)[CS], float2 (&u)[CS]) {
    float2 lo, hi, x[CS];
    whalo<CS>(m, lo, hi);
#pragma unroll
    for (int i = 0; i < CS; ++i) {
        const float2 l = (i == 0) ? lo : m[i - 1];
        const float2 r = (i == CS - 1) ? hi : m[i + 1];
        x[i] = f2fma(f2b(4.f), m[i], f2add(l, r));
    }
    float2 pd, de, E, F;
    float Ep, Fn;
    wsweep<CS>(W.hel, x, pd, de);
    wreduced(W.hel, W.rhel, pd, de, E, F, Ep, Fn);
    wback<CS>(W.hel, x, F, E, u);
}

// SALT increment dU/4 at this lane's nodes from the step's K weights
// wq_k = a_j/4 (dW_k + lambda_k dt): dU_i/4 = sum_j wq_{2j-2} sin(j theta_i) +
// wq_{2j-1} cos(j theta_i).  s1, c1: sin and cos of the angles of the first
// X and Y nodes; the harmonics' start values follow the Chebyshev recurrence
// in j.  Along a sub-chunk each harmonic's value v = a sin(j theta) + b cos(j theta)
// and its quadrature q = a cos(j theta) - b sin(j theta) are rotated together by
// the angle j 2 pi / n, so a node costs one rotation and one add per harmonic.
template <int CS>
__device__ __forceinline__ void wnoise(const ModelArgs<float>& A, const float* wq, float2 s1, float2 c1,
                                       float2 (&nq)[CS]) {
    const float2 twoc = f2add(c1, c1);
    float2 sj = s1, cj = c1, nsjm = f2b(0.f), ncjm = f2b(-1.f);   // nsjm = -sin((j-1) theta)
    for (int j = 0; j < A.K2; ++j) {
        const float a = wq[2 * j], b = wq[2 * j + 1];
        const float2 rc = f2b(A.rot_c[j]), rs = f2b(A.rot_s[j]), nrs = f2b(-A.rot_s[j]);
        float2 v = f2fma(f2b(a), sj, f2mul(f2b(b), cj));
        float2 q = f2fma(f2b(a), cj, f2mul(f2b(-b), sj));
#pragma unroll
        for (int i = 0; i < CS; ++i) {
            nq[i] = (j == 0) ? v : f2add(nq[i], v);
            if (i < CS - 1) {
                const float2 v2 = f2fma(v, rc, f2mul(q, rs));
                q = f2fma(q, rc, f2mul(v, nrs));
                v = v2;
            }
        }
        const float2 sn2 = f2fma(twoc, sj, nsjm), cn2 = f2fma(twoc, cj, ncjm);
        nsjm = f2mul(sj, f2b(-1.f));
        ncjm = f2mul(cj, f2b(-1.f));
        sj = sn2;
        cj = cn2;
    }
}

// One implicit-midpoint step of this warp's particle: (m, u) in/out.
// R0sm: this warp's [CS][32] float2 scratch for R0 = (M - mu dt/2 K) m0.
template <int CS>
__device__ __forceinline__ void wstep(const ModelArgs<float>& A, const WArgs& W, float2 (&m)[CS], float2 (&u)[CS],
                                      float2* R0sm, const float* wq, float2 s1, float2 c1, int& iters, int& flags) {
    const int lane = threadIdx.x & 31;
    // W0 = dt/8 u0 + dU/4 (registers) and R0 (shared memory), fixed for the step
    float2 W0[CS];
    {
        wnoise<CS>(A, wq, s1, c1, W0);
        const float2 dt8 = f2b(A.dt8);
#pragma unroll
        for (int i = 0; i < CS; ++i) W0[i] = f2fma(dt8, u[i], W0[i]);
        float2 lo, hi;
        whalo<CS>(m, lo, hi);
        const float2 c0p = f2b(A.c0p), b0p = f2b(A.b0p);
#pragma unroll
        for (int i = 0; i < CS; ++i) {
            const float2 l = (i == 0) ? lo : m[i - 1];
            const float2 r = (i == CS - 1) ? hi : m[i + 1];
            R0sm[i * 32 + lane] = f2fma(c0p, f2add(l, r), f2mul(b0p, m[i]));
        }
    }
    float2 mi[CS];
#pragma unroll
    for (int i = 0; i < CS; ++i) mi[i] = m[i];
    const float2 dt8 = f2b(A.dt8);
    for (int it = 1;; ++it) {
        // rhs_i = R0_i + w_{i-1} g_{i-1} - w_{i+1} g_i,  w = W0 + dt/8 u_it,  g_i = mb2_i + mb2_{i+1}
        float2 x[CS];
        {
            float2 w[CS], mb[CS];
#pragma unroll
            for (int i = 0; i < CS; ++i) {
                w[i] = f2fma(dt8, u[i], W0[i]);
                mb[i] = f2add(m[i], mi[i]);
            }
            float2 wl, wr, ml, mr;
            whalo<CS>(w, wl, wr);
            whalo<CS>(mb, ml, mr);
            float2 gp = f2add(ml, mb[0]);
#pragma unroll
            for (int i = 0; i < CS; ++i) {
                const float2 wprev = (i == 0) ? wl : w[i - 1];
                const float2 wnext = (i == CS - 1) ? wr : w[i + 1];
                const float2 g = f2add(mb[i], (i == CS - 1) ? mr : mb[i + 1]);
                x[i] = f2sub(f2fma(wprev, gp, R0sm[i * 32 + lane]), f2mul(wnext, g));
                gp = g;
            }
        }
        // (M + mu dt/2 K) m_new = rhs
        float2 pd, de, E, F;
        float Ep, Fn;
        wsweep<CS>(W.pic, x, pd, de);
        wreduced(W.pic, W.rpic, pd, de, E, F, Ep, Fn);
        float2 mn[CS];
        wback<CS>(W.pic, x, F, E, mn);
        float dmax = 0.f, mmax = 0.f;
#pragma unroll
        for (int i = 0; i < CS; ++i) {
            const float2 d = f2sub(mn[i], mi[i]);
            dmax = fmax3_nan(dmax, fabsf(d.x), fabsf(d.y));
            mmax = fmaxf(mmax, fmaxf(fabsf(mn[i].x), fabsf(mn[i].y)));
            mi[i] = mn[i];
        }
        // u_new = H^{-1} M m_new, the mass product's chunk ends from the reduced solve
        {
            const float2 lo = make_float2(Ep, E.x), hi = make_float2(F.y, Fn);
            const float2 four = f2b(4.f);
#pragma unroll
            for (int i = 0; i < CS; ++i) {
                const float2 l = (i == 0) ? lo : mn[i - 1];
                const float2 r = (i == CS - 1) ? hi : mn[i + 1];
                x[i] = f2fma(four, mn[i], f2add(l, r));
            }
            float2 hpd, hde, hE, hF;
            float hEp, hFn;
            wsweep<CS>(W.hel, x, hpd, hde);
            wreduced(W.hel, W.rhel, hpd, hde, hE, hF, hEp, hFn);
            wback<CS>(W.hel, x, hF, hE, u);
        }
        iters++;
        const float dm = warp_max_nan(dmax);
        const float mm = warp_max_nan(mmax);
        if (!(dm < INFINITY) || !(mm < INFINITY)) {
            flags |= SCH_DEV_NONFINITE;
            break;
        }
        if (dm <= A.tol * fmaxf(1.f, mm)) break;
        if (it >= A.max_iter) {
            flags |= SCH_DEV_NOCONVERGE;
            break;
        }
    }
#pragma unroll
    for (int i = 0; i < CS; ++i) m[i] = mi[i];
}

// this lane's 2 CS nodes of a particle row <-> the paired registers
template <int CS>
__device__ __forceinline__ void wload(const float* row, float2 (&v)[CS]) {
    const float4* p = reinterpret_cast<const float4*>(row + (threadIdx.x & 31) * 2 * CS);
#pragma unroll
    for (int q = 0; q < CS / 4; ++q) {
        const float4 a = p[q], b = p[CS / 4 + q];
        v[4 * q + 0] = make_float2(a.x, b.x);
        v[4 * q + 1] = make_float2(a.y, b.y);
        v[4 * q + 2] = make_float2(a.z, b.z);
        v[4 * q + 3] = make_float2(a.w, b.w);
    }
}

template <int CS>
__device__ __forceinline__ void wstore(float* row, const float2 (&v)[CS]) {
    float4* p = reinterpret_cast<float4*>(row + (threadIdx.x & 31) * 2 * CS);
#pragma unroll
    for (int q = 0; q < CS / 4; ++q) {
        p[q] = make_float4(v[4 * q].x, v[4 * q + 1].x, v[4 * q + 2].x, v[4 * q + 3].x);
        p[CS / 4 + q] = make_float4(v[4 * q].y, v[4 * q + 1].y, v[4 * q + 2].y, v[4 * q + 3].y);
    }
}

// observation misfit sum_j ((u(x_j) - y_j) / sigma)^2 over this lane's nodes;
// node mod stride and the observation index advance node by node
template <int CS>
__device__ __forceinline__ double wmisfit(const ModelArgs<float>& A, const float2 (&u)[CS], const float* y) {
    const int base = (threadIdx.x & 31) * 2 * CS;
    double acc = 0.0;
    int rem = base % A.stride;
    int j = base / A.stride + (rem != 0);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int i = 0; i < CS; ++i) {
            if (rem == 0) {
                const float r = ((c ? u[i].y : u[i].x) - y[j]) * A.sigma_inv;
                acc += (double)r * (double)r;
                ++j;
            }
            rem = (rem + 1 == A.stride) ? 0 : rem + 1;
        }
    }
    return acc;
}

// sin and cos of the angles of this lane's first X and Y nodes
template <int CS>
__device__ __forceinline__ void wangles(int n, float2& s1, float2& c1) {
    const int base = (threadIdx.x & 31) * 2 * CS;
    float sx, cx, sy, cy;
    node_angle<float>(base, n, sx, cx);
    node_angle<float>(base + CS, n, sy, cy);
    s1 = make_float2(sx, sy);
    c1 = make_float2(cx, cy);
}

template <int CS>
__host__ __device__ constexpr size_t wsmem_base() {
    return (size_t)CS * 32 * sizeof(float2);
}

// Occupancy: 8 one-warp CTAs per SM (255 registers a thread)
constexpr int WMINB = 8;

template <int CS>
__global__ void __launch_bounds__(32, WMINB) wwindow_kernel(ModelArgs<float> A, WArgs W, WindowIO<float> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* R0sm = reinterpret_cast<float2*>(smem_raw);
    float* noise = reinterpret_cast<float*>(smem_raw + wsmem_base<CS>());
    const int p = blockIdx.x;
    const size_t NK = (size_t)io.Ns * A.K;
    stage_noise(A, noise, io.dW + p * NK, io.lam ? io.lam + p * NK : nullptr, io.Ns);
    float2 s1, c1;
    wangles<CS>(A.n, s1, c1);
    float2 m[CS], u[CS];
    wload<CS>(io.m_in + (size_t)p * A.n, m);
    wu_from_m<CS>(W, m, u);
    __syncwarp();
    int iters = 0, flags = 0;
    for (int s = 0; s < io.Ns; ++s) wstep<CS>(A, W, m, u, R0sm, noise + s * A.K, s1, c1, iters, flags);
    wstore<CS>(io.m_out + (size_t)p * A.n, m);
    wstore<CS>(io.u_out + (size_t)p * A.n, u);
    if (io.y) {
        double mis = warp_sum(wmisfit<CS>(A, u, io.y));
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
template <int CS>
__global__ void __launch_bounds__(32, WMINB) wjitter_kernel(ModelArgs<float> A, WArgs W, JitterIO<float> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* R0sm = reinterpret_cast<float2*>(smem_raw);
    const int p = blockIdx.x;
    const int lane = threadIdx.x;
    const int Ns = io.Ns, K = A.K, NK = Ns * K;
    float* noise = reinterpret_cast<float*>(smem_raw + wsmem_base<CS>());
    float* cur = noise + NK;
    float* prop = noise + 2 * NK;
    float* dW = io.dW + (size_t)p * NK;
    const float* lam = io.lam ? io.lam + (size_t)p * NK : nullptr;
    for (int q = lane; q < NK; q += 32) cur[q] = dW[q];
    double nll0 = io.nll[p], lg0 = io.logG ? io.logG[p] : 0.0;
    float2 s1, c1;
    wangles<CS>(A.n, s1, c1);
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
        float2 m[CS], u[CS];
        wload<CS>(io.m_start + (size_t)p * A.n, m);
        wu_from_m<CS>(W, m, u);
        __syncwarp();
        int fl = 0;
        for (int s = 0; s < Ns; ++s) wstep<CS>(A, W, m, u, R0sm, noise + s * K, s1, c1, iters, fl);
        const double mis = warp_sum(wmisfit<CS>(A, u, io.y));
        const double gl = warp_sum(window_girsanov(A, prop, lam, Ns));
        const double nll1 = 0.5 * mis, lg1 = -gl;
        int acc = 0;
        if (lane == 0) {
            const double w0 = io.theta * (nll0 - lg0);
            const double w1 = io.theta * (nll1 - lg1);
            const double logU = log(uniform_open0(io.seed, SCH_TAG_PCN_ACCEPT, (uint64_t)(io.particle0 + p), ctr));
            acc = (fl == 0) && (logU < w0 - w1);
        }
        acc = __shfl_sync(FULL, acc, 0);
        if (acc) {
            nll0 = nll1;
            lg0 = lg1;
            for (int q = lane; q < NK; q += 32) cur[q] = prop[q];
            wstore<CS>(io.m_end + (size_t)p * A.n, m);
            wstore<CS>(io.u_end + (size_t)p * A.n, u);
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
