// Ensemble propagation of the viscous stochastic Camassa-Holm (SALT) equation
// on sm_103a: one CTA per particle, the whole periodic field held in
// registers across the steps of an assimilation window.
//
// Discretisation (Sec. 2 of the paper): P1 elements on n uniform periodic
// cells, Helmholtz relation (M + alpha^2 K) u = M m (Eq. sde1), implicit
// midpoint step (Eq. fde1):
//   M (m1 - m0) + mu dt K mbar + A(mbar, dv) = 0,
//   mbar = (m0 + m1)/2,  dv = dt (u0 + u1)/2 + dU,
// with the exact P1 advection operator
//   A(m, v)_i = 1/2 [ v_{i+1} (m_i + m_{i+1}) - v_{i-1} (m_{i-1} + m_i) ].
// Each step is solved by a linearly implicit Picard iteration: with dv frozen
// at the last iterate, the cyclic tridiagonal system
//   (M + mu dt/2 K + 1/2 A_dv) m1 = (M - mu dt/2 K - 1/2 A_dv) m0
// is solved, then u1 = H^{-1} M m1, until max|m1 - m1_prev| <= tol max(1, max|m1|).
//
// Thread t owns nodes [tC, tC + C).  Cyclic tridiagonal systems are solved by
// a partition method: each thread eliminates its chunk interior with a
// forward and a backward sweep, leaving one "first" and one "last" unknown per
// chunk; the first unknowns are eliminated locally, and the remaining cyclic
// system of one unknown per thread is solved by parallel cyclic reduction in
// shared memory.  For the constant Helmholtz matrix all sweep coefficients are
// the same in every chunk and are tabulated once per CTA.
#include "sch_internal.h"

namespace sch {

// --------------------------------------------------------------------------
// shared-memory layout of one particle CTA
// --------------------------------------------------------------------------
template <typename R, int C>
struct ConstTab {
    R rden[C], gam[C], alpp[C], gamp[C];
    R a, iBF, pa, pc, ae, ge;
    R k1[12], k2[12], f1, f2;
};

template <typename R, int C>
struct Smem {
    unsigned char* exch;
    Row4<R>* pcr;       // 2 * tp rows
    R* dbuf;            // 2 * tp values
    ConstTab<R, C>* hel;  // Helmholtz: (M + alpha^2 K)
    ConstTab<R, C>* aux;  // second constant system (mass or smoothing)
    R* noise;           // Ns * K weights of the current window
    R* extra;           // jitter: proposal noise (Ns * K) and drift (Ns * K)
};

template <typename R, int C>
__host__ __device__ inline size_t smem_bytes(int tp, int Ns, int K) {
    size_t b = EXCH_BYTES;
    b += 2 * (size_t)tp * sizeof(Row4<R>);
    b += 2 * (size_t)tp * sizeof(R);
    b += 2 * ((sizeof(ConstTab<R, C>) + 15) / 16 * 16);
    b += 3 * (size_t)Ns * K * sizeof(R);
    return (b + 15) / 16 * 16;
}

template <typename R, int C>
__device__ inline Smem<R, C> carve(unsigned char* base, int tp, int Ns, int K) {
    Smem<R, C> s;
    s.exch = base;
    base += EXCH_BYTES;
    s.pcr = reinterpret_cast<Row4<R>*>(base);
    base += 2 * (size_t)tp * sizeof(Row4<R>);
    s.dbuf = reinterpret_cast<R*>(base);
    base += 2 * (size_t)tp * sizeof(R);
    s.hel = reinterpret_cast<ConstTab<R, C>*>(base);
    base += (sizeof(ConstTab<R, C>) + 15) / 16 * 16;
    s.aux = reinterpret_cast<ConstTab<R, C>*>(base);
    base += (sizeof(ConstTab<R, C>) + 15) / 16 * 16;
    s.noise = reinterpret_cast<R*>(base);
    base += (size_t)Ns * K * sizeof(R);
    s.extra = reinterpret_cast<R*>(base);
    return s;
}

// --------------------------------------------------------------------------
// Constant symmetric circulant tridiagonal system (off-diagonal a, diagonal b):
// tabulate the chunk sweep and the reduced-system PCR coefficients.
// Called by one thread.
// --------------------------------------------------------------------------
template <typename R, int C>
__device__ void build_const(ConstTab<R, C>* T, R a, R b, int tp) {
    R al[C], ga[C];
    al[0] = R(-1);
    ga[0] = R(0);
    T->rden[0] = R(0);
    T->gam[0] = R(0);
#pragma unroll
    for (int i = 1; i < C; ++i) {
        const R r = R(1) / (b - a * ga[i - 1]);
        T->rden[i] = r;
        ga[i] = a * r;
        al[i] = -a * al[i - 1] * r;
        T->gam[i] = ga[i];
    }
    R ap = R(0), gp = R(-1);
    T->alpp[C - 1] = ap;
    T->gamp[C - 1] = gp;
    T->alpp[0] = R(0);
    T->gamp[0] = R(0);
#pragma unroll
    for (int i = C - 2; i >= 1; --i) {
        ap = al[i] - ga[i] * ap;
        gp = -ga[i] * gp;
        T->alpp[i] = ap;
        T->gamp[i] = gp;
    }
    R BF, CF;
    if (C == 2) {
        BF = b;
        CF = a;
    } else {
        BF = b - a * T->alpp[1];
        CF = -a * T->gamp[1];
    }
    T->a = a;
    T->iBF = R(1) / BF;
    T->pa = a * T->iBF;
    T->pc = CF * T->iBF;
    T->ae = al[C - 1];
    T->ge = ga[C - 1];
    R A = -T->ae * T->pa;
    R B = R(1) - T->ae * T->pc - T->ge * T->pa;
    R Cc = -T->ge * T->pc;
    int l = 0;
    for (int s = 1; s < (tp >> 1); s <<= 1, ++l) {
        const R k1 = A / B, k2 = Cc / B;
        T->k1[l] = k1;
        T->k2[l] = k2;
        const R nB = B - Cc * k1 - A * k2;
        A = -A * k1;
        Cc = -Cc * k2;
        B = nB;
    }
    const R e = A + Cc;
    const R det = B * B - e * e;
    T->f1 = B / det;
    T->f2 = -e / det;
}

// x = T^{-1} r for the tabulated constant system; r, x: this thread's chunk.
template <typename R, int C>
__device__ __forceinline__ void solve_const(const ConstTab<R, C>* T, const R (&r)[C], R (&x)[C],
                                            Exch& ex, R* dbuf) {
    const R a = T->a;
    R de[C];
    de[0] = R(0);
#pragma unroll
    for (int i = 1; i < C; ++i) de[i] = (r[i] - a * de[i - 1]) * T->rden[i];
    R dp[C];
    dp[C - 1] = R(0);
#pragma unroll
    for (int i = C - 2; i >= 1; --i) dp[i] = de[i] - T->gam[i] * dp[i + 1];
    const R DF = (C == 2) ? r[0] : r[0] - a * dp[1];
    const R pd = DF * T->iBF;
    R mine[1] = {pd}, nxt[1];
    from_next<R, 1>(ex, mine, nxt);
    const R D = de[C - 1] - T->ae * pd - T->ge * nxt[0];
    const R E = pcr_cyclic_const<R>(D, T->k1, T->k2, T->f1, T->f2, dbuf, ex.tp);
    R Eprev, Enext;
    both_neighbours(ex, E, Eprev, Enext);
    const R F = pd - T->pa * Eprev - T->pc * E;
    x[0] = F;
    x[C - 1] = E;
#pragma unroll
    for (int i = 1; i < C - 1; ++i) x[i] = dp[i] - T->alpp[i] * F - T->gamp[i] * E;
}

// u = H^{-1} M m for this thread's chunk
template <typename R, int C>
__device__ __forceinline__ void helmholtz(const ModelArgs<R>& A, const Smem<R, C>& S, Exch& ex,
                                          const R (&m)[C], R (&u)[C]) {
    R mp, mn;
    halo(ex, m[0], m[C - 1], mp, mn);
    R r[C];
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const R lo = (i == 0) ? mp : m[i - 1];
        const R hi = (i == C - 1) ? mn : m[i + 1];
        r[i] = A.h6 * (lo + R(4) * m[i] + hi);
    }
    solve_const<R, C>(S.hel, r, u, ex, S.dbuf);
}

// --------------------------------------------------------------------------
// One implicit-midpoint step for this thread's chunk.
// wq: the K noise weights of the step, already scaled by a_j / 4.
// --------------------------------------------------------------------------
template <typename R, int C>
__device__ __forceinline__ void sch_step(const ModelArgs<R>& A, const Smem<R, C>& S, Exch& ex,
                                         R (&m)[C], R (&u)[C], const R* wq, const R (&sn)[C],
                                         const R (&cs)[C], int& iters, int& flags) {
    // SALT increment dU/4 at the nodes (Chebyshev recurrence over harmonics)
    R W0[C];
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const R c2 = R(2) * cs[i];
        R sk = sn[i], ck = cs[i], sp = R(0), cp = R(1);
        R acc = R(0);
        for (int j = 0; j < A.K2; ++j) {
            acc += wq[2 * j] * sk + wq[2 * j + 1] * ck;
            const R s2 = c2 * sk - sp;
            const R k2 = c2 * ck - cp;
            sp = sk; cp = ck; sk = s2; ck = k2;
        }
        W0[i] = A.dt8 * u[i] + acc;
    }
    // per-step constants from m0: S_i = m_i + m_{i+1}; D0_i = c0p (m_{i-1} + m_{i+1}) + b0p m_i
    R mp, mn;
    halo(ex, m[0], m[C - 1], mp, mn);
    R Ssum[C], D0[C];
    const R Sprev = mp + m[0];
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const R lo = (i == 0) ? mp : m[i - 1];
        const R hi = (i == C - 1) ? mn : m[i + 1];
        Ssum[i] = m[i] + hi;
        D0[i] = A.c0p * (lo + hi) + A.b0p * m[i];
    }
    R mi[C], ui[C];
#pragma unroll
    for (int i = 0; i < C; ++i) { mi[i] = m[i]; ui[i] = u[i]; }

    for (int it = 1; it <= A.max_iter; ++it) {
        // w = dv / 4 at the current iterate
        R w[C];
#pragma unroll
        for (int i = 0; i < C; ++i) w[i] = W0[i] + A.dt8 * ui[i];
        R wp, wn;
        halo(ex, w[0], w[C - 1], wp, wn);
        // row i: a_i = c0 - w_{i-1}, c_i = c0 + w_{i+1}, b_i = b0 + w_{i+1} - w_{i-1},
        //        d_i = D0_i + w_{i-1} S_{i-1} - w_{i+1} S_i
        R al[C], ga[C], de[C];
        R a0, b0, c0, d0;
        {
            const R wl = wp, wr = (C > 1) ? w[1] : wn;
            a0 = A.c0 - wl;
            c0 = A.c0 + wr;
            b0 = A.b0 + wr - wl;
            d0 = D0[0] + wl * Sprev - wr * Ssum[0];
        }
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
            const R r = rcp(bi - ai * ga[i - 1]);
            ga[i] = ci * r;
            al[i] = -ai * al[i - 1] * r;
            de[i] = (di - ai * de[i - 1]) * r;
        }
        const R ae = al[C - 1], ge = ga[C - 1], dee = de[C - 1];
        // backward sweep: x_i = de_i - al_i F - ga_i E for interior rows
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
        const R pa = a0 * qF, pc = CF * qF, pd = DF * qF;
        R mine[3] = {pa, pc, pd}, nx[3];
        from_next<R, 3>(ex, mine, nx);
        const R RA = -ae * pa;
        const R RB = R(1) - ae * pc - ge * nx[0];
        const R RC = -ge * nx[1];
        const R RD = dee - ae * pd - ge * nx[2];
        const R E = pcr_cyclic<R>(RA, RB, RC, RD, S.pcr, ex.tp);
        R Ep, En;
        both_neighbours(ex, E, Ep, En);
        const R F = pd - pa * Ep - pc * E;
        R mnew[C];
        mnew[0] = F;
        mnew[C - 1] = E;
#pragma unroll
        for (int i = 1; i < C - 1; ++i) mnew[i] = de[i] - al[i] * F - ga[i] * E;
        // u at the new iterate
        R unew[C];
        helmholtz<R, C>(A, S, ex, mnew, unew);
        // convergence
        R dmax = R(0), mmax = R(0);
#pragma unroll
        for (int i = 0; i < C; ++i) {
            R dd = rabs(mnew[i] - mi[i]);
            if (!(dd == dd)) dd = R(INFINITY);
            dmax = fmax(dmax, dd);
            mmax = fmax(mmax, rabs(mnew[i]));
            mi[i] = mnew[i];
            ui[i] = unew[i];
        }
        block_max2(ex, dmax, mmax);
        iters++;
        if (!(dmax < R(INFINITY)) || !(mmax < R(INFINITY))) {
            flags |= SCH_DEV_NONFINITE;
            break;
        }
        if (dmax <= A.tol * fmax(R(1), mmax)) break;
        if (it == A.max_iter) flags |= SCH_DEV_NOCONVERGE;
    }
#pragma unroll
    for (int i = 0; i < C; ++i) { m[i] = mi[i]; u[i] = ui[i]; }
}

// load the Ns * K noise weights a_j/4 (dW + lambda dt) of a window into smem
template <typename R>
__device__ __forceinline__ void stage_noise(const ModelArgs<R>& A, R* dst, const R* dW, const R* lam,
                                            int Ns) {
    const int tot = Ns * A.K;
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
        const int k = q % A.K;
        R v = dW[q];
        if (lam) v += lam[q] * A.dt;
        dst[q] = A.amp4[k >> 1] * v;
    }
}

// the node angle sin/cos for this thread's chunk
template <typename R, int C>
__device__ __forceinline__ void node_trig(const ModelArgs<R>& A, int i0, R (&sn)[C], R (&cs)[C]) {
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const R t = R(2) * R(i0 + i) / R(A.n);
        sincospi(t, &sn[i], &cs[i]);
    }
}

// observation misfit of this thread's chunk (double)
template <typename R, int C>
__device__ __forceinline__ double chunk_misfit(const ModelArgs<R>& A, int i0, const R (&u)[C],
                                               const R* y) {
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const int node = i0 + i;
        if (node % A.stride == 0) {
            const R r = (u[i] - y[node / A.stride]) * A.sigma_inv;
            acc += (double)r * (double)r;
        }
    }
    return acc;
}

// Girsanov log-weight -sum (lambda dW + 1/2 lambda^2 dt) of a window (double)
template <typename R>
__device__ __forceinline__ double window_logG(const ModelArgs<R>& A, Exch& ex, const R* dW,
                                              const R* lam, int Ns) {
    double acc = 0.0;
    if (lam) {
        const int tot = Ns * A.K;
        for (int q = threadIdx.x; q < tot; q += blockDim.x) {
            const double l = lam[q], w = dW[q];
            acc += l * w + 0.5 * l * l * A.dt_d;
        }
    }
    return -block_sum(ex, acc);
}

template <typename R, int C>
__device__ __forceinline__ void load_chunk(const R* src, R (&v)[C]) {
#pragma unroll
    for (int i = 0; i < C; ++i) v[i] = src[i];
}
template <typename R, int C>
__device__ __forceinline__ void store_chunk(R* dst, const R (&v)[C]) {
#pragma unroll
    for (int i = 0; i < C; ++i) dst[i] = v[i];
}

// --------------------------------------------------------------------------
// kernels
// --------------------------------------------------------------------------
template <typename R, int C>
__global__ void __launch_bounds__(512) window_kernel(ModelArgs<R> A, WindowIO<R> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = blockIdx.x;
    const int tp = blockDim.x;
    Smem<R, C> S = carve<R, C>(smem_raw, tp, io.Ns, A.K);
    Exch ex{S.exch, 0, tp};
    if (threadIdx.x == 0) build_const<R, C>(S.hel, A.hel_a, A.hel_b, tp);
    stage_noise(A, S.noise, io.dW + (size_t)p * io.Ns * A.K,
                io.lam ? io.lam + (size_t)p * io.Ns * A.K : nullptr, io.Ns);
    __syncthreads();
    const int i0 = threadIdx.x * C;
    R m[C], u[C], sn[C], cs[C];
    load_chunk<R, C>(io.m_in + (size_t)p * A.n + i0, m);
    node_trig<R, C>(A, i0, sn, cs);
    helmholtz<R, C>(A, S, ex, m, u);
    int iters = 0, flags = 0;
    for (int s = 0; s < io.Ns; ++s)
        sch_step<R, C>(A, S, ex, m, u, S.noise + s * A.K, sn, cs, iters, flags);
    store_chunk<R, C>(io.m_out + (size_t)p * A.n + i0, m);
    store_chunk<R, C>(io.u_out + (size_t)p * A.n + i0, u);
    if (io.y) {
        const double mis = block_sum(ex, chunk_misfit<R, C>(A, i0, u, io.y));
        const double lg = window_logG(A, ex, io.dW + (size_t)p * io.Ns * A.K,
                                      io.lam ? io.lam + (size_t)p * io.Ns * A.K : nullptr, io.Ns);
        if (threadIdx.x == 0) {
            io.nll[p] = 0.5 * mis;
            if (io.logG) io.logG[p] = lg;
        }
    }
    if (threadIdx.x == 0) {
        if (io.iters) io.iters[p] = iters;
        if (io.status) io.status[p] = flags;
    }
}

// PCN jittering: n_iter proposals of the window noise, each re-run through the
// whole window from m_start and accepted with probability min(1, exp(w0 - w1)).
template <typename R, int C>
__global__ void __launch_bounds__(512) jitter_kernel(ModelArgs<R> A, JitterIO<R> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = blockIdx.x;
    const int tp = blockDim.x;
    const int Ns = io.Ns, K = A.K, NK = Ns * K;
    Smem<R, C> S = carve<R, C>(smem_raw, tp, Ns, K);
    Exch ex{S.exch, 0, tp};
    R* cur = S.extra;          // current dW (Ns * K)
    R* prop = S.extra + NK;    // proposal dW
    R* dW = io.dW + (size_t)p * NK;
    const R* lam = io.lam ? io.lam + (size_t)p * NK : nullptr;
    if (threadIdx.x == 0) build_const<R, C>(S.hel, A.hel_a, A.hel_b, tp);
    for (int q = threadIdx.x; q < NK; q += blockDim.x) cur[q] = dW[q];
    __shared__ double sh_state[4];
    __shared__ int sh_acc;
    if (threadIdx.x == 0) {
        sh_state[0] = io.nll[p];
        sh_state[1] = io.logG ? io.logG[p] : 0.0;
    }
    __syncthreads();
    const int i0 = threadIdx.x * C;
    R sn[C], cs[C];
    node_trig<R, C>(A, i0, sn, cs);
    const R sq = io.sq1mr2 * (R)sqrt(A.dt_d);
    int iters = 0, flags = 0, n_acc = 0, changed = 0;
    for (int j = 0; j < io.n_iter; ++j) {
        const uint64_t ctr = io.ctr + (uint64_t)j;
        // proposal dW' = rho dW + sqrt(1 - rho^2) sqrt(dt) z
        const int nblk = (K + 3) >> 2;
        for (int q = threadIdx.x; q < Ns * nblk; q += blockDim.x) {
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
        stage_noise(A, S.noise, prop, lam, Ns);
        __syncthreads();
        R m[C], u[C];
        load_chunk<R, C>(io.m_start + (size_t)p * A.n + i0, m);
        helmholtz<R, C>(A, S, ex, m, u);
        int fl = 0;
        for (int s = 0; s < Ns; ++s)
            sch_step<R, C>(A, S, ex, m, u, S.noise + s * K, sn, cs, iters, fl);
        const double mis = block_sum(ex, chunk_misfit<R, C>(A, i0, u, io.y));
        const double lg = window_logG(A, ex, prop, lam, Ns);
        if (threadIdx.x == 0) {
            const double nll1 = 0.5 * mis;
            const double w0 = io.theta * (sh_state[0] - sh_state[1]);
            const double w1 = io.theta * (nll1 - lg);
            const double logU = log(uniform_open0(io.seed, SCH_TAG_PCN_ACCEPT,
                                                  (uint64_t)(io.particle0 + p), ctr));
            const int acc = (fl == 0) && (logU < w0 - w1);
            sh_acc = acc;
            if (acc) {
                sh_state[0] = nll1;
                sh_state[1] = lg;
            }
        }
        __syncthreads();
        if (sh_acc) {
            for (int q = threadIdx.x; q < NK; q += blockDim.x) cur[q] = prop[q];
            store_chunk<R, C>(io.m_end + (size_t)p * A.n + i0, m);
            store_chunk<R, C>(io.u_end + (size_t)p * A.n + i0, u);
            n_acc++;
            changed = 1;
        }
        flags |= fl;
        __syncthreads();
    }
    if (changed)
        for (int q = threadIdx.x; q < NK; q += blockDim.x) dW[q] = cur[q];
    if (threadIdx.x == 0) {
        io.nll[p] = sh_state[0];
        if (io.logG) io.logG[p] = sh_state[1];
        if (io.accepts) io.accepts[p] = n_acc;
        if (io.iters) io.iters[p] = iters;
        if (io.status) io.status[p] = flags;
    }
}

// Helmholtz utilities: mode 0: u = H^{-1} M m ; mode 1: m = M^{-1} H u
template <typename R, int C>
__global__ void __launch_bounds__(512) helm_kernel(ModelArgs<R> A, const R* in, R* out, int mode) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = blockIdx.x;
    const int tp = blockDim.x;
    Smem<R, C> S = carve<R, C>(smem_raw, tp, 0, A.K);
    Exch ex{S.exch, 0, tp};
    if (threadIdx.x == 0) {
        build_const<R, C>(S.hel, A.hel_a, A.hel_b, tp);
        build_const<R, C>(S.aux, A.h6, R(4) * A.h6, tp);
    }
    __syncthreads();
    const int i0 = threadIdx.x * C;
    R v[C], w[C];
    load_chunk<R, C>(in + (size_t)p * A.n + i0, v);
    if (mode == 0) {
        helmholtz<R, C>(A, S, ex, v, w);
    } else {
        R vp, vn, r[C];
        halo(ex, v[0], v[C - 1], vp, vn);
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const R lo = (i == 0) ? vp : v[i - 1];
            const R hi = (i == C - 1) ? vn : v[i + 1];
            r[i] = A.hel_a * (lo + hi) + A.hel_b * v[i];
        }
        solve_const<R, C>(S.aux, r, w, ex, S.dbuf);
    }
    store_chunk<R, C>(out + (size_t)p * A.n + i0, w);
}

// Prior ensemble: u = u_truth + scale (a_p S^3 W_p + b_p), S the P1 solve of
// (U, v) + (U_x, v_x) = (f, v); then m = M^{-1} H u.
template <typename R, int C>
__global__ void __launch_bounds__(512) prior_kernel(ModelArgs<R> A, const R* u_truth, uint64_t seed,
                                                     R scale, R* m_out, R* u_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = blockIdx.x;
    const int tp = blockDim.x;
    Smem<R, C> S = carve<R, C>(smem_raw, tp, 0, A.K);
    Exch ex{S.exch, 0, tp};
    const R h = A.h;
    if (threadIdx.x == 0) {
        // smoothing operator M + K: off-diagonal h/6 - 1/h, diagonal 2h/3 + 2/h
        build_const<R, C>(S.hel, A.h6 - R(1) / h, R(4) * A.h6 + R(2) / h, tp);
        build_const<R, C>(S.aux, A.h6, R(4) * A.h6, tp);
    }
    __syncthreads();
    const int i0 = threadIdx.x * C;
    // cell values W_e = sqrt(h) z_e for cells e = i0 .. i0 + C - 1 (cell e = [x_e, x_{e+1}])
    R cell[C];
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const int e = i0 + i;
        R z[4];
        normal4<R>(seed, SCH_TAG_INIT, (uint64_t)(e >> 2), 0, (uint64_t)p, 0, z);
        cell[i] = (R)sqrt((double)h) * z[e & 3];
    }
    R ab[2];
    {
        R z[4];
        const int k0 = A.n;
        normal4<R>(seed, SCH_TAG_INIT, (uint64_t)(k0 >> 2), 0, (uint64_t)p, 0, z);
        ab[0] = z[k0 & 3];
        R z2[4];
        normal4<R>(seed, SCH_TAG_INIT, (uint64_t)((k0 + 1) >> 2), 0, (uint64_t)p, 0, z2);
        ab[1] = z2[(k0 + 1) & 3];
    }
    // rhs (W, phi_i) = h/2 (W_{i-1} + W_i)
    R cp, cn, r[C], U[C];
    halo(ex, cell[0], cell[C - 1], cp, cn);
#pragma unroll
    for (int i = 0; i < C; ++i) r[i] = R(0.5) * h * (((i == 0) ? cp : cell[i - 1]) + cell[i]);
    solve_const<R, C>(S.hel, r, U, ex, S.dbuf);
    for (int rep = 0; rep < 2; ++rep) {
        R up, un;
        halo(ex, U[0], U[C - 1], up, un);
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const R lo = (i == 0) ? up : U[i - 1];
            const R hi = (i == C - 1) ? un : U[i + 1];
            r[i] = A.h6 * (lo + R(4) * U[i] + hi);
        }
        solve_const<R, C>(S.hel, r, U, ex, S.dbuf);
    }
    R u[C];
#pragma unroll
    for (int i = 0; i < C; ++i) u[i] = u_truth[i0 + i] + scale * (ab[0] * U[i] + ab[1]);
    // m = M^{-1} H u
    R up, un;
    halo(ex, u[0], u[C - 1], up, un);
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const R lo = (i == 0) ? up : u[i - 1];
        const R hi = (i == C - 1) ? un : u[i + 1];
        r[i] = A.hel_a * (lo + hi) + A.hel_b * u[i];
    }
    R m[C];
    solve_const<R, C>(S.aux, r, m, ex, S.dbuf);
    store_chunk<R, C>(m_out + (size_t)p * A.n + i0, m);
    store_chunk<R, C>(u_out + (size_t)p * A.n + i0, u);
}

// dW[p][s][k] = sqrt(dt) z, z from block (k/4, s, particle0 + p, ctr)
template <typename R>
__global__ void draw_kernel(int N, int Ns, int K, R sqdt, uint64_t seed, uint64_t tag, uint64_t ctr,
                            int particle0, R* dW) {
    const int nblk = (K + 3) >> 2;
    const long long tot = (long long)N * Ns * nblk;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot;
         q += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(q % nblk);
        const int s = (int)((q / nblk) % Ns);
        const int p = (int)(q / ((long long)nblk * Ns));
        R z[4];
        normal4<R>(seed, tag, (uint64_t)b, (uint64_t)s, (uint64_t)(particle0 + p), ctr, z);
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
        const R r = (up[j * A.stride] - y[j]) * A.sigma_inv;
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

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------
template <typename R, int C>
int launch_window(const ModelArgs<R>& A, const WindowIO<R>& io, int N, cudaStream_t st) {
    const int tp = A.n / C;
    const size_t sm = smem_bytes<R, C>(tp, io.Ns, A.K);
    if (sm > 48 * 1024)
        cudaFuncSetAttribute(window_kernel<R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    window_kernel<R, C><<<N, tp, sm, st>>>(A, io);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

template <typename R, int C>
int launch_jitter(const ModelArgs<R>& A, const JitterIO<R>& io, int N, cudaStream_t st) {
    const int tp = A.n / C;
    const size_t sm = smem_bytes<R, C>(tp, io.Ns, A.K);
    if (sm > 48 * 1024)
        cudaFuncSetAttribute(jitter_kernel<R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    jitter_kernel<R, C><<<N, tp, sm, st>>>(A, io);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

template <typename R, int C>
int launch_helm(const ModelArgs<R>& A, const R* in, R* out, int mode, int N, cudaStream_t st) {
    const int tp = A.n / C;
    const size_t sm = smem_bytes<R, C>(tp, 0, A.K);
    if (sm > 48 * 1024)
        cudaFuncSetAttribute(helm_kernel<R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    helm_kernel<R, C><<<N, tp, sm, st>>>(A, in, out, mode);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

template <typename R, int C>
int launch_prior(const ModelArgs<R>& A, const R* u_truth, uint64_t seed, R scale, R* m, R* u, int N,
                 cudaStream_t st) {
    const int tp = A.n / C;
    const size_t sm = smem_bytes<R, C>(tp, 0, A.K);
    if (sm > 48 * 1024)
        cudaFuncSetAttribute(prior_kernel<R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    prior_kernel<R, C><<<N, tp, sm, st>>>(A, u_truth, seed, scale, m, u);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

template <typename R>
int launch_draw(int N, int Ns, int K, R sqdt, uint64_t seed, uint64_t tag, uint64_t ctr, int particle0,
                R* dW, cudaStream_t st) {
    const long long tot = (long long)N * Ns * ((K + 3) / 4);
    const int threads = 256;
    long long blocks = (tot + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    draw_kernel<R><<<(int)blocks, threads, 0, st>>>(N, Ns, K, sqdt, seed, tag, ctr, particle0, dW);
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

#define SCH_INSTANTIATE(R, C)                                                                        \
    template int launch_window<R, C>(const ModelArgs<R>&, const WindowIO<R>&, int, cudaStream_t);    \
    template int launch_jitter<R, C>(const ModelArgs<R>&, const JitterIO<R>&, int, cudaStream_t);    \
    template int launch_helm<R, C>(const ModelArgs<R>&, const R*, R*, int, int, cudaStream_t);       \
    template int launch_prior<R, C>(const ModelArgs<R>&, const R*, uint64_t, R, R*, R*, int,         \
                                    cudaStream_t);

SCH_INSTANTIATE(float, 8)
SCH_INSTANTIATE(double, 4)

template int launch_draw<float>(int, int, int, float, uint64_t, uint64_t, uint64_t, int, float*, cudaStream_t);
template int launch_draw<double>(int, int, int, double, uint64_t, uint64_t, uint64_t, int, double*,
                                 cudaStream_t);
template int launch_loglik<float>(const ModelArgs<float>&, int, const float*, const float*, const float*,
                                  const float*, int, double*, double*, cudaStream_t);
template int launch_loglik<double>(const ModelArgs<double>&, int, const double*, const double*,
                                   const double*, const double*, int, double*, double*, cudaStream_t);

template <typename R, int C>
size_t window_smem(int tp, int Ns, int K) { return smem_bytes<R, C>(tp, Ns, K); }
template size_t window_smem<float, 8>(int, int, int);
template size_t window_smem<double, 4>(int, int, int);

// y_j = u(x_j) + sigma z_j, z_j keyed (seed, SCH_TAG_OBS, (j / 4, 0, 0, ctr))
template <typename R>
__global__ void synth_obs_kernel(ModelArgs<R> A, const R* u, uint64_t seed, uint64_t ctr, R sigma, R* y) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= A.M) return;
    R z[4];
    normal4<R>(seed, SCH_TAG_OBS, (uint64_t)(j >> 2), 0, 0, ctr, z);
    y[j] = u[j * A.stride] + sigma * z[j & 3];
}

// ensemble mean per node and the truth-based node sums:
// ws[i] = mean_p u[p][i]; out[4] += u_a^2; out[5] += (u_a - mean)^2
template <typename R>
__global__ void diag_mean_kernel(ModelArgs<R> A, int N, const R* u, const R* ua, double* ws, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double a = 0.0, b = 0.0;
    if (i < A.n) {
        double s = 0.0;
        for (int p = 0; p < N; ++p) s += (double)u[(size_t)p * A.n + i];
        const double mean = s / N;
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

__global__ void diag_zero_kernel(double* out) {
    if (threadIdx.x < 8) out[threadIdx.x] = 0.0;
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

template <typename R>
int launch_diag(const ModelArgs<R>& A, int N, const R* u, const R* ua, double* ws, double* out, cudaStream_t st) {
    diag_zero_kernel<<<1, 32, 0, st>>>(out);
    diag_mean_kernel<R><<<(A.n + 255) / 256, 256, 0, st>>>(A, N, u, ua, ws, out);
    diag_particle_kernel<R><<<(N * 32 + 255) / 256, 256, 0, st>>>(A, N, u, ua, ws, out);
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
