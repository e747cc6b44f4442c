// Warp-group propagation for float fields (explicit-advection Picard solver of
// the implicit midpoint step, Eq. fde1) at n = 64 P CS W nodes: W warps carry
// one particle, one CTA per particle.  Warp w holds the n / W consecutive nodes
// [w n / W, (w + 1) n / W) in the register layout of the warp-per-particle
// kernels (sch_warp.cuh): lane l of warp w, thread t = 32 w + l, owns the 2 P CS
// consecutive nodes [2 P CS t, 2 P CS (t + 1)) as 2P sub-chunks paired into P
// float2 streams, so the stencil work, the sub-chunk sweeps and the noise
// synthesis are the warp kernels' own.
//
// What changes is the reduced system of a constant cyclic solve.  After the
// sub-chunk sweeps and the S = 2P-row lane partition, the unknowns are the
// lane-last values EL_g of the 32 W lanes g = 32 w + l of the particle, coupled
// cyclically: LA EL_{g-1} + LB EL_g + LC EL_{g+1} = LD_g.  Each warp solves its own
// 32 rows as if they were cyclic among themselves, y = T32^{-1} LD (the PCR of
// the warp kernels), leaving out of lane 31's row the two terms that come from
// the next warp's lane 0 (m_w).  The true system differs from that only in the
// couplings of lanes 0 and 31, so with a_w = EL^w_0 and b_w = EL^w_31
//   EL^w = y^w - (b_{w-1} - b_w) phi - (a_{w+1} - a_w + m_w / LC) psi,
//   phi = T32^{-1} (LA e_0),  psi = T32^{-1} (LC e_31),
// and the 2W values (a_w, b_w) solve a block-circulant 2W x 2W system whose
// inverse the host tabulates (GTab).  Every warp publishes four floats in shared
// memory (y_0, y_31 and lane 0's two reduced-row inputs pd_0, qd_0); after one CTA
// barrier each warp forms from all warps' floats the boundary values it needs,
// including the field values at the nodes just outside its own ends.  A Picard
// iteration costs two barriers (one per constant solve) and a step one more (the
// SALT increment at the nodes next to the warp's ends).  The stop test reads the
// whole particle's max|dm| and max|m|, published with the Helmholtz solve, so
// every warp takes the same decision.
//
// Exchanges alternate between two slot buffers: a warp reads a buffer before it
// arrives at the next barrier, and can write that buffer again only after the
// barrier that follows, so one barrier per exchange suffices.
#pragma once

#include "sch_warp.cuh"

namespace sch {

// one warp's entry of a cross-warp exchange
struct __align__(16) GSlot {
    float4 a;   // y_0, y_31, pd_0, qd_0 of a reduced solve; or a field's two end values
    float4 b;   // max|dm|, max|m| of the warp's Picard update (with the Helmholtz solve)
};

template <int W>
struct GShared {
    GSlot slot[2][W];
    double red[W][2];   // per-warp partial sums (misfit, Girsanov)
    double res[2];      // the particle's NLL and log G of a proposal
    int flag;           // the accept decision of a proposal
};

// per-lane vectors phi = T32^{-1} LA e_0 and psi = T32^{-1} LC e_31 of a table
__device__ __forceinline__ void glane_vectors(const RTab<float>& Q, const GTab& G, float& phi, float& psi) {
    const int lane = threadIdx.x & 31;
    phi = pcr32_const(lane == 0 ? G.LA : 0.f, Q);
    psi = pcr32_const(lane == 31 ? G.LC : 0.f, Q);
}

// The boundary values of the 2W system are four sums over its 2W inputs (y_0 and y_31 of
// every warp): lane L takes sum o = L / 8 (bprev, bself, aself, anext) and the inputs e =
// L % 8 + 8 t < 2W; its weights, fixed for the kernel, come from the table once.
constexpr int GNT = (2 * GW_MAX + 7) / 8;
template <int W>
__device__ __forceinline__ void glane_weights(const GTab& G, float (&cw)[GNT]) {
    const int lane = threadIdx.x & 31, o = lane >> 3;
    const float* tab = (o == 0) ? G.bprev : (o == 1) ? G.bself : (o == 2) ? G.aself : G.anext;
#pragma unroll
    for (int t = 0; t < GNT; ++t) {
        const int e = (lane & 7) + 8 * t;
        cw[t] = (e < 2 * W) ? tab[e] : 0.f;
    }
}

// The lane's outer chunk-end neighbours of a paired field (see whalo), with the
// values at the nodes outside the warp, Lv (before its first node) and Rv (after
// its last), taken by lanes 0 and 31.
template <int CS, int P>
__device__ __forceinline__ void gwhalo(const float2 (&v)[P][CS], float Lv, float Rv, float2& lo, float2& hi) {
    const int lane = threadIdx.x & 31;
    const float a = __shfl_sync(FULL, v[P - 1][CS - 1].y, (lane + 31) & 31);
    const float b = __shfl_sync(FULL, v[0][0].x, (lane + 1) & 31);
    lo = make_float2(lane == 0 ? Lv : a, v[P - 1][CS - 1].x);
    hi = make_float2(v[0][0].y, lane == 31 ? Rv : b);
}

// Exchange of a field's end values: lane 0 of every warp publishes its first node's
// value `first`, lane 31 its last node's `last`; returns the previous warp's last
// (Lv) and the next warp's first (Rv).  One CTA barrier.
template <int W>
__device__ __forceinline__ void gends(float first, float last, float& Lv, float& Rv, GShared<W>* gs, int w,
                                      int& ex) {
    const int lane = threadIdx.x & 31;
    GSlot* sl = gs->slot[ex & 1];
    const float l31 = __shfl_sync(FULL, last, 31);
    if (lane == 0) sl[w].a = make_float4(first, l31, 0.f, 0.f);
    __syncthreads();
    ++ex;
    Lv = sl[(w + W - 1) % W].a.y;
    Rv = sl[(w + 1) % W].a.x;
}

// Cross-warp reduced solve of a tabulated constant matrix (see the file comment).
// In: the sub-chunk reduced-row inputs pd, de (as wreduced), and the warp's stop-test
// maxima dm, mm to publish.  Out: E, F, Ep, Fn as wreduced, and Lv / Rv, the solved
// values at the nodes just before and just after this warp's nodes.  Returns the
// slot buffer the exchange used (valid until the next exchange).
template <int P, int W>
__device__ __forceinline__ const GSlot* gwreduced(const WTab& T, const RTab<float>& Q, const GTab& G, float phi,
                                                  float psi, const float (&cw)[GNT], const float2 (&pd)[P],
                                                  const float2 (&de)[P],
                                                  float2 (&E)[P], float2 (&F)[P], float& Ep, float& Fn, float& Lv,
                                                  float& Rv, GShared<W>* gs, int w, int& ex, float dm, float mm) {
    constexpr int S = 2 * P;
    static_assert(S >= 2, "lane partition of at least two rows");
    const int lane = threadIdx.x & 31;
    float pr[S], dr[S];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        pr[p] = pd[p].x;
        pr[p + P] = pd[p].y;
        dr[p] = de[p].x;
        dr[p + P] = de[p].y;
    }
    // lane 31 leaves out the next warp's first row (its part m_w comes back below)
    const float pdn = __shfl_sync(FULL, pr[0], (lane + 1) & 31);
    const float pd_next = (lane == 31) ? 0.f : pdn;
    float D[S];
#pragma unroll
    for (int r = 0; r < S; ++r) D[r] = dr[r] - T.ae * pr[r] - T.ge * ((r == S - 1) ? pd_next : pr[r + 1]);
    float dl[S], dp[S];
    dl[0] = 0.f;
#pragma unroll
    for (int r = 1; r < S; ++r) dl[r] = (D[r] - Q.A * dl[r - 1]) * Q.q[r];
    dp[S - 1] = 0.f;
    dp[0] = 0.f;
#pragma unroll
    for (int r = S - 2; r >= 1; --r) dp[r] = dl[r] - Q.ga[r] * dp[r + 1];
    const float DF = (S == 2) ? D[0] : D[0] - Q.Cc * dp[1];
    const float qd = DF * Q.iBF;
    const float nqdr = __shfl_sync(FULL, qd, (lane + 1) & 31);
    const float nqd = (lane == 31) ? 0.f : nqdr;
    const float LD = dl[S - 1] - Q.aeL * qd - Q.geL * nqd;
    const float y = pcr32_const(LD, Q);
    const float y31 = __shfl_sync(FULL, y, 31);
    GSlot* sl = gs->slot[ex & 1];
    if (lane == 0) {
        sl[w].a = make_float4(y, y31, pr[0], qd);
        sl[w].b = make_float4(dm, mm, 0.f, 0.f);
    }
    __syncthreads();
    ++ex;
    // boundary values: every warp's y_0, y_31 corrected by its m (the part of its lane 31's
    // row from the next warp), then the tabulated inverse of the 2W system, in warp order
    // relative to this warp (k = 0: this warp); lane L forms its inputs' terms of sum L / 8
    float part = 0.f;
#pragma unroll
    for (int t = 0; t < GNT; ++t) {
        const int e = (lane & 7) + 8 * t;
        if (8 * t < 2 * W) {
            const int k = e % W;
            const float4 s = sl[(w + k) % W].a, sn = sl[(w + k + 1) % W].a;
            const float mk = G.cq * sn.z + G.geL * sn.w;
            const float yh = (e < W) ? s.x - mk * G.p2_0 : s.y - mk * G.p2_31;
            part = fmaf(cw[t], yh, part);
        }
    }
    part += __shfl_xor_sync(FULL, part, 1);
    part += __shfl_xor_sync(FULL, part, 2);
    part += __shfl_xor_sync(FULL, part, 4);
    const float bp = __shfl_sync(FULL, part, 0), bs = __shfl_sync(FULL, part, 8);
    const float as = __shfl_sync(FULL, part, 16), an = __shfl_sync(FULL, part, 24);
    const float4 s1 = sl[(w + 1) % W].a;
    const float mw = G.cq * s1.z + G.geL * s1.w;
    const float EL = y - (bp - bs) * phi - (an - as + mw * G.iLC) * psi;
    const float Epr = __shfl_sync(FULL, EL, (lane + 31) & 31);
    Ep = (lane == 0) ? bp : Epr;
    const float Ff = qd - Q.qa * Ep - Q.qc * EL;
    float Er[S], Fr[S];
    Er[0] = Ff;
#pragma unroll
    for (int r = 1; r < S - 1; ++r) Er[r] = dp[r] - Q.alp[r] * Ff - Q.gap[r] * EL;
    Er[S - 1] = EL;
#pragma unroll
    for (int r = 0; r < S; ++r) Fr[r] = pr[r] - T.pa * ((r == 0) ? Ep : Er[r - 1]) - T.pc * Er[r];
    // the next warp's first node: its lane 0's first row, F = pd_0 - pa b_w - pc Ff
    const float Ffn = s1.w - Q.qa * bs - Q.qc * an;
    Rv = s1.z - T.pa * bs - T.pc * Ffn;
    Lv = bp;
    const float Fnr = __shfl_sync(FULL, Fr[0], (lane + 1) & 31);
    Fn = (lane == 31) ? Rv : Fnr;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        E[p] = make_float2(Er[p], Er[p + P]);
        F[p] = make_float2(Fr[p], Fr[p + P]);
    }
    return sl;
}

// The same solve when the lane-level system is diagonal to float rounding (GTab.ldiag:
// the Picard matrix at n = 4096 with 8-node sub-chunks couples neighbouring lanes by
// 1.9e-9 of the diagonal): EL_g = LD_g / LB.  Only lane 31's row needs the next warp's
// lane 0 (pd_0, qd_0), and lane 0's previous lane is the previous warp's lane 31, so each
// warp publishes pd_0, qd_0 and LD_0 of its lane 0 and the part of lane 31's LD that is
// its own; after one barrier every warp completes lane 31's row and forms the values
// outside its ends.  Outputs as gwreduced.
template <int P, int W>
__device__ __forceinline__ void gwreduced_ldiag(const WTab& T, const RTab<float>& Q, const GTab& G,
                                                const float2 (&pd)[P], const float2 (&de)[P], float2 (&E)[P],
                                                float2 (&F)[P], float& Ep, float& Fn, float& Lv, float& Rv,
                                                GShared<W>* gs, int w, int& ex) {
    constexpr int S = 2 * P;
    const int lane = threadIdx.x & 31;
    float pr[S], dr[S];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        pr[p] = pd[p].x;
        pr[p + P] = pd[p].y;
        dr[p] = de[p].x;
        dr[p + P] = de[p].y;
    }
    const float pdn = __shfl_sync(FULL, pr[0], (lane + 1) & 31);
    const float pd_next = (lane == 31) ? 0.f : pdn;
    float D[S];
#pragma unroll
    for (int r = 0; r < S; ++r) D[r] = dr[r] - T.ae * pr[r] - T.ge * ((r == S - 1) ? pd_next : pr[r + 1]);
    float dl[S], dp[S];
    dl[0] = 0.f;
#pragma unroll
    for (int r = 1; r < S; ++r) dl[r] = (D[r] - Q.A * dl[r - 1]) * Q.q[r];
    dp[S - 1] = 0.f;
    dp[0] = 0.f;
#pragma unroll
    for (int r = S - 2; r >= 1; --r) dp[r] = dl[r] - Q.ga[r] * dp[r + 1];
    const float DF = (S == 2) ? D[0] : D[0] - Q.Cc * dp[1];
    const float qd = DF * Q.iBF;
    const float nqdr = __shfl_sync(FULL, qd, (lane + 1) & 31);
    const float nqd = (lane == 31) ? 0.f : nqdr;
    const float LD = dl[S - 1] - Q.aeL * qd - Q.geL * nqd;   // lane 31: without the next warp's part
    const float ld31 = __shfl_sync(FULL, LD, 31);
    GSlot* sl = gs->slot[ex & 1];
    if (lane == 0) sl[w].a = make_float4(pr[0], qd, LD, ld31);
    __syncthreads();
    ++ex;
    const float4 sp = sl[(w + W - 1) % W].a, so = sl[w].a, sn = sl[(w + 1) % W].a;
    // lane 31's row of this warp and of the previous one, completed with the next warp's lane 0
    const float el31 = (so.w - (G.cq * sn.x + G.geL * sn.y)) * G.iLB;
    const float elp31 = (sp.w - (G.cq * so.x + G.geL * so.y)) * G.iLB;
    const float EL = (lane == 31) ? el31 : LD * G.iLB;
    const float Epr = __shfl_sync(FULL, EL, (lane + 31) & 31);
    Ep = (lane == 0) ? elp31 : Epr;
    const float Ff = qd - Q.qa * Ep - Q.qc * EL;
    float Er[S], Fr[S];
    Er[0] = Ff;
#pragma unroll
    for (int r = 1; r < S - 1; ++r) Er[r] = dp[r] - Q.alp[r] * Ff - Q.gap[r] * EL;
    Er[S - 1] = EL;
#pragma unroll
    for (int r = 0; r < S; ++r) Fr[r] = pr[r] - T.pa * ((r == 0) ? Ep : Er[r - 1]) - T.pc * Er[r];
    // the next warp's first node: its lane 0's first row
    const float el0n = sn.z * G.iLB;
    const float Ffn = sn.y - Q.qa * el31 - Q.qc * el0n;
    Rv = sn.x - T.pa * el31 - T.pc * Ffn;
    Lv = elp31;
    const float Fnr = __shfl_sync(FULL, Fr[0], (lane + 1) & 31);
    Fn = (lane == 31) ? Rv : Fnr;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        E[p] = make_float2(Er[p], Er[p + P]);
        F[p] = make_float2(Fr[p], Fr[p + P]);
    }
}

// per-lane vectors of the two tables and the CTA's exchange state
struct GLane {
    float phi_p, psi_p, phi_h, psi_h;
    float cw_p[GNT], cw_h[GNT];
};

// u = H^{-1} M m for this warp's nodes; m's outside values mL, mR in, u's out
template <int CS, int P, int W>
__device__ __forceinline__ void gwu_from_m(const WArgs& Wa, const GArgs& G, const GLane& gl, const float2 (&m)[P][CS],
                                           float mL, float mR, float2 (&u)[P][CS], float& uL, float& uR,
                                           GShared<W>* gs, int w, int& ex) {
    float2 lo, hi, x[P][CS];
    gwhalo<CS, P>(m, mL, mR, lo, hi);
    const float2 four = f2b(4.f);
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
        for (int i = 0; i < CS; ++i)
            x[p][i] = f2fma(four, m[p][i], f2add(wleft<CS, P>(m, p, i, lo), wright<CS, P>(m, p, i, hi)));
    float2 pd[P], de[P], E[P], F[P];
    float Ep, Fn;
    wsweep<CS, P>(Wa.hel, x, pd, de);
    gwreduced<P, W>(Wa.hel, Wa.rhel, G.hel, gl.phi_h, gl.psi_h, gl.cw_h, pd, de, E, F, Ep, Fn, uL, uR, gs, w, ex, 0.f,
                    0.f);
    wback<CS, P>(Wa.hel, x, F, E, u);
}

// A step's slot of the jitter's guess buffer: the converged m of the whole particle (n
// floats) in the register order of its threads: thread t's pairs 2k and 2k + 1 (pair
// e = p CS + i) form the float4 at index k TPB + t, TPB = 32 W threads, so that every
// 16-byte access of a warp is contiguous.  u is not kept: the step recomputes it from the
// guess (u = H^-1 M m, one Helmholtz solve), which costs less than moving it (a slot of
// m alone for the CTAs resident at once stays in L2 between two proposals).
template <int CS, int P, int W>
__device__ __forceinline__ void gguess_store(float* slot, const float2 (&m)[P][CS]) {
    constexpr int H = P * CS, TPB = 32 * W;
    float4* m4 = reinterpret_cast<float4*>(slot);
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < H / 2; ++k) {
        const int e0 = 2 * k, e1 = 2 * k + 1;
        const float2 a = m[e0 / CS][e0 % CS], b = m[e1 / CS][e1 % CS];
        m4[k * TPB + t] = make_float4(a.x, a.y, b.x, b.y);
    }
}

// The guess of a step for this thread's nodes, and for the nodes just outside its warp (the
// last node of the previous warp's lane 31, the first of the next warp's lane 0)
template <int CS, int P, int W>
__device__ __forceinline__ void gguess_load(const float* slot, float2 (&m)[P][CS], float& mL, float& mR) {
    constexpr int H = P * CS, TPB = 32 * W;
    static_assert(H % 2 == 0, "pairs loaded two at a time");
    const float4* m4 = reinterpret_cast<const float4*>(slot);
    const int t = threadIdx.x, w = t >> 5;
#pragma unroll
    for (int k = 0; k < H / 2; ++k) {
        const int e0 = 2 * k, e1 = 2 * k + 1;
        const float4 a = m4[k * TPB + t];
        m[e0 / CS][e0 % CS] = make_float2(a.x, a.y);
        m[e1 / CS][e1 % CS] = make_float2(a.z, a.w);
    }
    const int tl = (32 * w + TPB - 1) % TPB, tr = (32 * (w + 1)) % TPB;
    mL = m4[(H / 2 - 1) * TPB + tl].w;
    mR = m4[tr].x;
}

// The particle-wide state of a warp's nodes carried through a window: the fields and
// the values of m and u at the two nodes outside the warp.
template <int CS, int P>
struct GState {
    float2 m[P][CS], u[P][CS];
    float mL, mR, uL, uR;
};

// One implicit-midpoint step of the particle (warp w's share), W0 holding the step's
// dU/4 at this lane's nodes on entry (see wstep_core for the iteration).  R0sm is the
// warp's three [P][CS][32] float2 slots: R0 = (M - mu dt/2 K) m0, W0 and m0.
template <int CS, int P, int W, int PD>
__device__ __forceinline__ void gwstep_core(const ModelArgs<float>& A, const WArgs& Wa, const GArgs& G,
                                            const GLane& gl, GState<CS, P>& X, float2* R0sm, float2 (&W0)[P][CS],
                                            GShared<W>* gs, int w, int& ex, int& iters, int& flags,
                                            const float* gin = nullptr, float* gout = nullptr) {
    const int lane = threadIdx.x & 31;
    // the guess (if any) is read first, so that its latency passes in the barrier and the set-up
    // below; no warp can have written this step's slot of the current proposal yet (each writes
    // it at the end of its step, after the barriers that every warp reaches only after this read)
    float2 mi[P][CS];
    float miL = 0.f, miR = 0.f;
    if (gin) gguess_load<CS, P, W>(gin, mi, miL, miR);
    // the increment at the nodes next to this warp's ends
    float nqL, nqR;
    gends<W>(W0[0][0].x, W0[P - 1][CS - 1].y, nqL, nqR, gs, w, ex);
    const float dt8s = A.dt8;
    const float W0L = fmaf(dt8s, X.uL, nqL), W0R = fmaf(dt8s, X.uR, nqR);
    float2* W0sm = R0sm + P * CS * 32;
    float2* Msm = W0sm + P * CS * 32;
    {
        const float2 dt8 = f2b(A.dt8);
        float2 lo, hi;
        gwhalo<CS, P>(X.m, X.mL, X.mR, lo, hi);
        const float2 c0p = f2b(A.c0p), b0p = f2b(A.b0p);
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int i = 0; i < CS; ++i) {
                W0sm[(p * CS + i) * 32 + lane] = f2fma(dt8, X.u[p][i], W0[p][i]);
                R0sm[(p * CS + i) * 32 + lane] = f2fma(
                    c0p, f2add(wleft<CS, P>(X.m, p, i, lo), wright<CS, P>(X.m, p, i, hi)), f2mul(b0p, X.m[p][i]));
                Msm[(p * CS + i) * 32 + lane] = X.m[p][i];
            }
    }
    // the Picard iterate starts from the step's start state, or from the guess: the converged
    // m of this step in the call's previous proposal (read above) and its u = H^-1 M m
    if (gin) {
        gwu_from_m<CS, P, W>(Wa, G, gl, mi, miL, miR, X.u, X.uL, X.uR, gs, w, ex);
    } else {
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int i = 0; i < CS; ++i) mi[p][i] = X.m[p][i];
        miL = X.mL;
        miR = X.mR;
    }
    const float2 dt8 = f2b(A.dt8);
    float dm_prev = INFINITY;
    for (int it = 1;; ++it) {
        float2 x[P][CS];
        {
            float2 wv[P][CS], mb[P][CS];
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int i = 0; i < CS; ++i) {
                    wv[p][i] = f2fma(dt8, X.u[p][i], W0sm[(p * CS + i) * 32 + lane]);
                    mb[p][i] = f2add(Msm[(p * CS + i) * 32 + lane], mi[p][i]);
                }
            float2 wl, wr, ml, mr;
            gwhalo<CS, P>(wv, fmaf(dt8s, X.uL, W0L), fmaf(dt8s, X.uR, W0R), wl, wr);
            gwhalo<CS, P>(mb, X.mL + miL, X.mR + miR, ml, mr);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                float2 gp = f2add(wleft<CS, P>(mb, p, 0, ml), mb[p][0]);
#pragma unroll
                for (int i = 0; i < CS; ++i) {
                    const float2 g = f2add(mb[p][i], wright<CS, P>(mb, p, i, mr));
                    x[p][i] = f2sub(f2fma(wleft<CS, P>(wv, p, i, wl), gp, R0sm[(p * CS + i) * 32 + lane]),
                                    f2mul(wright<CS, P>(wv, p, i, wr), g));
                    gp = g;
                }
            }
        }
        // (M + mu dt/2 K) m_new = rhs
        float2 pd[P], de[P], E[P], F[P];
        float Ep, Fn;
        wsweep<CS, P>(Wa.pic, x, pd, de);
        if constexpr (PD)
            gwreduced_ldiag<P, W>(Wa.pic, Wa.rpic, G.pic, pd, de, E, F, Ep, Fn, miL, miR, gs, w, ex);
        else
            gwreduced<P, W>(Wa.pic, Wa.rpic, G.pic, gl.phi_p, gl.psi_p, gl.cw_p, pd, de, E, F, Ep, Fn, miL, miR, gs, w,
                            ex, 0.f, 0.f);
        float2 mn[P][CS];
        wback<CS, P>(Wa.pic, x, F, E, mn);
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
        const float dmw = warp_max_nan(dmax);
        const float mmw = warp_max_nan(mmax);
        // u_new = H^{-1} M m_new, published with this warp's stop-test maxima
        const GSlot* sl;
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
            wsweep<CS, P>(Wa.hel, x, hpd, hde);
            sl = gwreduced<P, W>(Wa.hel, Wa.rhel, G.hel, gl.phi_h, gl.psi_h, gl.cw_h, hpd, hde, hE, hF, hEp, hFn, X.uL,
                                 X.uR, gs, w, ex, dmw, mmw);
            wback<CS, P>(Wa.hel, x, hF, hE, X.u);
        }
        iters++;
        // the particle's maxima over every warp (NaN if any is NaN)
        float dm = 0.f, mm = 0.f;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const float4 b = sl[k].b;
            dm = fmax3_nan(dm, b.x, dm);
            mm = fmax3_nan(mm, b.y, mm);
        }
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
        for (int i = 0; i < CS; ++i) X.m[p][i] = mi[p][i];
    X.mL = miL;
    X.mR = miR;
    if (gout) gguess_store<CS, P, W>(gout, X.m);   // after the step's last exchange
}

// The step's SALT increment dU/4 at the lane's nodes, as wnoise (sch_warp.cuh) sums its
// even and odd parts E(d) = sum_j v_j cos(j d) and O(d) = sum_j q_j sin(j d) about the
// lane's centre.  Where the host fitted cos(j d) and sin(j d) / tau by polynomials in
// s = tau^2 (GArgs npc, npoly; tau = d / d_{H-1}), the lane instead accumulates the WNP
// coefficient pairs
//   (e_k, o_k) = sum_j (v_j c_jk, q_j s_jk),   E(d) = sum_k e_k s^k,  O(d) = tau sum_k o_k s^k,
// one packed FMA each a harmonic, and evaluates both at its H offsets by Horner's rule
// (tau and s are compile-time constants of the layout).
template <int CS, int P>
__device__ __forceinline__ void gnoise(const ModelArgs<float>& A, const WArgs& Wa, const GArgs& G, const float* wq,
                                       float sc, float cc, float2 (&nq)[P][CS]) {
    constexpr int H = P * CS, Q = H / 2;
    float2 EP[Q], OP[Q];
    if (G.npoly) {
        float2 eo[WNP];
#pragma unroll
        for (int k = 0; k < WNP; ++k) eo[k] = f2b(0.f);
        float sj = sc, cj = cc;
#pragma unroll 4
        for (int j = 0; j < A.K2; ++j) {
            const float2 ab = *reinterpret_cast<const float2*>(wq + 2 * j);
            const float2 vq = make_float2(fmaf(ab.x, sj, ab.y * cj), fmaf(ab.x, cj, -(ab.y * sj)));
#pragma unroll
            for (int k = 0; k < WNP; ++k) eo[k] = f2fma(vq, G.npc[j][k], eo[k]);
            const float sn = fmaf(sj, cc, cj * sc);
            cj = fmaf(cj, cc, -(sj * sc));
            sj = sn;
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            // tau of the offsets d_{H-1-q} and d_q, and their squares
            const float ta = (float)(2 * (H - 1 - q) + 1) / (float)(2 * H - 1);
            const float tb = (float)(2 * q + 1) / (float)(2 * H - 1);
            const float2 tq = make_float2(ta, tb), s2 = make_float2(ta * ta, tb * tb);
            float2 e = f2b(eo[WNP - 1].x), o = f2b(eo[WNP - 1].y);
#pragma unroll
            for (int k = WNP - 2; k >= 0; --k) {
                e = f2fma(e, s2, f2b(eo[k].x));
                o = f2fma(o, s2, f2b(eo[k].y));
            }
            EP[q] = e;
            OP[q] = f2mul(o, tq);
        }
    } else {
        wnoise_tab<CS, P>(A, Wa, wq, sc, cc, EP, OP);
    }
    wnoise_finish<CS, P>(EP, OP, nq);
}

// load a particle's window start: m from the row, its outside values, and u = H^{-1} M m
template <int CS, int P, int W>
__device__ __forceinline__ void gwstart(const WArgs& Wa, const GArgs& G, const GLane& gl, const float* row,
                                        GState<CS, P>& X, GShared<W>* gs, int w, int& ex) {
    wload<CS, P>(row, X.m);
    gends<W>(X.m[0][0].x, X.m[P - 1][CS - 1].y, X.mL, X.mR, gs, w, ex);
    gwu_from_m<CS, P, W>(Wa, G, gl, X.m, X.mL, X.mR, X.u, X.uL, X.uR, gs, w, ex);
}

// the sum of a double over the CTA (every thread receives it); two barriers
template <int W>
__device__ __forceinline__ void gsum2(GShared<W>* gs, double& a, double& b) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
        gs->red[w][0] = a;
        gs->red[w][1] = b;
    }
    __syncthreads();
    a = 0.0;
    b = 0.0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        a += gs->red[k][0];
        b += gs->red[k][1];
    }
    __syncthreads();
}

template <int CS, int P, int W>
__host__ __device__ constexpr size_t gsmem_base() {
    return (sizeof(GShared<W>) + 15) / 16 * 16 + (size_t)3 * W * P * CS * 32 * sizeof(float2);
}

// Resident CTAs per SM the kernels are compiled for: 32 W threads each, with at most
// 65536 / (3 x 32 W) registers a thread (168 at W = 4).  To get there the step's fixed
// fields W0 = dt/8 u0 + dU/4 and m0 live in shared memory beside R0, one [P][CS][32]
// float2 slot each per warp, read once per Picard iteration; against two CTAs with
// them in registers (233 registers) this ran the large-run filter 3% faster.
constexpr int GMINB = 3;
// n = 1024 in two warps of 16 nodes a lane (CS = 4, W = 2): seven 64-thread CTAs per SM (at most
// 146 registers), so that a 1024-particle launch is one wave on 152 SMs
template <int CS, int W>
constexpr int gminb() {
    return (CS == 4 && W == 2) ? 7 : GMINB;
}

template <int CS, int P, int W, int PD>
__global__ void __launch_bounds__(32 * W, gminb<CS, W>()) gwindow_kernel(ModelArgs<float> A, WArgs Wa, GArgs G,
                                                                WindowIO<float> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GShared<W>* gs = reinterpret_cast<GShared<W>*>(smem_raw);
    const int w = threadIdx.x >> 5;
    float2* R0sm = reinterpret_cast<float2*>(smem_raw + (sizeof(GShared<W>) + 15) / 16 * 16) + 3 * w * P * CS * 32;
    float* noise = reinterpret_cast<float*>(smem_raw + gsmem_base<CS, P, W>());
    const int p = blockIdx.x;
    const size_t NK = (size_t)io.Ns * A.K;
    stage_noise(A, noise, io.dW + p * NK, io.lam ? io.lam + p * NK : nullptr, io.Ns);
    GLane gl;
    glane_vectors(Wa.rpic, G.pic, gl.phi_p, gl.psi_p);
    glane_vectors(Wa.rhel, G.hel, gl.phi_h, gl.psi_h);
    glane_weights<W>(G.pic, gl.cw_p);
    glane_weights<W>(G.hel, gl.cw_h);
    float sc, cc;
    wcentre<CS, P>(A.n, sc, cc);
    int ex = 0;
    GState<CS, P> X;
    gwstart<CS, P, W>(Wa, G, gl, io.m_in + (size_t)p * A.n, X, gs, w, ex);   // its barriers also order the staging
    int iters = 0, flags = 0;
    for (int s = 0; s < io.Ns; ++s) {
        float2 W0[P][CS];
        gnoise<CS, P>(A, Wa, G, noise + s * A.K, sc, cc, W0);
        gwstep_core<CS, P, W, PD>(A, Wa, G, gl, X, R0sm, W0, gs, w, ex, iters, flags);
    }
    wstore<CS, P>(io.m_out + (size_t)p * A.n, X.m);
    wstore<CS, P>(io.u_out + (size_t)p * A.n, X.u);
    if (io.y) {
        double mis = wmisfit<CS, P>(A, X.u, io.y);
        double gl2 = window_girsanov(A, io.dW + p * NK, io.lam ? io.lam + p * NK : nullptr, io.Ns);
        gsum2<W>(gs, mis, gl2);
        if (threadIdx.x == 0) {
            io.nll[p] = 0.5 * mis;
            if (io.logG) io.logG[p] = -gl2;
        }
    }
    if (threadIdx.x == 0) {
        if (io.iters) io.iters[p] = iters;
        if (io.status) io.status[p] = flags;
    }
}

// PCN jittering (Sec. 3.1.2) with W warps per particle: as wjitter_kernel, the
// proposals drawn by the whole CTA, the decision taken by thread 0 and shared.
// PD: the Picard solve's lane-level system is diagonal (gwreduced_ldiag).
template <int CS, int P, int W, int PD>
__global__ void __launch_bounds__(32 * W, gminb<CS, W>()) gjitter_kernel(ModelArgs<float> A, WArgs Wa, GArgs G,
                                                                JitterIO<float> io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // a device-gated stage reads its temperature, and does nothing when inactive
    if (io.tstate && io.tstate[4] == 0.0) return;
    GShared<W>* gs = reinterpret_cast<GShared<W>*>(smem_raw);
    const int t = threadIdx.x, w = t >> 5;
    float2* R0sm = reinterpret_cast<float2*>(smem_raw + (sizeof(GShared<W>) + 15) / 16 * 16) + 3 * w * P * CS * 32;
    const double theta = io.tstate ? io.tstate[2] : io.theta;
    const int p = blockIdx.x;
    const int Ns = io.Ns, K = A.K, NK = Ns * K;
    float* noise = reinterpret_cast<float*>(smem_raw + gsmem_base<CS, P, W>());
    float* cur = noise + NK;
    float* prop = noise + 2 * NK;
    float* dW = io.dW + (size_t)p * NK;
    const float* lam = io.lam ? io.lam + (size_t)p * NK : nullptr;
    for (int q = t; q < NK; q += 32 * W) cur[q] = dW[q];
    double nll0 = io.nll[p], lg0 = io.logG ? io.logG[p] : 0.0;
    GLane gl;
    glane_vectors(Wa.rpic, G.pic, gl.phi_p, gl.psi_p);
    glane_vectors(Wa.rhel, G.hel, gl.phi_h, gl.psi_h);
    glane_weights<W>(G.pic, gl.cw_p);
    glane_weights<W>(G.hel, gl.cw_h);
    float sc, cc;
    wcentre<CS, P>(A.n, sc, cc);
    const float sq = io.sq1mr2 * (float)sqrt(A.dt_d);
    const int nblk = (K + 3) >> 2;
    int iters = 0, flags = 0, n_acc = 0, changed = 0, ex = 0;
    // Warm starts pay where successive proposals' trajectories nearly coincide (rho near one:
    // at 0.9999 the proposal moves the noise by 1.4% of its spread, and a step then takes 2.2
    // Picard iterations against 3.9 from the start state); for rho < 0.99 every proposal
    // starts from the step's start state.
    float* gbuf = (io.guess && io.rho >= 0.99f) ? io.guess : nullptr;
    bool gvalid = false;
    __syncthreads();
    for (int j = 0; j < io.n_iter; ++j) {
        const uint64_t ctr = io.ctr + (uint64_t)j;
        for (int q = t; q < Ns * nblk; q += 32 * W) {
            const int s = q / nblk, b = q % nblk;
            float z[4];
            normal4<float>(io.seed, SCH_TAG_PCN, (uint64_t)b, (uint64_t)s, (uint64_t)(io.particle0 + p), ctr, z);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 4 * b + e;
                if (k < K) prop[s * K + k] = io.rho * cur[s * K + k] + sq * z[e];
            }
        }
        __syncthreads();
        stage_noise(A, noise, prop, lam, Ns);
        GState<CS, P> X;
        gwstart<CS, P, W>(Wa, G, gl, io.m_start + (size_t)p * A.n, X, gs, w, ex);   // orders the staging
        int fl = 0;
        // the guess slots of this particle: a proposal starts cold unless the previous one of
        // this call finished cleanly (then it starts from that one's per-step states), and it
        // leaves its own states for the next one (the last proposal leaves nothing)
        float* gbase = gbuf ? gbuf + (size_t)p * Ns * A.n : nullptr;
        for (int s = 0; s < Ns; ++s) {
            float2 W0[P][CS];
            gnoise<CS, P>(A, Wa, G, noise + s * K, sc, cc, W0);
            float* slot = gbase ? gbase + (size_t)s * A.n : nullptr;
            gwstep_core<CS, P, W, PD>(A, Wa, G, gl, X, R0sm, W0, gs, w, ex, iters, fl, gvalid ? slot : nullptr,
                                      j + 1 < io.n_iter ? slot : nullptr);
        }
        gvalid = gbase && fl == 0;   // the same in every thread: the flags follow CTA-wide decisions
        double mis = wmisfit<CS, P>(A, X.u, io.y);
        double gsum = window_girsanov(A, prop, lam, Ns);
        gsum2<W>(gs, mis, gsum);
        const double nll1 = 0.5 * mis, lg1 = -gsum;
        if (t == 0) {
            const double w0 = theta * (nll0 - lg0);
            const double w1 = theta * (nll1 - lg1);
            const double logU = log(uniform_open0(io.seed, SCH_TAG_PCN_ACCEPT, (uint64_t)(io.particle0 + p), ctr));
            gs->flag = (fl == 0) && (logU < w0 - w1);
        }
        __syncthreads();
        const int acc = gs->flag;
        if (acc) {
            nll0 = nll1;
            lg0 = lg1;
            for (int q = t; q < NK; q += 32 * W) cur[q] = prop[q];
            wstore<CS, P>(io.m_end + (size_t)p * A.n, X.m);
            wstore<CS, P>(io.u_end + (size_t)p * A.n, X.u);
            n_acc++;
            changed = 1;
        }
        flags |= fl;
        __syncthreads();
    }
    if (changed)
        for (int q = t; q < NK; q += 32 * W) dW[q] = cur[q];
    if (t == 0) {
        io.nll[p] = nll0;
        if (io.logG) io.logG[p] = lg0;
        if (io.accepts) io.accepts[p] = n_acc;
        if (io.iters) io.iters[p] = iters;
        if (io.status) io.status[p] = flags;
    }
}

}  // namespace sch
