// C-ABI entry points of the SCH particle-filter library (include/sch.h):
// argument checks on the host, then one kernel launch (or a few) on the
// caller's stream.  No entry point synchronises or allocates device memory.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "sch_internal.h"

using namespace sch;

struct sch_ctx {
    sch_params p;
    int C, tp;
    int Q;            // Brownian motions per step: K (modes) or n (Matern)
    int matern;       // 1 for SCH_NOISE_MATERN
    int wcs;          // sub-chunk length of the warp-per-particle or warp-group kernels, 0 = CTA kernels
    int gw;           // warps per particle of the warp-group kernels, 0 = not the group layout
    WArgs wa;
    GArgs ga;
    ModelArgs<float> af;
    ModelArgs<double> ad;
    void* jws;        // caller-owned jitter workspace (sch_set_jitter_workspace), or null
    size_t jws_bytes;
};

namespace {

// Chunk-partition coefficients of a constant symmetric tridiagonal matrix for
// chunks of up to HMAX rows, in double precision (the kernels' CTab and WTab
// are casts of it).
constexpr int HMAX = 32;
struct HTab {
    double rden[HMAX], gam[HMAX], alpp[HMAX], gamp[HMAX];
    double a, iBF, pa, pc, ae, ge;
};

// Chunk-partition coefficients of the symmetric circulant tridiagonal matrix
// with off-diagonal a and diagonal b, for chunks of C rows (double precision).
void ctab_host(double a, double b, int C, HTab& T) {
    double al[HMAX], ga[HMAX];
    memset(&T, 0, sizeof(T));
    al[0] = -1.0;
    ga[0] = 0.0;
    for (int i = 1; i < C; ++i) {
        const double r = 1.0 / (b - a * ga[i - 1]);
        T.rden[i] = r;
        ga[i] = a * r;
        al[i] = -a * al[i - 1] * r;
        T.gam[i] = ga[i];
    }
    double ap = 0.0, gp = -1.0;
    T.alpp[C - 1] = ap;
    T.gamp[C - 1] = gp;
    for (int i = C - 2; i >= 1; --i) {
        ap = al[i] - ga[i] * ap;
        gp = -ga[i] * gp;
        T.alpp[i] = ap;
        T.gamp[i] = gp;
    }
    const double BF = (C == 2) ? b : b - a * T.alpp[1];
    const double CF = (C == 2) ? a : -a * T.gamp[1];
    T.a = a;
    T.iBF = 1.0 / BF;
    T.pa = a * T.iBF;
    T.pc = CF * T.iBF;
    T.ae = al[C - 1];
    T.ge = ga[C - 1];
}

// Reduced cyclic system of chunk table T for TP threads: lane-level sweep over
// RR = TP/32 rows and the 32-lane PCR coefficients (double precision).
void rtab_host(const HTab& T, int TP, RTab<double>& Q) {
    memset(&Q, 0, sizeof(Q));
    const double A = -T.ae * T.pa, B = 1.0 - T.ae * T.pc - T.ge * T.pa, Cc = -T.ge * T.pc;
    Q.A = A;
    Q.B = B;
    Q.Cc = Cc;
    const int RR = TP / 32;
    double LA = A, LB = B, LC = Cc;
    if (RR > 1) {
        double alf[16], gaf[16];
        alf[0] = -1.0;
        gaf[0] = 0.0;
        for (int r = 1; r < RR; ++r) {
            const double q = 1.0 / (B - A * gaf[r - 1]);
            Q.q[r] = q;
            gaf[r] = Cc * q;
            alf[r] = -A * alf[r - 1] * q;
            Q.ga[r] = gaf[r];
        }
        Q.aeL = alf[RR - 1];
        Q.geL = gaf[RR - 1];
        double ap = 0.0, gp = -1.0;
        Q.alp[RR - 1] = ap;
        Q.gap[RR - 1] = gp;
        for (int r = RR - 2; r >= 1; --r) {
            ap = alf[r] - gaf[r] * ap;
            gp = -gaf[r] * gp;
            Q.alp[r] = ap;
            Q.gap[r] = gp;
        }
        const double BF = (RR == 2) ? B : B - Cc * Q.alp[1];
        const double CF = (RR == 2) ? Cc : -Cc * Q.gap[1];
        Q.iBF = 1.0 / BF;
        Q.qa = A * Q.iBF;
        Q.qc = CF * Q.iBF;
        LA = -Q.aeL * Q.qa;
        LB = 1.0 - Q.aeL * Q.qc - Q.geL * Q.qa;
        LC = -Q.geL * Q.qc;
    }
    double a = LA, b = LB, c = LC;
    for (int l = 0; l < 4; ++l) {
        const double k1 = a / b, k2 = c / b;
        Q.k1[l] = k1;
        Q.k2[l] = k2;
        const double nb = b - c * k1 - a * k2;
        a = -a * k1;
        c = -c * k2;
        b = nb;
    }
    const double e = a + c, det = b * b - e * e;
    Q.f1 = b / det;
    Q.f2 = -e / det;
}

// chunk sweep of table T on a right-hand side r: the reduced "first" row value
// pd, the "last" row value de and the interior particular solution dp
void chunk_sweep(const HTab& T, int C, const double* r, double& pd, double& de, double* dp) {
    double d[8];
    d[0] = 0.0;
    for (int i = 1; i < C; ++i) d[i] = (r[i] - T.a * d[i - 1]) * T.rden[i];
    for (int i = 0; i < C; ++i) dp[i] = 0.0;
    for (int i = C - 2; i >= 1; --i) dp[i] = d[i] - T.gam[i] * dp[i + 1];
    const double DF = (C == 2) ? r[0] : r[0] - T.a * dp[1];
    pd = DF * T.iBF;
    de = d[C - 1];
}

// the Helmholtz interface rows as linear functionals of the Picard chunk solution
void hbasis_host(const HTab& P, const HTab& H, int C, double h6, HBasis<double>& B) {
    memset(&B, 0, sizeof(B));
    double wpd[8], wde[8], dp[8], r[8];
    for (int j = 0; j < C; ++j) {
        for (int i = 0; i < C; ++i) r[i] = (i == j) ? 1.0 : 0.0;
        chunk_sweep(H, C, r, wpd[j], wde[j], dp);
    }
    auto mass_c = [&](const double* x, double* out) {
        for (int j = 0; j < C; ++j) {
            const double lo = (j > 0) ? x[j - 1] : 0.0, hi = (j < C - 1) ? x[j + 1] : 0.0;
            out[j] = h6 * (lo + 4.0 * x[j] + hi);
        }
    };
    for (int i = 1; i < C - 1; ++i) {
        double e[8], me[8];
        for (int j = 0; j < C; ++j) e[j] = (j == i) ? 1.0 : 0.0;
        mass_c(e, me);
        double a = 0.0, b = 0.0;
        for (int j = 0; j < C; ++j) {
            a += wpd[j] * me[j];
            b += wde[j] * me[j];
        }
        B.apd[i] = a;
        B.ade[i] = b;
    }
    double phF[8], phE[8], mF[8], mE[8];
    for (int i = 0; i < C; ++i) {
        phF[i] = (i == 0) ? 1.0 : (i == C - 1 ? 0.0 : -P.alpp[i]);
        phE[i] = (i == C - 1) ? 1.0 : (i == 0 ? 0.0 : -P.gamp[i]);
    }
    mass_c(phF, mF);
    mass_c(phE, mE);
    for (int j = 0; j < C; ++j) {
        B.cpF += wpd[j] * mF[j];
        B.cpE += wpd[j] * mE[j];
        B.cdF += wde[j] * mF[j];
        B.cdE += wde[j] * mE[j];
    }
    B.cpEp = h6 * wpd[0];
    B.cpFn = h6 * wpd[C - 1];
    B.cdEp = h6 * wde[0];
    B.cdFn = h6 * wde[C - 1];
}

template <typename R>
void cast_rtab(const RTab<double>& s, RTab<R>& d) {
    d.A = (R)s.A;
    d.B = (R)s.B;
    d.Cc = (R)s.Cc;
    for (int i = 0; i < 16; ++i) {
        d.q[i] = (R)s.q[i];
        d.ga[i] = (R)s.ga[i];
        d.alp[i] = (R)s.alp[i];
        d.gap[i] = (R)s.gap[i];
    }
    d.qa = (R)s.qa;
    d.qc = (R)s.qc;
    d.iBF = (R)s.iBF;
    d.aeL = (R)s.aeL;
    d.geL = (R)s.geL;
    for (int l = 0; l < 4; ++l) {
        d.k1[l] = (R)s.k1[l];
        d.k2[l] = (R)s.k2[l];
    }
    d.f1 = (R)s.f1;
    d.f2 = (R)s.f2;
}

template <typename R>
void cast_hb(const HBasis<double>& s, HBasis<R>& d) {
    for (int i = 0; i < 8; ++i) {
        d.apd[i] = (R)s.apd[i];
        d.ade[i] = (R)s.ade[i];
    }
    d.cpF = (R)s.cpF; d.cpE = (R)s.cpE; d.cpEp = (R)s.cpEp; d.cpFn = (R)s.cpFn;
    d.cdF = (R)s.cdF; d.cdE = (R)s.cdE; d.cdEp = (R)s.cdEp; d.cdFn = (R)s.cdFn;
}

template <typename R>
void cast_tab(const HTab& s, CTab<R>& d) {
    for (int i = 0; i < 8; ++i) {
        d.rden[i] = (R)s.rden[i];
        d.gam[i] = (R)s.gam[i];
        d.alpp[i] = (R)s.alpp[i];
        d.gamp[i] = (R)s.gamp[i];
    }
    d.a = (R)s.a;
    d.iBF = (R)s.iBF;
    d.pa = (R)s.pa;
    d.pc = (R)s.pc;
    d.ae = (R)s.ae;
    d.ge = (R)s.ge;
}

template <typename R>
void fill_args(const sch_params& p, int C, ModelArgs<R>& A) {
    memset(&A, 0, sizeof(A));
    const double h = p.L / p.n;
    A.n = p.n;
    A.K = p.K;
    A.K2 = p.K / 2;
    A.M = p.M;
    A.stride = p.n / p.M;
    A.max_iter = p.max_iter;
    A.solver = (p.solver != SCH_SOLVER_AUTO) ? p.solver : (p.dtype == SCH_F32 ? SCH_SOLVER_EA : SCH_SOLVER_LI);
    A.h = (R)h;
    A.dt = (R)p.dt;
    A.c0 = (R)(h / 6.0 - p.mu * p.dt / (2.0 * h));
    A.b0 = (R)(2.0 * h / 3.0 + p.mu * p.dt / h);
    A.c0p = (R)(h / 6.0 + p.mu * p.dt / (2.0 * h));
    A.b0p = (R)(2.0 * h / 3.0 - p.mu * p.dt / h);
    A.dt8 = (R)(p.dt / 8.0);
    A.h6 = (R)(h / 6.0);
    A.tol = (R)p.tol;
    const double a2 = p.alpha * p.alpha;
    A.hel_a = (R)(h / 6.0 - a2 / h);
    A.hel_b = (R)(2.0 * h / 3.0 + 2.0 * a2 / h);
    A.sigma_inv = (R)(1.0 / p.sigma);
    A.dt_d = p.dt;
    for (int j = 0; j < p.K / 2; ++j) {
        A.amp4[j] = (R)(0.25 * p.amps[j]);
        A.rot_c[j] = (R)cos(2.0 * M_PI * (j + 1) / p.n);
        A.rot_s[j] = (R)sin(2.0 * M_PI * (j + 1) / p.n);
        const double sh = sin(M_PI * (j + 1) / p.n);
        A.rot_d[j] = (R)(-4.0 * sh * sh);
    }
    const int TP = p.n / C;
    HTab th, tm, ts, tpic;
    RTab<double> q;
    ctab_host(h / 6.0 - a2 / h, 2.0 * h / 3.0 + 2.0 * a2 / h, C, th);
    ctab_host(h / 6.0, 2.0 * h / 3.0, C, tm);
    ctab_host(h / 6.0 - 1.0 / h, 2.0 * h / 3.0 + 2.0 / h, C, ts);
    ctab_host(h / 6.0 - p.mu * p.dt / (2.0 * h), 2.0 * h / 3.0 + p.mu * p.dt / h, C, tpic);
    cast_tab(th, A.hel);
    cast_tab(tm, A.mass);
    cast_tab(ts, A.smooth);
    cast_tab(tpic, A.pic);
    rtab_host(th, TP, q);
    cast_rtab(q, A.rhel);
    rtab_host(tm, TP, q);
    cast_rtab(q, A.rmass);
    rtab_host(ts, TP, q);
    cast_rtab(q, A.rsmooth);
    rtab_host(tpic, TP, q);
    cast_rtab(q, A.rpic);
    HBasis<double> hb;
    hbasis_host(tpic, th, C, h / 6.0, hb);
    cast_hb(hb, A.hb);
    if (p.noise == SCH_NOISE_MATERN) {
        // Q = n cell weights per step replace the K mode weights
        A.K = p.n;
        A.K2 = 0;
        const double k2 = 1.0 / (p.kappa * p.kappa);
        HTab tg;
        ctab_host(h / 6.0 - k2 / h, 2.0 * h / 3.0 + 2.0 * k2 / h, C, tg);
        cast_tab(tg, A.matern);
        rtab_host(tg, TP, q);
        cast_rtab(q, A.rmatern);
        A.mz = (R)(p.eta * sqrt(h) / 8.0);
        A.mk = p.matern_k;
    }
}

// the warp-per-particle tables: sub-chunks of CS nodes, 64-row reduced systems
void wtab_cast(const HTab& s, const RTab<double>& q, int CS, WTab& d) {
    memset(&d, 0, sizeof(d));
    for (int i = 0; i < CS; ++i) {
        d.rden[i] = (float)s.rden[i];
        d.nar[i] = (float)(-s.a * s.rden[i]);
        d.ngam[i] = (float)(-s.gam[i]);
        d.nalpp[i] = (float)(-s.alpp[i]);
        d.ngamp[i] = (float)(-s.gamp[i]);
    }
    d.na = (float)(-s.a);
    d.iBF = (float)s.iBF;
    d.pa = (float)s.pa;
    d.pc = (float)s.pc;
    d.ae = (float)s.ae;
    d.ge = (float)s.ge;
    d.diag = fmax(fabs(q.A), fabs(q.Cc)) <= ldexp(fabs(q.B), -30) ? 1 : 0;
    d.iB = (float)(1.0 / q.B);
}

bool invert_dense(int n, double* a, double* inv);

// The polynomial form of the lane-centred noise (GArgs npc, npoly): for harmonic j <= K/2
// and x = j d_{H-1}, the polynomials in s of degree WNP - 1 that interpolate cos(x sqrt s)
// and sin(x sqrt s) / sqrt s at the WNP Chebyshev points of [0, 1].  npoly = 1 when they
// reproduce cos(j d_m) and sin(j d_m) to 2^-30 at every offset d_m = tau_m d_{H-1}, m < H
// (tau_m = (m + 1/2) / (H - 1/2)), and need fewer packed FMAs a lane than the tables:
// K/2 WNP for the sums over j and H/2 (2 WNP - 1) for the evaluation, against K/2 H.
// Only the warp-group kernels compile the polynomial form: in the one-warp layout
// (d_{H-1} near 2 pi / 64) it would qualify for K = 10 at n = 1024 alone, and save 4 of
// 80 packed FMAs there.
static void fill_noise_poly(const sch_params& p, int H, GArgs& G) {
    G.npoly = 0;
    const int K2 = p.K / 2, Q = H / 2;
    if (Q < 1 || Q > WNQ_MAX || K2 < 1 || K2 > SCH_MAX_K / 2) return;
    if (K2 * WNP + Q * (2 * WNP - 1) >= K2 * 2 * Q) return;
    const double dmax = 2.0 * M_PI * (H - 0.5) / p.n;
    double V[WNP * WNP], Vi[WNP * WNP], sn[WNP];
    for (int i = 0; i < WNP; ++i) {
        sn[i] = 0.5 * (1.0 + cos(M_PI * (i + 0.5) / WNP));
        for (int k = 0; k < WNP; ++k) V[i * WNP + k] = pow(sn[i], k);
    }
    if (!invert_dense(WNP, V, Vi)) return;
    double err = 0.0;
    for (int j = 1; j <= K2; ++j) {
        const double x = j * dmax;
        double fc[WNP], fs[WNP], cc[WNP], cs[WNP];
        for (int i = 0; i < WNP; ++i) {
            const double r = sqrt(sn[i]);
            fc[i] = cos(x * r);
            fs[i] = sin(x * r) / r;
        }
        for (int k = 0; k < WNP; ++k) {
            cc[k] = cs[k] = 0.0;
            for (int i = 0; i < WNP; ++i) {
                cc[k] += Vi[k * WNP + i] * fc[i];
                cs[k] += Vi[k * WNP + i] * fs[i];
            }
            G.npc[j - 1][k] = make_float2((float)cc[k], (float)cs[k]);
        }
        for (int m = 0; m < H; ++m) {
            const double t = (m + 0.5) / (H - 0.5), s = t * t;
            double ec = 0.0, es = 0.0;
            for (int k = WNP - 1; k >= 0; --k) {
                ec = ec * s + cc[k];
                es = es * s + cs[k];
            }
            err = fmax(err, fmax(fabs(ec - cos(x * t)), fabs(t * es - sin(x * t))));
        }
    }
    G.npoly = err <= ldexp(1.0, -30) ? 1 : 0;
}

void fill_wargs(const sch_params& p, int CS, int rows, WArgs& W) {
    memset(&W, 0, sizeof(W));
    const double h = p.L / p.n;
    const double a2 = p.alpha * p.alpha;
    HTab tp, th;
    RTab<double> q;
    ctab_host(h / 6.0 - p.mu * p.dt / (2.0 * h), 2.0 * h / 3.0 + p.mu * p.dt / h, CS, tp);
    // the Helmholtz matrix scaled by 6/h: its right-hand side is m_{i-1} + 4 m_i + m_{i+1}
    ctab_host((h / 6.0 - a2 / h) * 6.0 / h, (2.0 * h / 3.0 + 2.0 * a2 / h) * 6.0 / h, CS, th);
    rtab_host(tp, rows, q);
    cast_rtab(q, W.rpic);
    wtab_cast(tp, q, CS, W.pic);
    rtab_host(th, rows, q);
    cast_rtab(q, W.rhel);
    wtab_cast(th, q, CS, W.hel);
    // the mode-noise tables about the lane centre: rows / 64 streams of CS pairs, H nodes a half
    const int H = rows / 64 * CS;
    for (int j = 1; j <= p.K / 2 && j <= SCH_MAX_K / 2; ++j)
        for (int q = 0; q < H / 2 && q < WNQ_MAX; ++q) {
            const double dl = 2.0 * M_PI * (H - 1 - q + 0.5) / p.n, dr = 2.0 * M_PI * (q + 0.5) / p.n;
            W.nco[j - 1][q] = make_float2((float)cos(j * dl), (float)cos(j * dr));
            W.nsi[j - 1][q] = make_float2((float)sin(j * dl), (float)sin(j * dr));
        }
    if (p.noise == SCH_NOISE_MATERN) {
        // the Matern operator scaled by 6/h like the Helmholtz one, and the weights likewise
        const double k2 = 1.0 / (p.kappa * p.kappa);
        HTab tg;
        ctab_host((h / 6.0 - k2 / h) * 6.0 / h, (2.0 * h / 3.0 + 2.0 * k2 / h) * 6.0 / h, CS, tg);
        rtab_host(tg, rows, q);
        cast_rtab(q, W.rmat);
        wtab_cast(tg, q, CS, W.mat);
        W.mzw = (float)(p.eta * sqrt(h) / 8.0 * 6.0 / h);
    }
}

// In-place inverse of a dense n x n matrix (Gauss-Jordan with partial pivoting,
// double precision); returns false if it is singular to working precision.
bool invert_dense(int n, double* a, double* inv) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) inv[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(a[r * n + c]) > fabs(a[piv * n + c])) piv = r;
        if (!(fabs(a[piv * n + c]) > 0.0)) return false;
        if (piv != c)
            for (int j = 0; j < n; ++j) {
                double t = a[c * n + j];
                a[c * n + j] = a[piv * n + j];
                a[piv * n + j] = t;
                t = inv[c * n + j];
                inv[c * n + j] = inv[piv * n + j];
                inv[piv * n + j] = t;
            }
        const double d = 1.0 / a[c * n + c];
        for (int j = 0; j < n; ++j) {
            a[c * n + j] *= d;
            inv[c * n + j] *= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = a[r * n + c];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                a[r * n + j] -= f * a[c * n + j];
                inv[r * n + j] -= f * inv[c * n + j];
            }
        }
    }
    return true;
}

// The cross-warp reduced solve of sub-chunk table T with the lane partition of Q
// (S rows per lane) for W warps per particle (see GTab and sch_group.cuh).
bool gtab_host(const HTab& T, const RTab<double>& Q, int S, int W, GTab& G) {
    memset(&G, 0, sizeof(G));
    if (S < 2 || W < 2 || W > GW_MAX) return false;
    // the cyclic system of the lane-last unknowns (the rows of the warps' 32-lane PCR)
    const double LA = -Q.aeL * Q.qa, LB = 1.0 - Q.aeL * Q.qc - Q.geL * Q.qa, LC = -Q.geL * Q.qc;
    double t32[32 * 32], ti[32 * 32];
    memset(t32, 0, sizeof(t32));
    for (int l = 0; l < 32; ++l) {
        t32[l * 32 + (l + 31) % 32] += LA;
        t32[l * 32 + l] += LB;
        t32[l * 32 + (l + 1) % 32] += LC;
    }
    if (!invert_dense(32, t32, ti)) return false;
    // phi = T32^-1 LA e_0, psi = T32^-1 LC e_31, p2 = T32^-1 e_31 at lanes 0 and 31
    const double phi0 = ti[0 * 32 + 0] * LA, phi31 = ti[31 * 32 + 0] * LA;
    const double psi0 = ti[0 * 32 + 31] * LC, psi31 = ti[31 * 32 + 31] * LC;
    // z = (a_0 .. a_{W-1}, b_0 .. b_{W-1}) from the corrected (y_0, y_31) of every warp:
    //   a_w + phi_0 (b_{w-1} - b_w) + psi_0 (a_{w+1} - a_w) = y_0(w)
    //   b_w + phi_31 (b_{w-1} - b_w) + psi_31 (a_{w+1} - a_w) = y_31(w)
    const int n2 = 2 * W;
    double sm[4 * GW_MAX * GW_MAX], gi[4 * GW_MAX * GW_MAX];
    memset(sm, 0, sizeof(sm));
    for (int w = 0; w < W; ++w) {
        const int wp = (w + W - 1) % W, wn = (w + 1) % W;
        double* ra = sm + w * n2;
        double* rb = sm + (W + w) * n2;
        ra[w] += 1.0;
        ra[W + wp] += phi0;
        ra[W + w] -= phi0;
        ra[wn] += psi0;
        ra[w] -= psi0;
        rb[W + w] += 1.0;
        rb[W + wp] += phi31;
        rb[W + w] -= phi31;
        rb[wn] += psi31;
        rb[w] -= psi31;
    }
    if (!invert_dense(n2, sm, gi)) return false;
    // weights of warp 0's b_{-1}, b_0, a_0, a_1 (block circulant: the same for every warp,
    // indexed relative to it)
    const int rows[4] = {W + W - 1, W, 0, 1 % W};
    float* dst[4] = {G.bprev, G.bself, G.aself, G.anext};
    for (int q = 0; q < 4; ++q)
        for (int j = 0; j < n2; ++j) dst[q][j] = (float)gi[rows[q] * n2 + j];
    G.LA = (float)LA;
    G.LC = (float)LC;
    G.iLC = (float)(1.0 / LC);
    G.p2_0 = (float)ti[0 * 32 + 31];
    G.p2_31 = (float)ti[31 * 32 + 31];
    G.cq = (float)(T.ge * Q.q[S - 1]);
    G.geL = (float)Q.geL;
    G.ldiag = fmax(fabs(LA), fabs(LC)) <= ldexp(fabs(LB), -26) ? 1 : 0;
    G.iLB = (float)(1.0 / LB);
    return true;
}

// the warp-group tables: sub-chunks of CS nodes, S = 4 rows per lane, W warps
bool fill_gargs(const sch_params& p, int CS, int W, GArgs& G) {
    const double h = p.L / p.n;
    const double a2 = p.alpha * p.alpha;
    HTab tp, th;
    RTab<double> q;
    const int S = 4;
    ctab_host(h / 6.0 - p.mu * p.dt / (2.0 * h), 2.0 * h / 3.0 + p.mu * p.dt / h, CS, tp);
    ctab_host((h / 6.0 - a2 / h) * 6.0 / h, (2.0 * h / 3.0 + 2.0 * a2 / h) * 6.0 / h, CS, th);
    rtab_host(tp, 32 * S, q);
    if (!gtab_host(tp, q, S, W, G.pic)) return false;
    rtab_host(th, 32 * S, q);
    return gtab_host(th, q, S, W, G.hel);
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

extern "C" {

int sch_create(const sch_params* params, sch_ctx** ctx) {
    if (!params || !ctx) return SCH_ERR_ARG;
    const sch_params& p = *params;
    if (!(p.L > 0) || !(p.dt > 0) || !(p.alpha > 0) || !(p.mu >= 0) || !(p.sigma > 0) || !(p.tol > 0))
        return SCH_ERR_ARG;
    if (p.n <= 0 || p.M <= 0 || p.n % p.M != 0 || p.max_iter < 1) return SCH_ERR_ARG;
    if (p.K < 2 || p.K > SCH_MAX_K || (p.K & 1)) return SCH_ERR_ARG;
    if (p.dtype != SCH_F32 && p.dtype != SCH_F64) return SCH_ERR_ARG;
    if (p.solver < SCH_SOLVER_AUTO || p.solver > SCH_SOLVER_EA) return SCH_ERR_ARG;
    const int C = (p.dtype == SCH_F32) ? 8 : 4;
    if (p.n % C != 0) return SCH_ERR_UNSUPPORTED;
    const int tp = p.n / C;
    if (!pow2(tp) || tp < 32 || tp > 512) return SCH_ERR_UNSUPPORTED;
    if (p.noise != SCH_NOISE_MODES && p.noise != SCH_NOISE_MATERN) return SCH_ERR_ARG;
    const int solver = (p.solver != SCH_SOLVER_AUTO) ? p.solver : (p.dtype == SCH_F32 ? SCH_SOLVER_EA : SCH_SOLVER_LI);
    const bool matern = p.noise == SCH_NOISE_MATERN;
    if (matern) {
        if (!(p.kappa > 0) || !(p.eta >= 0) || p.matern_k < 1 || p.matern_k > 8) return SCH_ERR_ARG;
        if (solver != (p.dtype == SCH_F32 ? SCH_SOLVER_EA : SCH_SOLVER_LI)) return SCH_ERR_UNSUPPORTED;
    }
    const bool warp_fits = p.dtype == SCH_F32 && solver == SCH_SOLVER_EA && (p.n == 256 || p.n == 512 || p.n == 1024);
    if (p.layout == SCH_LAYOUT_WARP && !warp_fits) return SCH_ERR_UNSUPPORTED;
    // one warp per particle wherever it fits, with either noise model, unless another layout is asked for
    const bool warp_ok = warp_fits && (p.layout == SCH_LAYOUT_AUTO || p.layout == SCH_LAYOUT_WARP);
    // several warps per particle: float fields, explicit advection, the mode expansion,
    // n = 2048 or 4096; with 16 nodes a lane also n = 1024 (two warps per particle)
    const bool group_n = p.n == 2048 || p.n == 4096 || (p.n == 1024 && p.layout == SCH_LAYOUT_GROUP16);
    const bool group_fits = p.dtype == SCH_F32 && solver == SCH_SOLVER_EA && !matern && group_n;
    if ((p.layout == SCH_LAYOUT_GROUP || p.layout == SCH_LAYOUT_GROUP16) && !group_fits) return SCH_ERR_UNSUPPORTED;
    if (p.layout < SCH_LAYOUT_AUTO || p.layout > SCH_LAYOUT_GROUP16) return SCH_ERR_ARG;
    const bool group_ok = group_fits && p.layout != SCH_LAYOUT_CTA && p.layout != SCH_LAYOUT_WARP;
    sch_ctx* c = (sch_ctx*)calloc(1, sizeof(sch_ctx));
    if (!c) return SCH_ERR_ARG;
    c->p = p;
    c->C = C;
    c->tp = tp;
    c->matern = matern ? 1 : 0;
    c->Q = matern ? p.n : p.K;
    fill_args(p, C, c->af);
    fill_args(p, C, c->ad);
    if (warp_ok) {
        // one warp per particle: 32 lanes x 2P sub-chunks of wcs nodes, a reduced system of 64 P rows
        const int P = warp_streams(p.n);
        c->wcs = p.n / (64 * P);
        fill_wargs(p, c->wcs, 64 * P, c->wa);
    } else if (group_ok) {
        // W warps per particle, each lane 2 streams x 2 sub-chunks of wcs nodes: 32 nodes a
        // lane (SCH_LAYOUT_GROUP, the default) or 16 (SCH_LAYOUT_GROUP16)
        const int lane_nodes = (p.layout == SCH_LAYOUT_GROUP16) ? 16 : 32;
        c->wcs = lane_nodes / 4;
        c->gw = p.n / (32 * lane_nodes);
        fill_wargs(p, c->wcs, 128, c->wa);
        if (!fill_gargs(p, c->wcs, c->gw, c->ga)) {
            free(c);
            return SCH_ERR_UNSUPPORTED;
        }
        fill_noise_poly(p, 2 * c->wcs, c->ga);   // H = 2 wcs nodes a lane half
    }
    *ctx = c;
    return SCH_OK;
}

int sch_destroy(sch_ctx* ctx) {
    free(ctx);
    return SCH_OK;
}

int sch_layout(const sch_ctx* ctx) {
    if (!ctx) return SCH_ERR_ARG;
    if (ctx->gw) return ctx->wcs == 4 ? SCH_LAYOUT_GROUP16 : SCH_LAYOUT_GROUP;
    return ctx->wcs ? SCH_LAYOUT_WARP : SCH_LAYOUT_CTA;
}

int sch_noise_dim(const sch_ctx* ctx) {
    if (!ctx) return SCH_ERR_ARG;
    return ctx->Q;
}

int sch_noise_form(const sch_ctx* ctx) {
    if (!ctx) return SCH_ERR_ARG;
    if (!ctx->wcs || ctx->matern) return SCH_NOISE_FORM_OTHER;
    return (ctx->gw && ctx->ga.npoly) ? SCH_NOISE_FORM_POLY : SCH_NOISE_FORM_TABLE;
}

size_t pf_resample_workspace_bytes(int N, size_t row_bytes_total) {
    return (size_t)(N > 0 ? N : 0) * row_bytes_total;
}

int sch_u_from_m(sch_ctx* ctx, int N, const void* m, void* u, void* stream) {
    if (!ctx || N < 0 || (N > 0 && (!m || !u))) return SCH_ERR_ARG;
    if (N == 0) return SCH_OK;
    if (ctx->p.dtype == SCH_F32)
        return launch_helm<float, 8>(ctx->af, (const float*)m, (float*)u, 0, N, S(stream));
    return launch_helm<double, 4>(ctx->ad, (const double*)m, (double*)u, 0, N, S(stream));
}

int sch_m_from_u(sch_ctx* ctx, int N, const void* u, void* m, void* stream) {
    if (!ctx || N < 0 || (N > 0 && (!m || !u))) return SCH_ERR_ARG;
    if (N == 0) return SCH_OK;
    if (ctx->p.dtype == SCH_F32)
        return launch_helm<float, 8>(ctx->af, (const float*)u, (float*)m, 1, N, S(stream));
    return launch_helm<double, 4>(ctx->ad, (const double*)u, (double*)m, 1, N, S(stream));
}

int sch_draw_increments(sch_ctx* ctx, int N, int nsteps, uint64_t seed, uint64_t tag, uint64_t ctr,
                        int particle0, void* dW, void* stream) {
    if (!ctx || N < 0 || nsteps < 0 || particle0 < 0) return SCH_ERR_ARG;
    if (N == 0 || nsteps == 0) return SCH_OK;
    if (!dW) return SCH_ERR_ARG;
    const double sq = sqrt(ctx->p.dt);
    // the FP32 Matern noise (one normal per cell) comes from Philox4x32-10
    if (ctx->p.dtype == SCH_F32)
        return launch_draw<float>(N, nsteps, ctx->Q, (float)sq, seed, tag, ctr, particle0, ctx->matern,
                                  (float*)dW, S(stream));
    return launch_draw<double>(N, nsteps, ctx->Q, sq, seed, tag, ctr, particle0, 0, (double*)dW, S(stream));
}

int sch_ensemble_step(sch_ctx* ctx, int N, int nsteps, const void* m, void* m_out, void* u_out,
                      const void* dW, const void* lambda, const void* y, double* nll, double* logG,
                      int32_t* iters, int32_t* status, void* stream) {
    if (!ctx || N < 0 || nsteps < 0) return SCH_ERR_ARG;
    if (N == 0) return SCH_OK;
    if (!m || !m_out || !u_out || (nsteps > 0 && !dW)) return SCH_ERR_ARG;
    if (y && !nll) return SCH_ERR_ARG;
    if (nsteps > 4096) return SCH_ERR_ARG;
    // the Matern kernels hold one step's n cell weights in shared memory, the others a window's noise
    const size_t sm = ctx->matern ? 0
                      : ctx->gw ? gwindow_smem(ctx->wcs, ctx->gw, nsteps, ctx->Q)
                      : ctx->wcs ? wwindow_smem(ctx->wcs, nsteps, ctx->Q)
                      : (ctx->p.dtype == SCH_F32) ? window_smem<float, 8>(ctx->tp, nsteps, ctx->Q)
                                                  : window_smem<double, 4>(ctx->tp, nsteps, ctx->Q);
    if (sm > 200 * 1024) return SCH_ERR_UNSUPPORTED;
    if (ctx->p.dtype == SCH_F32) {
        WindowIO<float> io{nsteps, (const float*)m, (float*)m_out, (float*)u_out, (const float*)dW,
                           (const float*)lambda, (const float*)y, nll, logG, iters, status};
        if (ctx->matern)
            return ctx->wcs ? launch_wwindow_matern(ctx->wcs, ctx->af, ctx->wa, io, N, S(stream))
                            : launch_window_matern<float, 8>(ctx->af, io, N, S(stream));
        if (ctx->gw) return launch_gwindow(ctx->wcs, ctx->gw, ctx->af, ctx->wa, ctx->ga, io, N, S(stream));
        if (ctx->wcs) return launch_wwindow(ctx->wcs, ctx->af, ctx->wa, io, N, S(stream));
        return ctx->af.solver == SCH_SOLVER_EA ? launch_window<float, 8, SCH_SOLVER_EA>(ctx->af, io, N, S(stream))
                                               : launch_window<float, 8, SCH_SOLVER_LI>(ctx->af, io, N, S(stream));
    }
    WindowIO<double> io{nsteps, (const double*)m, (double*)m_out, (double*)u_out, (const double*)dW,
                        (const double*)lambda, (const double*)y, nll, logG, iters, status};
    if (ctx->matern) return launch_window_matern<double, 4>(ctx->ad, io, N, S(stream));
    return ctx->ad.solver == SCH_SOLVER_EA ? launch_window<double, 4, SCH_SOLVER_EA>(ctx->ad, io, N, S(stream))
                                           : launch_window<double, 4, SCH_SOLVER_LI>(ctx->ad, io, N, S(stream));
}

int sch_loglik(sch_ctx* ctx, int N, const void* u, const void* y, const void* dW, const void* lambda,
               int nsteps, double* nll, double* logG, void* stream) {
    if (!ctx || N < 0 || nsteps < 0) return SCH_ERR_ARG;
    if (N == 0) return SCH_OK;
    if (!u || !y || !nll) return SCH_ERR_ARG;
    if (lambda && !dW) return SCH_ERR_ARG;
    if (ctx->p.dtype == SCH_F32)
        return launch_loglik<float>(ctx->af, N, (const float*)u, (const float*)y, (const float*)dW,
                                    (const float*)lambda, nsteps, nll, logG, S(stream));
    return launch_loglik<double>(ctx->ad, N, (const double*)u, (const double*)y, (const double*)dW,
                                 (const double*)lambda, nsteps, nll, logG, S(stream));
}

int pf_temper(int N, const double* nll, const double* logG, double theta, double ess_min, double* wbar,
              double* out, void* stream) {
    if (N <= 0 || N > 16384 || !nll || !wbar || !out) return SCH_ERR_ARG;
    if (!(theta >= 0.0 && theta < 1.0) || !(ess_min > 0.0) || ess_min > N) return SCH_ERR_ARG;
    return launch_temper(N, nll, logG, theta, nullptr, ess_min, 0, wbar, out, S(stream));
}

int pf_temper_halving(int N, const double* nll, const double* logG, double theta, double ess_min, double* wbar,
                      double* out, void* stream) {
    if (N <= 0 || N > 16384 || !nll || !wbar || !out) return SCH_ERR_ARG;
    if (!(theta >= 0.0 && theta < 1.0) || !(ess_min > 0.0) || ess_min > N) return SCH_ERR_ARG;
    return launch_temper(N, nll, logG, theta, nullptr, ess_min, 1, wbar, out, S(stream));
}

int pf_temper_dev(int N, const double* nll, const double* logG, const double* theta_dev, double ess_min, int mode,
                  double* wbar, double* out, void* stream) {
    if (N <= 0 || N > 16384 || !nll || !theta_dev || !wbar || !out) return SCH_ERR_ARG;
    if (!(ess_min > 0.0) || ess_min > N || (mode != PF_TEMPER_LARGEST && mode != PF_TEMPER_HALVING)) return SCH_ERR_ARG;
    return launch_temper(N, nll, logG, 0.0, theta_dev, ess_min, mode == PF_TEMPER_HALVING, wbar, out, S(stream));
}

int pf_resample_gated(int N, const double* wbar, uint64_t seed, uint64_t stage_ctr, const double* gate,
                      int32_t* idx, void* stream) {
    if (N <= 0 || N > 8192 || !wbar || !gate || !idx) return SCH_ERR_ARG;
    return launch_resample_idx(N, wbar, seed, stage_ctr, gate, idx, S(stream));
}

int pf_resample(int N, const double* wbar, uint64_t seed, uint64_t stage_ctr, int32_t* idx, int n_arrays,
                void* const* arrays, const size_t* row_bytes, void* ws, size_t ws_bytes, void* stream) {
    if (N <= 0 || N > 8192 || !wbar || !idx || n_arrays < 0) return SCH_ERR_ARG;
    size_t total = 0;
    for (int a = 0; a < n_arrays; ++a) {
        if (!arrays || !row_bytes || !arrays[a] || row_bytes[a] == 0 || row_bytes[a] % 16 != 0 ||
            ((uintptr_t)arrays[a] & 15))
            return SCH_ERR_ARG;
        total += row_bytes[a];
    }
    // every array's slice of the workspace starts on a 16-byte boundary: N * row_bytes[a] is a multiple of 16
    if (n_arrays > 0 && (!ws || ((uintptr_t)ws & 15) || ws_bytes < pf_resample_workspace_bytes(N, total)))
        return SCH_ERR_WORKSPACE;
    int rc = launch_resample_idx(N, wbar, seed, stage_ctr, nullptr, idx, S(stream));
    if (rc != SCH_OK) return rc;
    unsigned char* w = (unsigned char*)ws;
    for (int a = 0; a < n_arrays; ++a) {
        rc = launch_gather(N, idx, arrays[a], w, row_bytes[a], S(stream));
        if (rc != SCH_OK) return rc;
        rc = launch_copy(w, arrays[a], (size_t)N * row_bytes[a], S(stream));
        if (rc != SCH_OK) return rc;
    }
    return SCH_OK;
}

int pf_gather_rows(int N, const int32_t* idx, const void* src, void* dst, size_t row_bytes, void* stream) {
    if (N < 0 || row_bytes % 4 != 0) return SCH_ERR_ARG;
    if (N == 0 || row_bytes == 0) return SCH_OK;
    const uintptr_t al = row_bytes % 16 == 0 ? 15 : (row_bytes % 8 == 0 ? 7 : 3);
    if (!idx || !src || !dst || ((uintptr_t)src & al) || ((uintptr_t)dst & al) || src == dst) return SCH_ERR_ARG;
    return launch_gather(N, idx, src, dst, row_bytes, S(stream));
}

int sch_synth_obs(sch_ctx* ctx, const void* u, uint64_t seed, uint64_t ctr, void* y, void* stream) {
    if (!ctx || !u || !y) return SCH_ERR_ARG;
    if (ctx->p.dtype == SCH_F32)
        return launch_synth_obs<float>(ctx->af, (const float*)u, seed, ctr, (float*)y, S(stream));
    return launch_synth_obs<double>(ctx->ad, (const double*)u, seed, ctr, (double*)y, S(stream));
}

int pf_diagnostics(sch_ctx* ctx, int N, const void* u, const void* u_truth, double* ws, double* out,
                   void* stream) {
    if (!ctx || N < 2 || !u || !u_truth || !ws || !out) return SCH_ERR_ARG;
    if (ctx->p.dtype == SCH_F32)
        return launch_diag<float>(ctx->af, N, (const float*)u, (const float*)u_truth, ws, out, S(stream));
    return launch_diag<double>(ctx->ad, N, (const double*)u, (const double*)u_truth, ws, out, S(stream));
}

namespace {

int jitter_impl(sch_ctx* ctx, int N, int nsteps, int n_iter, double theta, const double* tstate, double rho,
                uint64_t seed, uint64_t ctr, const void* m_start, void* dW, const void* lambda, const void* y,
                double* nll, double* logG, void* m_end, void* u_end, int32_t* accepts, int32_t* iters,
                int32_t* status, void* stream) {
    if (!ctx || N < 0 || nsteps <= 0 || n_iter < 0) return SCH_ERR_ARG;
    if (!(rho >= 0.0 && rho <= 1.0) || !(theta >= 0.0 && theta <= 1.0)) return SCH_ERR_ARG;
    if (N == 0 || n_iter == 0) return SCH_OK;
    if (!m_start || !dW || !y || !nll || !m_end || !u_end) return SCH_ERR_ARG;
    if (lambda && !logG) return SCH_ERR_ARG;
    const size_t sm = ctx->matern ? 0
                      : ctx->gw ? gjitter_smem(ctx->wcs, ctx->gw, nsteps, ctx->Q)
                      : ctx->wcs ? wjitter_smem(ctx->wcs, nsteps, ctx->Q)
                      : (ctx->p.dtype == SCH_F32) ? jitter_smem<float, 8>(ctx->tp, nsteps, ctx->Q)
                                                  : jitter_smem<double, 4>(ctx->tp, nsteps, ctx->Q);
    if (sm > 200 * 1024) return SCH_ERR_UNSUPPORTED;
    const double sq = sqrt(1.0 - rho * rho);
    if (ctx->p.dtype == SCH_F32) {
        JitterIO<float> io{nsteps, n_iter, 0, theta, tstate, (float)rho, (float)sq, seed, ctr,
                           (const float*)m_start, (float*)dW, (const float*)lambda, (const float*)y, nll, logG,
                           (float*)m_end, (float*)u_end, accepts, iters, status};
        if (ctx->matern)
            return ctx->wcs ? launch_wjitter_matern(ctx->wcs, ctx->af, ctx->wa, io, N, S(stream))
                            : launch_jitter_matern<float, 8>(ctx->af, io, N, S(stream));
        if (ctx->gw) {
            if (ctx->jws && ctx->jws_bytes >= sch_jitter_workspace_bytes(ctx, N, nsteps)) io.guess = (float*)ctx->jws;
            return launch_gjitter(ctx->wcs, ctx->gw, ctx->af, ctx->wa, ctx->ga, io, N, S(stream));
        }
        if (ctx->wcs) return launch_wjitter(ctx->wcs, ctx->af, ctx->wa, io, N, S(stream));
        return ctx->af.solver == SCH_SOLVER_EA ? launch_jitter<float, 8, SCH_SOLVER_EA>(ctx->af, io, N, S(stream))
                                               : launch_jitter<float, 8, SCH_SOLVER_LI>(ctx->af, io, N, S(stream));
    }
    JitterIO<double> io{nsteps, n_iter, 0, theta, tstate, rho, sq, seed, ctr, (const double*)m_start,
                        (double*)dW, (const double*)lambda, (const double*)y, nll, logG, (double*)m_end,
                        (double*)u_end, accepts, iters, status};
    if (ctx->matern) return launch_jitter_matern<double, 4>(ctx->ad, io, N, S(stream));
    return ctx->ad.solver == SCH_SOLVER_EA ? launch_jitter<double, 4, SCH_SOLVER_EA>(ctx->ad, io, N, S(stream))
                                           : launch_jitter<double, 4, SCH_SOLVER_LI>(ctx->ad, io, N, S(stream));
}

}  // namespace

size_t sch_jitter_workspace_bytes(const sch_ctx* ctx, int N, int nsteps) {
    if (!ctx || N <= 0 || nsteps <= 0 || !ctx->gw) return 0;
    return (size_t)N * nsteps * ctx->p.n * sizeof(float);
}

int sch_set_jitter_workspace(sch_ctx* ctx, void* ws, size_t bytes) {
    if (!ctx) return SCH_ERR_ARG;
    if (ws && (reinterpret_cast<uintptr_t>(ws) % 16 != 0)) return SCH_ERR_ARG;
    ctx->jws = bytes ? ws : nullptr;
    ctx->jws_bytes = ws ? bytes : 0;
    return SCH_OK;
}

int pf_jitter(sch_ctx* ctx, int N, int nsteps, int n_iter, double theta, double rho, uint64_t seed,
              uint64_t ctr, const void* m_start, void* dW, const void* lambda, const void* y, double* nll,
              double* logG, void* m_end, void* u_end, int32_t* accepts, int32_t* iters, int32_t* status,
              void* stream) {
    return jitter_impl(ctx, N, nsteps, n_iter, theta, nullptr, rho, seed, ctr, m_start, dW, lambda, y, nll, logG,
                       m_end, u_end, accepts, iters, status, stream);
}

int pf_jitter_dev(sch_ctx* ctx, int N, int nsteps, int n_iter, const double* tstate, double rho, uint64_t seed,
                  uint64_t ctr, const void* m_start, void* dW, const void* lambda, const void* y, double* nll,
                  double* logG, void* m_end, void* u_end, int32_t* accepts, int32_t* iters, int32_t* status,
                  void* stream) {
    if (!tstate) return SCH_ERR_ARG;
    return jitter_impl(ctx, N, nsteps, n_iter, 0.0, tstate, rho, seed, ctr, m_start, dW, lambda, y, nll, logG,
                       m_end, u_end, accepts, iters, status, stream);
}

int pf_gated_stages(sch_ctx* ctx, int N, int nsteps, int n_stages, int first_stage, double ess_min, int mode,
                    double rho, int n_jitter, uint64_t seed, uint64_t cycle, const void* y, void* const* bufs_a,
                    void* const* bufs_b, const double* theta0, double* wbar, int32_t* idx, double* touts,
                    int32_t* accepts, int32_t* iters, int32_t* status, void* const* events, void* stream) {
    if (!ctx || N <= 0 || nsteps <= 0 || n_stages < 1 || first_stage < 0 || n_jitter < 0) return SCH_ERR_ARG;
    if (!y || !bufs_a || !bufs_b || !theta0 || !wbar || !idx || !touts) return SCH_ERR_ARG;
    for (int a = 0; a < PF_STAGE_ARRAYS - 1; ++a)
        if (!bufs_a[a] || !bufs_b[a]) return SCH_ERR_ARG;
    if ((bufs_a[PF_STAGE_ARRAYS - 1] == nullptr) != (bufs_b[PF_STAGE_ARRAYS - 1] == nullptr)) return SCH_ERR_ARG;
    const size_t b = ctx->p.dtype == SCH_F32 ? 4 : 8;
    const size_t rows[PF_STAGE_ARRAYS] = {ctx->p.n * b, ctx->p.n * b, ctx->p.n * b, (size_t)nsteps * ctx->Q * b,
                                          8, 8, (size_t)nsteps * ctx->Q * b};
    void* cur[PF_STAGE_ARRAYS];
    void* nxt[PF_STAGE_ARRAYS];
    for (int a = 0; a < PF_STAGE_ARRAYS; ++a) {
        cur[a] = bufs_a[a];
        nxt[a] = bufs_b[a];
    }
    cudaStream_t st = S(stream);
    for (int k = 0; k < n_stages; ++k) {
        const uint64_t stage_ctr = cycle * 1024 + (uint64_t)(first_stage + k);
        double* out = touts + (size_t)k * 5;
        int rc = pf_temper_dev(N, (const double*)cur[PF_NLL], (const double*)cur[PF_LOGG],
                               k == 0 ? theta0 : touts + (size_t)(k - 1) * 5 + 2, ess_min, mode, wbar, out, stream);
        if (rc != SCH_OK) return rc;
        rc = pf_resample_gated(N, wbar, seed, stage_ctr, out + 4, idx, stream);
        if (rc != SCH_OK) return rc;
        // every state array in one gather launch, then the copies swap roles
        const void* gs[PF_STAGE_ARRAYS];
        void* gd[PF_STAGE_ARRAYS];
        size_t gr[PF_STAGE_ARRAYS];
        int na = 0;
        for (int a = 0; a < PF_STAGE_ARRAYS; ++a) {
            if (!cur[a]) continue;
            gs[na] = cur[a];
            gd[na] = nxt[a];
            gr[na] = rows[a];
            ++na;
        }
        rc = launch_gather_multi(N, idx, na, gs, gd, gr, st);
        if (rc != SCH_OK) return rc;
        for (int a = 0; a < PF_STAGE_ARRAYS; ++a) {
            void* t = cur[a];
            cur[a] = nxt[a];
            nxt[a] = t;
        }
        if (events && events[2 * k]) cudaEventRecord((cudaEvent_t)events[2 * k], st);
        rc = pf_jitter_dev(ctx, N, nsteps, n_jitter, out, rho, seed, stage_ctr * (uint64_t)n_jitter, cur[PF_M_START],
                           cur[PF_DW], cur[PF_LAMBDA], y, (double*)cur[PF_NLL], (double*)cur[PF_LOGG], cur[PF_M_END],
                           cur[PF_U_END], accepts, iters ? iters + (size_t)k * N : nullptr, status, stream);
        if (rc != SCH_OK) return rc;
        if (events && events[2 * k + 1]) cudaEventRecord((cudaEvent_t)events[2 * k + 1], st);
    }
    return SCH_OK;
}

static bool mala_args_ok(const sch_ctx* ctx, int N, int nsteps, int particle0, double theta, double h) {
    return ctx && N >= 0 && nsteps > 0 && particle0 >= 0 && h > 0.0 && theta >= 0.0 && theta <= 1.0;
}

int pf_mala_propose(sch_ctx* ctx, int N, int nsteps, double theta, double h, uint64_t seed, uint64_t ctr,
                    int particle0, const void* dW, const void* lambda, const void* gJ, void* dW_prop, void* stream) {
    if (!mala_args_ok(ctx, N, nsteps, particle0, theta, h)) return SCH_ERR_ARG;
    if (N == 0) return SCH_OK;
    if (!dW || !gJ || !dW_prop) return SCH_ERR_ARG;
    const int K = ctx->Q;
    if (ctx->p.dtype == SCH_F32)
        return launch_mala_propose<float>(N, nsteps, K, theta, h, ctx->p.dt, (const float*)dW, (const float*)lambda,
                                          (const float*)gJ, seed, ctr, particle0, (float*)dW_prop, S(stream));
    return launch_mala_propose<double>(N, nsteps, K, theta, h, ctx->p.dt, (const double*)dW, (const double*)lambda,
                                       (const double*)gJ, seed, ctr, particle0, (double*)dW_prop, S(stream));
}

int pf_mala_accept(sch_ctx* ctx, int N, int nsteps, double theta, double h, uint64_t seed, uint64_t ctr,
                   int particle0, void* dW, const void* dW_prop, const void* lambda, double* J, const double* J_prop,
                   void* gJ, const void* gJ_prop, int32_t* accepts, void* stream) {
    if (!mala_args_ok(ctx, N, nsteps, particle0, theta, h)) return SCH_ERR_ARG;
    if (N == 0) return SCH_OK;
    if (!dW || !dW_prop || !J || !J_prop || !gJ || !gJ_prop) return SCH_ERR_ARG;
    const int NK = nsteps * ctx->Q;
    if (ctx->p.dtype == SCH_F32)
        return launch_mala_accept<float>(N, NK, theta, h, ctx->p.dt, seed, ctr, particle0, (float*)dW,
                                         (const float*)dW_prop, (const float*)lambda, J, J_prop, (float*)gJ,
                                         (const float*)gJ_prop, accepts, S(stream));
    return launch_mala_accept<double>(N, NK, theta, h, ctx->p.dt, seed, ctr, particle0, (double*)dW,
                                      (const double*)dW_prop, (const double*)lambda, J, J_prop, (double*)gJ,
                                      (const double*)gJ_prop, accepts, S(stream));
}

int sch_prior_sample(sch_ctx* ctx, int N, const void* u_truth, uint64_t seed, double scale, void* m, void* u,
                     void* stream) {
    if (!ctx || N < 0) return SCH_ERR_ARG;
    if (N == 0) return SCH_OK;
    if (!u_truth || !m || !u) return SCH_ERR_ARG;
    if (ctx->p.dtype == SCH_F32)
        return launch_prior<float, 8>(ctx->af, (const float*)u_truth, seed, (float)scale, (float*)m, (float*)u,
                                      N, S(stream), 0, 0);
    return launch_prior<double, 4>(ctx->ad, (const double*)u_truth, seed, scale, (double*)m, (double*)u, N,
                                   S(stream), 0, 0);
}

int sch_prior_exp1(sch_ctx* ctx, int N, uint64_t seed, int particle0, void* m, void* u, void* stream) {
    if (!ctx || N < 0 || particle0 < 0) return SCH_ERR_ARG;
    if (N == 0) return SCH_OK;
    if (!m || !u) return SCH_ERR_ARG;
    if (ctx->p.dtype == SCH_F32)
        return launch_prior<float, 8>(ctx->af, nullptr, seed, 0.0f, (float*)m, (float*)u, N, S(stream), 1,
                                      particle0);
    return launch_prior<double, 4>(ctx->ad, nullptr, seed, 0.0, (double*)m, (double*)u, N, S(stream), 1, particle0);
}

static size_t adjoint_ws_per(const sch_ctx* ctx, int nsteps, int ckpt) {
    const size_t ncp = (size_t)((nsteps + ckpt - 1) / ckpt);
    const size_t b = (ctx->p.dtype == SCH_F32) ? sizeof(float) : sizeof(double);
    return (ncp + 2 * (size_t)(ckpt + 1)) * (size_t)ctx->p.n * b;
}

size_t sch_adjoint_workspace_bytes(const sch_ctx* ctx, int N, int nsteps, int ckpt) {
    if (!ctx || N <= 0 || nsteps <= 0 || ckpt <= 0) return 0;
    return (size_t)N * adjoint_ws_per(ctx, nsteps, ckpt);
}

// elements per particle of pf_nudge's workspace: the window start and the adjoint's
// region, and with the Matern noise the optimiser's vectors (nudge_matern_ws_elems)
static size_t nudge_ws_per(const sch_ctx* ctx, int nsteps, int ckpt) {
    const size_t b = (ctx->p.dtype == SCH_F32) ? sizeof(float) : sizeof(double);
    const size_t adj = (adjoint_ws_per(ctx, nsteps, ckpt) + (size_t)ctx->p.n * b) / b;
    return ctx->matern ? nudge_matern_ws_elems(adj, (size_t)nsteps * ctx->Q, b) : adj;
}

size_t pf_nudge_workspace_bytes(const sch_ctx* ctx, int N, int nsteps, int ckpt) {
    if (!ctx || N <= 0 || nsteps <= 0 || ckpt <= 0) return 0;
    const size_t b = (ctx->p.dtype == SCH_F32) ? sizeof(float) : sizeof(double);
    return (size_t)N * nudge_ws_per(ctx, nsteps, ckpt) * b;
}

int sch_adjoint_window(sch_ctx* ctx, int N, int nsteps, int ckpt, const void* m_start, const void* dW,
                       const void* lambda, const void* y, double* J, void* g_lambda, void* g_dW, void* g_m0,
                       int32_t* iters, int32_t* status, void* ws, size_t ws_bytes, void* stream) {
    if (!ctx || N < 0 || nsteps <= 0 || ckpt <= 0 || nsteps > 4096) return SCH_ERR_ARG;
    if (N == 0) return SCH_OK;
    if (!m_start || !dW || !y || !J || !g_lambda) return SCH_ERR_ARG;
    if (!ws || ws_bytes < sch_adjoint_workspace_bytes(ctx, N, nsteps, ckpt)) return SCH_ERR_WORKSPACE;
    const size_t per = adjoint_ws_per(ctx, nsteps, ckpt);
    if (ctx->matern) {
        // one step's cell weights in shared memory, gradients per cell (Q = n)
        if (ctx->p.dtype == SCH_F32) {
            AdjointIO<float> io{nsteps, ckpt, (const float*)m_start, (const float*)dW, (const float*)lambda,
                                (const float*)y, J, (float*)g_lambda, (float*)g_dW, (float*)g_m0, (float*)ws,
                                per / sizeof(float), iters, status};
            return launch_adjoint_matern<float, 8>(ctx->af, io, N, S(stream));
        }
        AdjointIO<double> io{nsteps, ckpt, (const double*)m_start, (const double*)dW, (const double*)lambda,
                             (const double*)y, J, (double*)g_lambda, (double*)g_dW, (double*)g_m0, (double*)ws,
                             per / sizeof(double), iters, status};
        return launch_adjoint_matern<double, 4>(ctx->ad, io, N, S(stream));
    }
    if (ctx->p.dtype == SCH_F32) {
        if (adjoint_smem<float, 8>(ctx->tp, nsteps, ctx->p.K) > 200 * 1024) return SCH_ERR_UNSUPPORTED;
        AdjointIO<float> io{nsteps, ckpt, (const float*)m_start, (const float*)dW, (const float*)lambda,
                            (const float*)y, J, (float*)g_lambda, (float*)g_dW, (float*)g_m0, (float*)ws,
                            per / sizeof(float), iters, status};
        return ctx->af.solver == SCH_SOLVER_EA ? launch_adjoint<float, 8, SCH_SOLVER_EA>(ctx->af, io, N, S(stream))
                                               : launch_adjoint<float, 8, SCH_SOLVER_LI>(ctx->af, io, N, S(stream));
    }
    if (adjoint_smem<double, 4>(ctx->tp, nsteps, ctx->p.K) > 200 * 1024) return SCH_ERR_UNSUPPORTED;
    AdjointIO<double> io{nsteps, ckpt, (const double*)m_start, (const double*)dW, (const double*)lambda,
                         (const double*)y, J, (double*)g_lambda, (double*)g_dW, (double*)g_m0, (double*)ws,
                         per / sizeof(double), iters, status};
    return ctx->ad.solver == SCH_SOLVER_EA ? launch_adjoint<double, 4, SCH_SOLVER_EA>(ctx->ad, io, N, S(stream))
                                           : launch_adjoint<double, 4, SCH_SOLVER_LI>(ctx->ad, io, N, S(stream));
}

int pf_nudge(sch_ctx* ctx, int N, int nsteps, int mode, int max_iter, double gtol, int ckpt, uint64_t seed,
             uint64_t ctr, const void* m_start, const void* y, void* lambda, void* dW, double* J, int32_t* iters,
             int32_t* status, void* ws, size_t ws_bytes, void* stream) {
    if (!ctx || N < 0 || nsteps <= 0 || ckpt <= 0 || max_iter < 0 || nsteps > 4096) return SCH_ERR_ARG;
    if (mode != PF_NUDGE_SEQUENTIAL && mode != PF_NUDGE_OPEN_LOOP) return SCH_ERR_ARG;
    if (!(gtol >= 0.0)) return SCH_ERR_ARG;
    if (N == 0) return SCH_OK;
    if (!m_start || !y || !lambda || !dW || !J) return SCH_ERR_ARG;
    if (!ws || ws_bytes < pf_nudge_workspace_bytes(ctx, N, nsteps, ckpt)) return SCH_ERR_WORKSPACE;
    const size_t per = nudge_ws_per(ctx, nsteps, ckpt);
    if (ctx->matern) {
        // one drift per cell; the optimiser's vectors in the workspace, one step's weights in smem
        if (ctx->p.dtype == SCH_F32) {
            NudgeIO<float> io{nsteps, ckpt, mode, max_iter, 0, gtol, seed, ctr, (const float*)m_start,
                              (const float*)y, (float*)lambda, (float*)dW, J, (float*)ws, per, iters, status};
            return launch_nudge_matern<float, 8>(ctx->af, io, N, S(stream));
        }
        NudgeIO<double> io{nsteps, ckpt, mode, max_iter, 0, gtol, seed, ctr, (const double*)m_start,
                           (const double*)y, (double*)lambda, (double*)dW, J, (double*)ws, per, iters, status};
        return launch_nudge_matern<double, 4>(ctx->ad, io, N, S(stream));
    }
    if (ctx->p.dtype == SCH_F32) {
        if (nudge_smem<float, 8>(ctx->tp, nsteps, ctx->p.K) > 200 * 1024) return SCH_ERR_UNSUPPORTED;
        NudgeIO<float> io{nsteps, ckpt, mode, max_iter, 0, gtol, seed, ctr, (const float*)m_start,
                          (const float*)y, (float*)lambda, (float*)dW, J, (float*)ws, per, iters, status};
        return ctx->af.solver == SCH_SOLVER_EA ? launch_nudge<float, 8, SCH_SOLVER_EA>(ctx->af, io, N, S(stream))
                                               : launch_nudge<float, 8, SCH_SOLVER_LI>(ctx->af, io, N, S(stream));
    }
    if (nudge_smem<double, 4>(ctx->tp, nsteps, ctx->p.K) > 200 * 1024) return SCH_ERR_UNSUPPORTED;
    NudgeIO<double> io{nsteps, ckpt, mode, max_iter, 0, gtol, seed, ctr, (const double*)m_start,
                       (const double*)y, (double*)lambda, (double*)dW, J, (double*)ws, per, iters, status};
    return ctx->ad.solver == SCH_SOLVER_EA ? launch_nudge<double, 4, SCH_SOLVER_EA>(ctx->ad, io, N, S(stream))
                                           : launch_nudge<double, 4, SCH_SOLVER_LI>(ctx->ad, io, N, S(stream));
}

}  // extern "C"
