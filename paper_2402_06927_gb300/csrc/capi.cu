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
    ModelArgs<float> af;
    ModelArgs<double> ad;
};

namespace {

// Chunk-partition coefficients of the symmetric circulant tridiagonal matrix
// with off-diagonal a and diagonal b, for chunks of C rows (double precision).
void ctab_host(double a, double b, int C, CTab<double>& T) {
    double al[8], ga[8];
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

template <typename R>
void cast_tab(const CTab<double>& s, CTab<R>& d) {
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
    for (int j = 0; j < p.K / 2; ++j) A.amp4[j] = (R)(0.25 * p.amps[j]);
    CTab<double> t;
    ctab_host(h / 6.0 - a2 / h, 2.0 * h / 3.0 + 2.0 * a2 / h, C, t);
    cast_tab(t, A.hel);
    ctab_host(h / 6.0, 2.0 * h / 3.0, C, t);
    cast_tab(t, A.mass);
    ctab_host(h / 6.0 - 1.0 / h, 2.0 * h / 3.0 + 2.0 / h, C, t);
    cast_tab(t, A.smooth);
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
    const int C = (p.dtype == SCH_F32) ? 8 : 4;
    if (p.n % C != 0) return SCH_ERR_UNSUPPORTED;
    const int tp = p.n / C;
    if (!pow2(tp) || tp < 32 || tp > 512) return SCH_ERR_UNSUPPORTED;
    sch_ctx* c = (sch_ctx*)calloc(1, sizeof(sch_ctx));
    if (!c) return SCH_ERR_ARG;
    c->p = p;
    c->C = C;
    c->tp = tp;
    fill_args(p, C, c->af);
    fill_args(p, C, c->ad);
    *ctx = c;
    return SCH_OK;
}

int sch_destroy(sch_ctx* ctx) {
    free(ctx);
    return SCH_OK;
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
    if (ctx->p.dtype == SCH_F32)
        return launch_draw<float>(N, nsteps, ctx->p.K, (float)sq, seed, tag, ctr, particle0, (float*)dW,
                                  S(stream));
    return launch_draw<double>(N, nsteps, ctx->p.K, sq, seed, tag, ctr, particle0, (double*)dW, S(stream));
}

int sch_ensemble_step(sch_ctx* ctx, int N, int nsteps, const void* m, void* m_out, void* u_out,
                      const void* dW, const void* lambda, const void* y, double* nll, double* logG,
                      int32_t* iters, int32_t* status, void* stream) {
    if (!ctx || N < 0 || nsteps < 0) return SCH_ERR_ARG;
    if (N == 0) return SCH_OK;
    if (!m || !m_out || !u_out || (nsteps > 0 && !dW)) return SCH_ERR_ARG;
    if (y && !nll) return SCH_ERR_ARG;
    if (nsteps > 4096) return SCH_ERR_ARG;
    const size_t sm = (ctx->p.dtype == SCH_F32) ? window_smem<float, 8>(ctx->tp, nsteps, ctx->p.K)
                                                 : window_smem<double, 4>(ctx->tp, nsteps, ctx->p.K);
    if (sm > 200 * 1024) return SCH_ERR_UNSUPPORTED;
    if (ctx->p.dtype == SCH_F32) {
        WindowIO<float> io{nsteps, (const float*)m, (float*)m_out, (float*)u_out, (const float*)dW,
                           (const float*)lambda, (const float*)y, nll, logG, iters, status};
        return launch_window<float, 8>(ctx->af, io, N, S(stream));
    }
    WindowIO<double> io{nsteps, (const double*)m, (double*)m_out, (double*)u_out, (const double*)dW,
                        (const double*)lambda, (const double*)y, nll, logG, iters, status};
    return launch_window<double, 4>(ctx->ad, io, N, S(stream));
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
    return launch_temper(N, nll, logG, theta, ess_min, wbar, out, S(stream));
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
    int rc = launch_resample_idx(N, wbar, seed, stage_ctr, idx, S(stream));
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

int pf_jitter(sch_ctx* ctx, int N, int nsteps, int n_iter, double theta, double rho, uint64_t seed,
              uint64_t ctr, const void* m_start, void* dW, const void* lambda, const void* y, double* nll,
              double* logG, void* m_end, void* u_end, int32_t* accepts, int32_t* iters, int32_t* status,
              void* stream) {
    if (!ctx || N < 0 || nsteps <= 0 || n_iter < 0) return SCH_ERR_ARG;
    if (!(rho >= 0.0 && rho <= 1.0) || !(theta >= 0.0 && theta <= 1.0)) return SCH_ERR_ARG;
    if (N == 0 || n_iter == 0) return SCH_OK;
    if (!m_start || !dW || !y || !nll || !m_end || !u_end) return SCH_ERR_ARG;
    if (lambda && !logG) return SCH_ERR_ARG;
    const size_t sm = (ctx->p.dtype == SCH_F32) ? jitter_smem<float, 8>(ctx->tp, nsteps, ctx->p.K)
                                                 : jitter_smem<double, 4>(ctx->tp, nsteps, ctx->p.K);
    if (sm > 200 * 1024) return SCH_ERR_UNSUPPORTED;
    const double sq = sqrt(1.0 - rho * rho);
    if (ctx->p.dtype == SCH_F32) {
        JitterIO<float> io{nsteps, n_iter, 0, theta, (float)rho, (float)sq, seed, ctr, (const float*)m_start,
                           (float*)dW, (const float*)lambda, (const float*)y, nll, logG, (float*)m_end,
                           (float*)u_end, accepts, iters, status};
        return launch_jitter<float, 8>(ctx->af, io, N, S(stream));
    }
    JitterIO<double> io{nsteps, n_iter, 0, theta, rho, sq, seed, ctr, (const double*)m_start, (double*)dW,
                        (const double*)lambda, (const double*)y, nll, logG, (double*)m_end, (double*)u_end,
                        accepts, iters, status};
    return launch_jitter<double, 4>(ctx->ad, io, N, S(stream));
}

int sch_prior_sample(sch_ctx* ctx, int N, const void* u_truth, uint64_t seed, double scale, void* m, void* u,
                     void* stream) {
    if (!ctx || N < 0) return SCH_ERR_ARG;
    if (N == 0) return SCH_OK;
    if (!u_truth || !m || !u) return SCH_ERR_ARG;
    if (ctx->p.dtype == SCH_F32)
        return launch_prior<float, 8>(ctx->af, (const float*)u_truth, seed, (float)scale, (float*)m, (float*)u,
                                      N, S(stream));
    return launch_prior<double, 4>(ctx->ad, (const double*)u_truth, seed, scale, (double*)m, (double*)u, N,
                                   S(stream));
}

}  // extern "C"
