/*
 * sch.h -- C ABI of the GB300 (sm_103a) particle-filter library for the
 * viscous stochastic Camassa-Holm (SALT) equation.
 *
 * Method: Cotter, Crisan, Singh, "Data assimilation for the stochastic
 * Camassa-Holm equation using particle filtering" (arXiv 2402.06927).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an int status: SCH_OK (0) or a negative SCH_ERR_*.
 *    Argument errors are detected on the host before anything is launched.
 *  - Array arguments are DEVICE pointers owned by the caller (for instance
 *    PyTorch tensors), row-major and contiguous.  "real" means the field
 *    precision chosen in sch_params.dtype: double for SCH_F64, float for
 *    SCH_F32.  Log-weights, likelihoods and weights are always double.
 *  - Particle data (the (X_start, dW) representation of Sec. 3.1.2):
 *      m, u      real   [N][n]       momentum and velocity nodal values
 *      dW        real   [N][Ns][K]   Brownian increments of the window
 *      lambda    real   [N][Ns][K]   nudging drift (NULL means zero)
 *      y         real   [M]          observations at x_j = j L / M
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy stream).
 *    Calls are asynchronous on that stream, allocate no device memory and do
 *    not synchronise; sch_create / sch_destroy allocate and free the host-side
 *    context.  Device-side failures (Picard non-convergence, non-finite
 *    values) are reported per particle in the optional int32 `status` array:
 *    bit SCH_DEV_NOCONVERGE or SCH_DEV_NONFINITE; 0 = fine.
 *  - Sizes: n must equal C * TP with TP a power of two in [32, 512], where
 *    C = 8 for SCH_F32 and C = 4 for SCH_F64 (so n in {256 .. 4096} for f32,
 *    {128 .. 2048} for f64); n % M == 0; K even, 2 <= K <= 64.
 *
 * Random numbers: Philox4x64-10 (Salmon et al., SC'11), key (seed, purpose),
 * counter (block, step, particle, stream counter); normals by Box-Muller on
 * 53-bit uniforms.  Purposes are the SCH_TAG_* values below.
 */
#ifndef SCH_H_
#define SCH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SCH_OK = 0,
    SCH_ERR_ARG = -1,          /* bad size, pointer or parameter */
    SCH_ERR_CUDA = -2,         /* a CUDA runtime call failed */
    SCH_ERR_NOCONVERGE = -3,   /* returned by host helpers that read status */
    SCH_ERR_NONFINITE = -4,
    SCH_ERR_WORKSPACE = -5,    /* workspace missing or too small */
    SCH_ERR_UNSUPPORTED = -6   /* size outside the compiled configurations */
};

enum { SCH_DEV_NOCONVERGE = 1, SCH_DEV_NONFINITE = 2 };

enum { SCH_F64 = 0, SCH_F32 = 1 };

/* Picard iteration used to solve each implicit-midpoint step (the paper names
 * none; both reach the same fixed point of Eq. fde1 to params.tol):
 *   SCH_SOLVER_LI  linearly implicit: dv frozen at the last iterate, the cyclic
 *                  tridiagonal (M + mu dt/2 K + 1/2 A_dv) solved each iteration;
 *   SCH_SOLVER_EA  explicit advection: A(mbar, dv) at the last iterate moved to
 *                  the right-hand side, so only the constant matrices
 *                  M + mu dt/2 K and M + alpha^2 K are solved (cheaper
 *                  iterations, slower contraction);
 *   SCH_SOLVER_AUTO  EA for SCH_F32, LI for SCH_F64. */
enum { SCH_SOLVER_AUTO = 0, SCH_SOLVER_LI = 1, SCH_SOLVER_EA = 2 };

/* Kernel layout of sch_ensemble_step and pf_jitter:
 *   SCH_LAYOUT_CTA     one CTA of n/8 (float) or n/4 (double) threads per particle;
 *   SCH_LAYOUT_WARP    one warp per particle, packed f32x2 arithmetic: float
 *                      fields, the SCH_SOLVER_EA solver and n = 256, 512 or 1024
 *                      only (sch_create returns SCH_ERR_UNSUPPORTED otherwise);
 *   SCH_LAYOUT_GROUP   n/1024 warps per particle (one CTA), each warp holding 1024
 *                      consecutive nodes in the WARP layout's registers (32 a lane);
 *                      the cyclic solves are completed across the warps through
 *                      shared memory, one CTA barrier per solve: float fields,
 *                      SCH_SOLVER_EA, the mode expansion and n = 2048 or 4096 only;
 *   SCH_LAYOUT_GROUP16 the same with 16 nodes a lane (n/512 warps per particle),
 *                      also at n = 1024 (two warps per particle; only when asked
 *                      for: AUTO takes WARP there);
 *   SCH_LAYOUT_AUTO    WARP where it applies (with either noise model), else
 *                      GROUP where it applies, else CTA.
 * All compute the same iteration; results agree to rounding. */
enum { SCH_LAYOUT_AUTO = 0, SCH_LAYOUT_CTA = 1, SCH_LAYOUT_WARP = 2, SCH_LAYOUT_GROUP = 3,
       SCH_LAYOUT_GROUP16 = 4 };

/* SALT noise model (sch_params.noise):
 *   SCH_NOISE_MODES   dU = sum_k xi_k (dW_k + lambda_k dt) over K mode functions
 *                     (the expansion Sec. 2 contrasts with its own); Q = K
 *                     Brownian motions per step;
 *   SCH_NOISE_MATERN  the paper's Matern field (Eq. noise_solve, Eq. noise_solve2):
 *                     one Brownian motion per cell, dW_h = sum_c h^{-1/2} 1_c dW_c
 *                     in DG0, and matern_k chained P1 solves
 *                     (U_j, v) + kappa^-2 (U_j', v') = eta (dW_h, v) for j = 1,
 *                     (U_{j-1}, v) after, dU = U_k; Q = n.  The drift lambda is a
 *                     DG0 field added to dW (dW_c + lambda_c dt).  Default solver
 *                     of the precision; the warp layout where it fits (FP32,
 *                     n = 256, 512, 1024) unless SCH_LAYOUT_CTA is asked for.  The adjoint, nudging and MALA
 *                     entry points take it: gradients and drifts per cell, and pf_nudge
 *                     keeps the optimiser's vectors in its workspace.
 * Every noise array dW, lambda of this API is [N][nsteps][Q]. */
enum { SCH_NOISE_MODES = 0, SCH_NOISE_MATERN = 1 };

enum {
    SCH_TAG_PRIOR_DW = 1, SCH_TAG_PCN = 2, SCH_TAG_PCN_ACCEPT = 3, SCH_TAG_RESAMPLE = 4,
    SCH_TAG_TRUTH = 5, SCH_TAG_OBS = 6, SCH_TAG_INIT = 7, SCH_TAG_NUDGE = 8,
    SCH_TAG_MALA = 9, SCH_TAG_MALA_ACCEPT = 10
};

#define SCH_MAX_K 64

/* Model and observation parameters (Sec. 2 and Sec. 3 of the paper). */
typedef struct {
    double L;            /* period of the domain [0, L) */
    int32_t n;           /* cells = nodes of the periodic P1 mesh, h = L / n */
    double alpha;        /* Helmholtz length: m = u - alpha^2 u_xx (Eq. CHe1) */
    double mu;           /* viscosity */
    double dt;           /* model time step */
    int32_t K;           /* number of SALT mode functions (even) */
    double amps[SCH_MAX_K / 2];  /* a_j, j = 1..K/2: xi_{2j-2} = a_j sin(2 pi j x/L),
                                    xi_{2j-1} = a_j cos(2 pi j x/L) */
    int32_t M;           /* observation points x_j = j L / M (on nodes); in every
                            observation vector y [M] an entry that is NaN is not
                            observed (e.g. Exp 2's half domain, Sec. 4) */
    double sigma;        /* observation noise standard deviation */
    double tol;          /* Picard stop: max|dm| <= tol * max(1, max|m|) */
    int32_t max_iter;    /* Picard iteration limit per step */
    int32_t dtype;       /* SCH_F64 or SCH_F32: precision of fields, dW, lambda */
    int32_t solver;      /* SCH_SOLVER_* */
    int32_t layout;      /* SCH_LAYOUT_* */
    int32_t noise;       /* SCH_NOISE_MODES (0) or SCH_NOISE_MATERN */
    double kappa;        /* Matern: inverse length scale, > 0 */
    double eta;          /* Matern: amplitude, >= 0 */
    int32_t matern_k;    /* Matern: number of chained solves, 1 .. 8 */
} sch_params;

typedef struct sch_ctx sch_ctx;

/* Create a context: validates the parameters and precomputes the scalar
 * coefficients of the discretisation (host memory only; no device call).
 * Returns SCH_ERR_ARG / SCH_ERR_UNSUPPORTED for invalid or uncompiled sizes. */
int sch_create(const sch_params* params, sch_ctx** ctx);
int sch_destroy(sch_ctx* ctx);

/* The kernel layout a context runs sch_ensemble_step and pf_jitter with:
 * SCH_LAYOUT_CTA, SCH_LAYOUT_WARP, SCH_LAYOUT_GROUP or SCH_LAYOUT_GROUP16
 * (SCH_LAYOUT_AUTO resolved); SCH_ERR_ARG for a NULL context.  Host only. */
int sch_layout(const sch_ctx* ctx);

/* Q, the Brownian motions per model step: K for SCH_NOISE_MODES, n for
 * SCH_NOISE_MATERN (the last axis of every dW and lambda array); SCH_ERR_ARG for
 * a NULL context.  Host only. */
int sch_noise_dim(const sch_ctx* ctx);

/* How the warp and warp-group kernels synthesise the mode noise of Eq. sde1 at a
 * lane's nodes (Sec. 2's K SALT modes; both forms sum the same trigonometric series
 * about the lane's centre):
 *   SCH_NOISE_FORM_TABLE  tabulated cos(j d), sin(j d) of the lane's node offsets d;
 *   SCH_NOISE_FORM_POLY   per harmonic, polynomials in (d / d_max)^2 fitted on the host
 *                         (Chebyshev interpolation, double precision), chosen in the
 *                         warp-group layouts when they reproduce cos(j d) and sin(j d) to
 *                         2^-30 at every offset and take the lane fewer operations than
 *                         the tables;
 *   SCH_NOISE_FORM_OTHER  neither (the CTA layout, the Matern noise).
 * SCH_ERR_ARG for a NULL context.  Host only. */
enum { SCH_NOISE_FORM_OTHER = 0, SCH_NOISE_FORM_TABLE = 1, SCH_NOISE_FORM_POLY = 2 };
int sch_noise_form(const sch_ctx* ctx);

/* Workspace bytes pf_resample needs to gather `row_bytes_total` bytes per
 * particle in place for N particles. */
size_t pf_resample_workspace_bytes(int N, size_t row_bytes_total);

/* u = H^{-1} M m for every particle: the Helmholtz relation of Eq. sde1
 * (first line), (u, psi) + alpha^2 (u_x, psi_x) = (m, psi) on P1.
 * m, u: real [N][n]. */
int sch_u_from_m(sch_ctx* ctx, int N, const void* m, void* u, void* stream);

/* m = M^{-1} (M + alpha^2 K) u: the P1 momentum of a velocity (Eq. CHe1). */
int sch_m_from_u(sch_ctx* ctx, int N, const void* u, void* m, void* stream);

/* Draw dW[p][s][k] = sqrt(dt) z, z ~ N(0,1) from Philox keyed
 * (seed, tag) and counter (k / 4, s, particle0 + p, ctr).  dW: real [N][nsteps][K].
 * The prior of the window increments: iid N(0, dt) (Sec. 3.1.2).  The generator is
 * Philox4x64-10 (Box-Muller on 53-bit uniforms), except for an FP32 context with the
 * Matern noise, which draws from Philox4x32-10 (key (seed mod 2^32, (seed >> 32) mod
 * 2^16 + 2^16 tag), counter words mod 2^32, Box-Muller on 32-bit uniforms); the PCN
 * proposals of pf_jitter on such a context come from the same generator. */
int sch_draw_increments(sch_ctx* ctx, int N, int nsteps, uint64_t seed, uint64_t tag,
                        uint64_t ctr, int particle0, void* dW, void* stream);

/* Ensemble propagation (Sec. 2, Eq. fde1): advance each particle `nsteps`
 * implicit-midpoint steps with SALT increments
 *   dU^s(x_i) = sum_k xi_k(x_i) (dW[p][s][k] + lambda[p][s][k] dt),
 * each step solved by linearly implicit Picard iteration to params.tol.
 *   m      real [N][n]  in: start momentum; out: end momentum (may alias m_out)
 *   m_out  real [N][n]  out (may equal m)
 *   u_out  real [N][n]  out: end velocity
 *   dW, lambda          real [N][nsteps][K]; lambda may be NULL
 *   y      real [M]     optional: when non-NULL the kernel also writes the
 *                       observation NLL (Eq. loglikeq) of the end state into
 *                       nll[N] and the Girsanov log-weight into logG[N]
 *                       (Eq. girsanov DG approx), both double
 *   iters  int32 [N]    optional: Picard iterations summed over the steps
 *   status int32 [N]    optional: SCH_DEV_* flags */
int sch_ensemble_step(sch_ctx* ctx, int N, int nsteps, const void* m, void* m_out, void* u_out,
                      const void* dW, const void* lambda, const void* y, double* nll,
                      double* logG, int32_t* iters, int32_t* status, void* stream);

/* Observation log-likelihood and Girsanov weight of given end states:
 *   nll[p]  = 1/2 sum_j ((u[p][j n/M] - y_j) / sigma)^2      (Eq. loglikeq)
 *   logG[p] = -sum_{s,k} (lambda dW + 1/2 lambda^2 dt)        (Eq. girsanov DG approx)
 * u real [N][n]; dW, lambda real [N][nsteps][K] (lambda NULL => logG = 0;
 * dW may then be NULL too).  Differences in real, sums in double. */
int sch_loglik(sch_ctx* ctx, int N, const void* u, const void* y, const void* dW,
               const void* lambda, int nsteps, double* nll, double* logG, void* stream);

/* Adaptive tempering (Sec. 3.1.2): given nll[N] and logG[N] (double; logG may
 * be NULL for zero), phi = nll - logG = -log W~, and the current temperature
 * theta, find the largest dtheta in (0, 1 - theta] with
 * ESS(exp(-dtheta phi)) >= ess_min (Eq. ess): the whole step if it passes,
 * else the root of the monotone ESS(dtheta) - ess_min on [0, 1 - theta],
 * bracketed to a relative width of 2^-46 (Illinois regula falsi with
 * bisection safeguards) and taken from the passing side; a root below
 * (1 - theta) 2^-60 gives (1 - theta) 2^-60.  Writes wbar[N] (double, normalised weights at
 * dtheta) and out[4] = {dtheta, ESS at dtheta, theta_new, ESS of the whole
 * remaining step}; theta_new is exactly 1.0 when the remaining step was taken.
 * N <= 16384. */
int pf_temper(int N, const double* nll, const double* logG, double theta, double ess_min,
              double* wbar, double* out, void* stream);

/* Adaptive tempering by halving (Sec. 3.1.2, "repeatedly reduces dtheta until the
 * condition holds", read literally): the first of dtheta = (1 - theta) 2^-k,
 * k = 0, 1, .., 60, with ESS >= ess_min; if none passes, (1 - theta) 2^-60.
 * Arguments, outputs and errors as pf_temper. */
int pf_temper_halving(int N, const double* nll, const double* logG, double theta, double ess_min,
                      double* wbar, double* out, void* stream);

/* Device-gated tempering stage, for a cycle whose stages are all enqueued without a
 * host round trip.  The temperature is read from the device scalar theta_dev (the
 * previous stage's out[2], or a device 0.0 for the first stage).  mode:
 * PF_TEMPER_LARGEST (as pf_temper) or PF_TEMPER_HALVING (as pf_temper_halving).
 * Writes out[5]: out[0..3] as pf_temper, out[4] = 1 when the stage is active.  A
 * stage that starts at theta >= 1 is inactive: it writes {0, 0, 1, 0, 0} and leaves
 * wbar untouched. */
enum { PF_TEMPER_LARGEST = 0, PF_TEMPER_HALVING = 1 };
int pf_temper_dev(int N, const double* nll, const double* logG, const double* theta_dev, double ess_min,
                  int mode, double* wbar, double* out, void* stream);

/* Systematic resampling (Sec. 3.1.1) on exact integers: q_i = floor(wbar_i 2^50),
 * C_j = q_0 + .. + q_j, T = C_{N-1}; slot i takes the smallest j with
 * C_j > floor((i 2^53 + U) T / (N 2^53)), U = (Philox (seed, SCH_TAG_RESAMPLE,
 * counter (0, 0, 0, stage_ctr)) word 0) >> 11.  Writes idx[N] (int32).
 * If n_arrays > 0, also gathers each arrays[a] (device pointer, N rows of
 * row_bytes[a] bytes, rows 16-byte aligned) in place: row i <- old row idx[i],
 * staged through `ws` (ws_bytes >= pf_resample_workspace_bytes).  `arrays` and
 * `row_bytes` are host arrays.  N <= 8192 (SCH_ERR_ARG beyond). */
int pf_resample(int N, const double* wbar, uint64_t seed, uint64_t stage_ctr, int32_t* idx,
                int n_arrays, void* const* arrays, const size_t* row_bytes, void* ws,
                size_t ws_bytes, void* stream);

/* Allocation-free variant of pf_resample (the paper has no counterpart; it
 * exists for the way some programs are built, not for the method).
 *
 * Some callers cannot call cudaMalloc, or pass in device scratch, at the point
 * where they resample: a host application that fixes its device memory
 * budget at start-up and forbids later allocations, a plugin running inside a
 * framework that owns every device allocation through its own allocator, or a
 * latency-critical loop that cannot afford cudaMalloc's possible implicit
 * device synchronisation.  This entry point computes the same offspring
 * indices as pf_resample and gathers the arrays in place, but stages each
 * array in a scratch buffer that the library itself holds: a file-scope
 * __device__ array of PF_RESAMPLE_STATIC_BYTES (16 MiB), which every GPU that
 * loads the library keeps until the process exits.  It calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *
 * Limits and rules:
 *  - each array must satisfy N * row_bytes[a] <= PF_RESAMPLE_STATIC_BYTES,
 *    otherwise the call returns SCH_ERR_WORKSPACE before launching anything;
 *    other arguments as for pf_resample (N <= 8192, 16-byte rows);
 *  - the first call on a device (with that device current) looks up the
 *    scratch's device address with cudaGetSymbolAddress and caches it; make
 *    that first call before any stream capture;
 *  - every call on a device shares the one scratch buffer, which keeps the
 *    last call's contents (nothing in it needs to start at zero: each array is
 *    fully written before it is read back).  Calls whose execution overlaps on
 *    the GPU (on different streams, or from several host threads) race on the
 *    scratch and must be serialised by the caller;
 *  - the cached address belongs to the device's current context: after
 *    cudaDeviceReset on a device, do not call pf_resample_static on that device
 *    again in the same process (the address would be stale).
 */
#define PF_RESAMPLE_STATIC_BYTES (16u * 1024u * 1024u)
int pf_resample_static(int N, const double* wbar, uint64_t seed, uint64_t stage_ctr, int32_t* idx,
                       int n_arrays, void* const* arrays, const size_t* row_bytes, void* stream);

/* Out-of-place row gather: dst row i = src row idx[i]; rows of row_bytes
 * bytes (a multiple of 4; src and dst aligned to the largest of 16, 8, 4 that
 * divides row_bytes). */
int pf_gather_rows(int N, const int32_t* idx, const void* src, void* dst, size_t row_bytes,
                   void* stream);

/* Offspring indices of a device-gated stage: as pf_resample without arrays when
 * *gate != 0 (gate: device pointer to the stage's out[4] of pf_temper_dev); the
 * identity idx[i] = i when the stage is inactive, so row gathers stay valid. */
int pf_resample_gated(int N, const double* wbar, uint64_t seed, uint64_t stage_ctr, const double* gate,
                      int32_t* idx, void* stream);

/* PCN jittering at temperature theta (Sec. 3.1.2): n_iter Metropolis moves of
 * each particle's window noise.  Iteration j proposes
 *   dW' = rho dW + sqrt(1 - rho^2) sqrt(dt) z,  z keyed (seed, SCH_TAG_PCN, ctr + j),
 * re-runs the whole window from m_start with dW' (and lambda), and accepts iff
 *   log U < w0 - w1,  w = theta (NLL - logG),  U keyed (seed, SCH_TAG_PCN_ACCEPT, ctr + j).
 * In/out: dW, nll, logG, m_end, u_end (the current state; updated on accept).
 * accepts int32 [N] (out, accepted moves); iters, status optional as above. */
int pf_jitter(sch_ctx* ctx, int N, int nsteps, int n_iter, double theta, double rho,
              uint64_t seed, uint64_t ctr, const void* m_start, void* dW, const void* lambda,
              const void* y, double* nll, double* logG, void* m_end, void* u_end,
              int32_t* accepts, int32_t* iters, int32_t* status, void* stream);

/* Optional jitter workspace, caller-owned device memory of at least
 * sch_jitter_workspace_bytes(ctx, N, nsteps) bytes (16-byte aligned; the size is 0 where
 * the layout does not use it: only SCH_LAYOUT_GROUP / GROUP16 does).  Once set, every
 * pf_jitter, pf_jitter_dev and pf_gated_stages call on the context with at most N
 * particles and nsteps steps and rho >= 0.99 starts the Picard iterations of each
 * proposal after the first from the converged per-step states of the call's previous
 * proposal (when that one finished cleanly: its m, kept in the workspace, and
 * u = H^-1 M m), instead of from each step's start state.
 * The fixed point and the stop test are unchanged, so results move only within the
 * Picard tolerance; successive proposals at rho near one need about 40% fewer
 * iterations.  The workspace serves one jitter call at a time: calls on several streams
 * that share a context must not overlap.  ws NULL (or bytes 0) clears it; a workspace
 * too small for a call is ignored by that call.  sch_set_jitter_workspace returns
 * SCH_ERR_ARG for a misaligned ws. */
size_t sch_jitter_workspace_bytes(const sch_ctx* ctx, int N, int nsteps);
int sch_set_jitter_workspace(sch_ctx* ctx, void* ws, size_t bytes);

/* pf_jitter for a device-gated stage: theta = tstate[2] and nothing is done when
 * tstate[4] == 0 (tstate: device pointer to the stage's out[5] of pf_temper_dev). */
int pf_jitter_dev(sch_ctx* ctx, int N, int nsteps, int n_iter, const double* tstate, double rho,
                  uint64_t seed, uint64_t ctr, const void* m_start, void* dW, const void* lambda,
                  const void* y, double* nll, double* logG, void* m_end, void* u_end,
                  int32_t* accepts, int32_t* iters, int32_t* status, void* stream);

/* MALA jitter of the window noise: the gradient-informed jitter that Sec. 5 lists as
 * future work, on the target of the PCN jitter (Sec. 3.1.2),
 *   U(dW) = theta (NLL - log G) + |dW|^2 / (2 dt) = theta (J + sum lambda dW) + |dW|^2 / (2 dt),
 * J the window cost of sch_adjoint_window, grad U = theta (dJ/ddW + lambda) + dW / dt,
 * preconditioner C = dt (the prior covariance of dW).  One iteration j:
 *   pf_mala_propose  dW' = dW - (h/2) dt grad U(dW) + sqrt(h dt) z, z ~ N(0, 1) keyed
 *                    (seed, SCH_TAG_MALA) at counter (k / 4, step, particle0 + p, ctr);
 *   sch_adjoint_window at dW', giving J' and gJ' = dJ'/ddW';
 *   pf_mala_accept   accepts iff log u < U(dW) - U(dW') + log q(dW | dW') - log q(dW' | dW)
 *                    and U(dW') is finite, log q(b | a) = -|b - a + (h/2) dt grad U(a)|^2
 *                    / (2 h dt), u keyed (seed, SCH_TAG_MALA_ACCEPT) at counter
 *                    (0, 0, particle0 + p, ctr); on acceptance dW, J and gJ take the
 *                    proposal's values and accepts[p] (may be NULL) grows by one.
 * dW, dW_prop, lambda (NULL: no drift), gJ, gJ_prop: real [N][nsteps][K], device;
 * J, J_prop: double [N], device.  h > 0, theta in [0, 1], else SCH_ERR_ARG; N = 0 is a
 * no-op.  Both enqueue one kernel on the stream and allocate nothing. */
int pf_mala_propose(sch_ctx* ctx, int N, int nsteps, double theta, double h, uint64_t seed, uint64_t ctr,
                    int particle0, const void* dW, const void* lambda, const void* gJ, void* dW_prop,
                    void* stream);
int pf_mala_accept(sch_ctx* ctx, int N, int nsteps, double theta, double h, uint64_t seed, uint64_t ctr,
                   int particle0, void* dW, const void* dW_prop, const void* lambda, double* J,
                   const double* J_prop, void* gJ, const void* gJ_prop, int32_t* accepts, void* stream);

/* n_stages device-gated stages of an assimilation cycle (Sec. 3.1.2) enqueued in one
 * call, with no host round trip: for stage k, pf_temper_dev (temperature from
 * theta0 for k = 0, else from stage k-1), pf_resample_gated with counter
 * cycle * 1024 + first_stage + k, out-of-place row gathers of every state array
 * from bufs_a to bufs_b, then pf_jitter_dev (jitter counter stage counter x
 * n_jitter; n_jitter = 0 jitters nothing, which with a tiny ess_min is the bootstrap
 * filter).  A stage reached at temperature one does nothing but copy the rows.
 * bufs_a[PF_STAGE_ARRAYS], bufs_b[PF_STAGE_ARRAYS]: device pointers in the order
 * PF_M_START, PF_M_END, PF_U_END, PF_DW, PF_NLL, PF_LOGG, PF_LAMBDA (the last may be
 * NULL in both); every stage gathers a -> b and swaps the roles, so after n_stages
 * stages the state is in bufs_a if n_stages is even, else in bufs_b.
 *   touts   double [n_stages][5]: each stage's pf_temper_dev result
 *   iters   int32 [n_stages][N] or NULL; accepts, status as pf_jitter
 *   events  NULL or 2 n_stages cudaEvent_t recorded around each jitter launch
 * Argument errors are caught before the first launch. */
enum { PF_M_START = 0, PF_M_END, PF_U_END, PF_DW, PF_NLL, PF_LOGG, PF_LAMBDA, PF_STAGE_ARRAYS };
int pf_gated_stages(sch_ctx* ctx, int N, int nsteps, int n_stages, int first_stage, double ess_min,
                    int mode, double rho, int n_jitter, uint64_t seed, uint64_t cycle, const void* y,
                    void* const* bufs_a, void* const* bufs_b, const double* theta0, double* wbar,
                    int32_t* idx, double* touts, int32_t* accepts, int32_t* iters, int32_t* status,
                    void* const* events, void* stream);

/* Synthetic observations of a truth velocity: y_j = u(x_j) + sigma z_j with
 * z_j keyed (seed, SCH_TAG_OBS, (j / 4, 0, 0, ctr)).  u real [n], y real [M]. */
int sch_synth_obs(sch_ctx* ctx, const void* u, uint64_t seed, uint64_t ctr, void* y, void* stream);

/* Ensemble diagnostics against a truth velocity (Sec. 4.1.1): out[0] = EMRE,
 * out[1] = RB, out[2] = RES, out[3] = RMSE of the ensemble mean over the nodes
 * (out[4..7] are scratch).  u real [N][n], u_truth real [n], ws double [n]
 * (caller-owned scratch for the ensemble mean), out double [8].  N >= 2. */
int pf_diagnostics(sch_ctx* ctx, int N, const void* u, const void* u_truth, double* ws, double* out,
                   void* stream);

/* ---------------------------------------------------------------------------
 * Nudging (Sec. 3.1.3): drifts lambda that lower the window cost
 *   J(lambda) = NLL(u_end) + 1/2 sum_{s,k} lambda_{s,k}^2 dt,
 * with gradients from a hand-written reverse-mode adjoint of the converged
 * implicit-midpoint steps (the paper computes them with an automated adjoint).
 * The adjoint and the optimiser run in the context's default Picard solver
 * (SCH_SOLVER_LI for SCH_F64, SCH_SOLVER_EA for SCH_F32); a context created
 * with the other solver gets SCH_ERR_UNSUPPORTED.
 * ------------------------------------------------------------------------- */

/* Workspace for sch_adjoint_window: per particle, the states at every ckpt-th
 * step plus 2 (ckpt + 1) segment states of n reals. */
size_t sch_adjoint_workspace_bytes(const sch_ctx* ctx, int N, int nsteps, int ckpt);

/* J, dJ/dlambda, dJ/d dW and dJ/dm_start of the window cost for every particle:
 * a forward pass storing the state every ckpt steps, then per segment a
 * forward recomputation and the adjoint steps in reverse order.  With
 * ckpt >= nsteps the window is one segment: the forward pass keeps every state
 * and the reverse sweep recomputes nothing (the same results).  The adjoint
 * of a step solves J1^T psi = g by the transposed Picard fixed point to
 * params.tol (Eq. fde1 differentiated at its solution).
 *   m_start real [N][n]; dW, lambda real [N][nsteps][K] (lambda may be NULL);
 *   y real [M]; J double [N] out; g_lambda real [N][nsteps][K] out;
 *   g_dW real [N][nsteps][K] out (optional); g_m0 real [N][n] out (optional);
 *   iters int32 [N] optional (Picard + adjoint iterations); status optional.
 *   ws: device workspace of ws_bytes >= sch_adjoint_workspace_bytes. */
int sch_adjoint_window(sch_ctx* ctx, int N, int nsteps, int ckpt, const void* m_start, const void* dW,
                       const void* lambda, const void* y, double* J, void* g_lambda, void* g_dW, void* g_m0,
                       int32_t* iters, int32_t* status, void* ws, size_t ws_bytes, void* stream);

enum { PF_NUDGE_SEQUENTIAL = 0, PF_NUDGE_OPEN_LOOP = 1 };

/* Workspace for pf_nudge: the adjoint's plus one start state per particle. */
size_t pf_nudge_workspace_bytes(const sch_ctx* ctx, int N, int nsteps, int ckpt);

/* Per-particle nudging by L-BFGS (two-loop recursion, memory 6, Armijo
 * backtracking) on J with the adjoint gradient, stopping when
 * max |dJ/dlambda| <= gtol or after max_iter iterations (per stage).
 *   mode PF_NUDGE_SEQUENTIAL: the adapted schedule of Sec. 3.1.3 -- for
 *     n = 0..nsteps-1 optimise lambda^n with later increments and drifts zero,
 *     then reveal dW^n = sqrt(dt) z, z keyed (seed, SCH_TAG_NUDGE,
 *     (k / 4, n, particle, ctr)), and advance the start state one step;
 *   mode PF_NUDGE_OPEN_LOOP: optimise all drifts at once with every increment
 *     zero (lambda in: the starting guess), then reveal every increment with
 *     the same keys.
 * Out: lambda, dW real [N][nsteps][K]; J double [N] (cost at the last
 * optimisation); iters int32 [N] (L-BFGS iterations, optional); status. */
int pf_nudge(sch_ctx* ctx, int N, int nsteps, int mode, int max_iter, double gtol, int ckpt, uint64_t seed,
             uint64_t ctr, const void* m_start, const void* y, void* lambda, void* dW, double* J, int32_t* iters,
             int32_t* status, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Learned drift proposal (not in the paper): a 1D convolutional network that
 * maps a particle's window-start velocity and the innovation of the window's
 * observations to nudging drifts lambda [Ns][K], trained on drifts produced by
 * pf_nudge.  Any drift keeps the particle weights consistent through the
 * Girsanov factor (Eq. girsanov DG approx), so the network only changes how
 * close the proposal lands to the observations; the optimiser stays as the
 * fallback and as the standard the network is measured against.
 *   x0 = (u_start, (y - u_start(x_obs)) / sigma at the observation nodes)   [2][n]
 *   4 x (circular convolution, kernel 5, stride 2, C channels, ReLU)    -> [C][n/16]
 *   F[c][2(j-1)], F[c][2j-1] = (1/P) sum_q h[c][q] sin, cos(2 pi j q / P), P = n/16
 *   lambda = Wh F + bh
 * Parameters are one FP32 vector (per layer w[C][Cin][5], b[C]; then Wh[K Ns][C K],
 * bh[K Ns]); activations and gradients are FP32 in memory.  The contractions
 * (every convolution, the mode projection and the head, forward and backward)
 * run in the shape's precision:
 *   NN_FP32  FP32 operands, FP32 accumulation (CUDA cores; the check path);
 *   NN_BF16  operands rounded to BF16, FP32 accumulation (tensor cores,
 *            mma.sync m16n8k16); Adam keeps FP32 master weights.
 * ------------------------------------------------------------------------- */
enum { NN_FP32 = 0, NN_BF16 = 1 };
typedef struct {
    int32_t n;       /* nodes (multiple of 16 and of M) */
    int32_t K;       /* drift modes (even) */
    int32_t Ns;      /* steps per window */
    int32_t C;       /* channels */
    int32_t M;       /* observation points */
    float sigma;     /* observation noise, scales the innovation */
    int32_t precision;  /* NN_FP32 or NN_BF16 (anything else: an invalid shape) */
} nn_shape;

/* Number of FP32 parameters (0 for an invalid shape or precision). */
size_t nn_param_count(const nn_shape* shape);
/* Workspace bytes for a batch of B samples (activations and gradients). */
size_t nn_workspace_bytes(const nn_shape* shape, int B);
/* lambda_out float [B][Ns][K] for u_start float [B][n] and observations y float
 * [B][M] with row stride y_stride floats (0: one y shared by the batch). */
int nn_forward(const nn_shape* shape, int B, const float* params, const float* u_start, const float* y,
               int y_stride, float* lambda_out, void* ws, size_t ws_bytes, void* stream);
/* Loss L = 1/(2B) sum (lambda - target)^2 (double, device scalar) and its
 * gradient with respect to every parameter (float [nn_param_count]). */
int nn_backward(const nn_shape* shape, int B, const float* params, const float* u_start, const float* y,
                int y_stride, const float* target, float* grads, double* loss, void* ws, size_t ws_bytes,
                void* stream);
/* One Adam step (Kingma and Ba) at step number t >= 1 over count parameters:
 * m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
 * p <- p - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
int nn_adam_step(size_t count, float* params, const float* grads, float* m, float* v, int t, float lr, float b1,
                 float b2, float eps, void* stream);

/* Prior ensemble about a truth velocity (a reading of Eq. init_solve): for
 * particle p, W_p is a DG0 field with cell values sqrt(h) z (z keyed
 * (seed, SCH_TAG_INIT, (b, 0, p, 0))), S = (M + K)^{-1} M-type P1 smoothing
 * applied three times, u = u_truth + scale (a_p S^3 W_p + b_p) with a_p, b_p
 * the next two normals; writes m and u (real [N][n]).  u_truth real [n]. */
int sch_prior_sample(sch_ctx* ctx, int N, const void* u_truth, uint64_t seed, double scale,
                     void* m, void* u, void* stream);

/* The initial ensemble of Exp 1 (Sec. 4.1, Eq. init_solve): for member p, W_p is a DG0
 * field with cell values sqrt(h) z (z keyed (seed, SCH_TAG_INIT, (b, 0, particle0 + p, 0))),
 * U^{0,1} solves (U, v) + (U', v') = (|W_p|, v), U^{0,j+1} the same with right-hand side
 * (U^{0,j}, v), and u = a_p^2 U^{0,3} + b_p^2 with a_p, b_p the next two normals.  The
 * truth is a member drawn under another seed.  Writes m and u (real [N][n]). */
int sch_prior_exp1(sch_ctx* ctx, int N, uint64_t seed, int particle0, void* m, void* u, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SCH_H_ */
