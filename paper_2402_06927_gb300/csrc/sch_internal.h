// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/sch.h"
#include "sch_device.cuh"

namespace sch {

// Streaming multiprocessors of the current device, queried once per device (grid sizes of
// the grid-stride kernels are multiples of it).  1 if the query fails.
inline int device_sms() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (cache[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
}

// A constant symmetric circulant tridiagonal matrix (off-diagonal a, diagonal b)
// in chunk-partitioned form: the forward/backward sweep coefficients of a
// chunk of C <= 8 rows and the coefficients of its reduced "first" and "last"
// rows, identical in every chunk.  Computed on the host in double precision.
template <typename R>
struct CTab {
    R rden[8], gam[8], alpp[8], gamp[8];
    R a, iBF, pa, pc, ae, ge;
};

// The reduced cyclic system of a constant matrix: one unknown E_t per chunk,
// rows A E_{t-1} + B E_t + C E_{t+1} = D_t with the same A, B, C everywhere.
// Warp 0 solves it with lanes owning RR = TP/32 consecutive rows: a lane-level
// partition sweep (coefficients q, ga, al, alp, gap), then a cyclic PCR over
// the 32 lanes (level multipliers k1, k2 and the closing 2x2 weights f1, f2).
template <typename R>
struct RTab {
    R A, B, Cc;
    R q[16], ga[16], alp[16], gap[16];
    R qa, qc, iBF, aeL, geL;
    R k1[4], k2[4], f1, f2;
};

// Linear functionals used by the explicit-advection step to build the
// Helmholtz interface rows of a chunk from the interface values of the
// preceding constant solve: hpd = sum_i apd_i dp_i + cpF F + cpE E + cpEp E_{t-1}
// + cpFn F_{t+1}, and the same for hde with ade, cd*.
template <typename R>
struct HBasis {
    R apd[8], ade[8];
    R cpF, cpE, cpEp, cpFn, cdF, cdE, cdEp, cdFn;
};

// Precomputed scalars of the discretised model, passed by value to kernels
// (so that every thread reads them from the constant parameter bank).
template <typename R>
struct ModelArgs {
    int n, K, K2, M, stride, max_iter, solver;
    R h, dt;
    R c0, b0;      // left operator M + mu dt/2 K: off-diagonal, diagonal
    R c0p, b0p;    // right operator M - mu dt/2 K: off-diagonal, diagonal
    R dt8;         // dt / 8
    R h6;          // h / 6
    R tol;
    R hel_a, hel_b;  // Helmholtz H = M + alpha^2 K: off-diagonal, diagonal
    R sigma_inv;
    double dt_d;
    R amp4[SCH_MAX_K / 2];  // a_j / 4
    CTab<R> hel;            // M + alpha^2 K
    CTab<R> mass;           // M
    CTab<R> smooth;         // M + K (the (I - d_xx) smoothing of the prior)
    CTab<R> pic;            // M + mu dt/2 K (explicit-advection Picard matrix)
    R rot_c[SCH_MAX_K / 2], rot_s[SCH_MAX_K / 2];   // cos(j 2 pi / n), sin(j 2 pi / n), j = 1..K/2
    R rot_d[SCH_MAX_K / 2];  // 2 cos(j 2 pi / n) - 2 = -4 sin^2(j pi / n): the node-to-node recurrence
    RTab<R> rhel, rmass, rsmooth, rpic;
    HBasis<R> hb;
    CTab<R> matern;         // M + kappa^-2 K (Matern noise)
    RTab<R> rmatern;
    R mz;                   // Matern cell weight scale eta sqrt(h) / 8
    int mk;                 // Matern solves per step
};

// Sub-chunk coefficients of a constant symmetric circulant tridiagonal matrix
// (off-diagonal a) for the warp-per-particle kernels, whose lanes hold two
// sub-chunks of CS <= WCS_MAX nodes as float pairs.  The coefficients are
// scalars: each multiplies both halves of a pair through two scalar FMAs that
// read it straight from the parameter bank.
constexpr int WCS_MAX = 16;

struct WTab {
    float rden[WCS_MAX];     // 1 / pivot of row i (i >= 1)
    float nar[WCS_MAX];      // -a / pivot of row i
    float ngam[WCS_MAX];     // -gam_i: back-sweep coefficient
    float nalpp[WCS_MAX];    // -alpp_i: weight of the sub-chunk's first value
    float ngamp[WCS_MAX];    // -gamp_i: weight of the sub-chunk's last value
    float na, iBF;           // -a, 1 / pivot of the reduced first row
    float pa, pc, ae, ge;    // reduced-row coupling coefficients
    // 1 when the 64-row reduced system A E_{t-1} + B E_t + C E_{t+1} = D_t is
    // diagonal to 2^-30 (|A|, |C| <= 2^-30 |B|): then E_t = D_t / B to well
    // below float rounding and the kernels skip the cross-lane PCR
    int diag;
    float iB;                // 1 / B
};

// Mode-noise synthesis about each lane's centre (wnoise in sch_warp.cuh): a lane's
// 2H nodes lie at the offsets -d_{H-1} .. -d_0, d_0 .. d_{H-1} from its centre, d_m =
// (m + 1/2) 2 pi / n, with H = P CS <= 2 WNQ_MAX.  With tau = d / d_{H-1} in (0, 1]
// and s = tau^2, harmonic j's cos(j d) and sin(j d) / tau are smooth functions of s on
// [0, 1]; where j d_{H-1} is small for every j <= K/2 the host fits each (GArgs npc) with a
// polynomial of WNP coefficients in s (Chebyshev interpolation), and a lane then
// forms the WNP sums over j once and evaluates them at its H offsets.
constexpr int WNQ_MAX = 8;
constexpr int WNP = 4;

struct WArgs {
    WTab pic, hel;           // M + mu dt/2 K ;  (6/h)(M + alpha^2 K)
    RTab<float> rpic, rhel;  // their 64-row reduced systems (two rows per lane)
    WTab mat;                // Matern noise: (6/h)(M + kappa^-2 K)
    RTab<float> rmat;
    float mzw;               // Matern cell weight scale (6/h) eta sqrt(h) / 8
    // for harmonic j = 1..K/2 and q < H/2: nco[j-1][q] = (cos j d_{H-1-q}, cos j d_q) and
    // nsi[j-1][q] = (sin j d_{H-1-q}, sin j d_q)
    float2 nco[SCH_MAX_K / 2][WNQ_MAX], nsi[SCH_MAX_K / 2][WNQ_MAX];
};

// Cross-warp reduced solve of a constant table for the warp-group kernels
// (sch_group.cuh), W <= GW_MAX warps per particle.  The lane-last unknowns of the
// 32 W lanes satisfy LA EL_{g-1} + LB EL_g + LC EL_{g+1} = LD_g (cyclic).  Each warp
// solves its 32 rows as a cyclic system of their own, y = T32^{-1} LD; p2_0, p2_31
// are entries 0 and 31 of T32^{-1} e_31, the response to the part m = cq pd_0 +
// geL qd_0 of lane 31's row that comes from the next warp's lane 0.  The warp's
// boundary values b_{w-1}, b_w (lane 31 of the previous and of this warp) and
// a_w, a_{w+1} (lane 0 of this and of the next warp) are sums over k < W of the
// tabulated weights times y_0 (entry k) and y_31 (entry W + k) of warp w + k, both
// corrected by that warp's m.  Computed on the host in double precision.
constexpr int GW_MAX = 8;
struct GTab {
    float LA, LC, iLC;
    float p2_0, p2_31;
    float cq, geL;
    float bprev[2 * GW_MAX], bself[2 * GW_MAX], aself[2 * GW_MAX], anext[2 * GW_MAX];
    // 1 when the lane-level system is diagonal to 2^-26 (|LA|, |LC| <= 2^-26 |LB|): then
    // EL_g = LD_g / LB to well below float rounding, and the solve needs neither the PCR
    // nor the 2W system, only the neighbouring warps' boundary rows
    int ldiag;
    float iLB;
};

struct GArgs {
    GTab pic, hel;          // the cross-warp solves of M + mu dt/2 K and (6/h)(M + alpha^2 K)
    // the polynomial form of the lane-centred noise (gnoise in sch_group.cuh):
    // npc[j-1][k] = (c_k, s_k) with cos(j d) ~ sum_k c_k s^k and sin(j d) ~ tau sum_k s_k s^k,
    // k < WNP.  npoly = 1 when those fits hold to 2^-30 at every offset and cost the lane
    // fewer operations than the tables of WArgs; otherwise the tables are used
    float2 npc[SCH_MAX_K / 2][WNP];
    int npoly;
};

template <typename R>
struct WindowIO {
    int Ns;
    const R* m_in;
    R* m_out;
    R* u_out;
    const R* dW;
    const R* lam;
    const R* y;
    double* nll;
    double* logG;
    int32_t* iters;
    int32_t* status;
};

template <typename R>
struct JitterIO {
    int Ns, n_iter, particle0;
    double theta;
    const double* tstate;   // device-gated stage: theta = tstate[2], active = tstate[4] != 0 (or null)
    R rho, sq1mr2;
    uint64_t seed, ctr;
    const R* m_start;
    R* dW;
    const R* lam;
    const R* y;
    double* nll;
    double* logG;
    R* m_end;
    R* u_end;
    int32_t* accepts;
    int32_t* iters;
    int32_t* status;
    // optional (warp-group kernels): per particle and step the converged m of the call's
    // previous proposal, [N][Ns][n] in the kernel's register order; null: every proposal
    // starts its Picard iterations from the step's start state
    R* guess = nullptr;
};

template <typename R>
struct AdjointIO {
    int Ns, ck;
    const R* m_start;
    const R* dW;
    const R* lam;
    const R* y;
    double* J;
    R* g_lam;     // [N][Ns][K]
    R* g_dW;      // [N][Ns][K] or null
    R* g_m0;      // [N][n] or null
    R* ws;        // per-particle scratch: ncp checkpoints + 2 (ck + 1) states of n values
    size_t ws_per;
    int32_t* iters;
    int32_t* status;
};

template <typename R>
struct NudgeIO {
    int Ns, ck, mode, max_iter, particle0;
    double gtol;
    uint64_t seed, ctr;
    const R* m_start;
    const R* y;
    R* lam;       // [N][Ns][K] in: start (open loop), out: drift
    R* dW;        // [N][Ns][K] out: the revealed increments
    double* J;    // [N] out: final cost
    R* ws;
    size_t ws_per;
    int32_t* iters;   // [N] out: L-BFGS iterations
    int32_t* status;
};

template <typename R, int C, int S>
int launch_adjoint(const ModelArgs<R>& A, const AdjointIO<R>& io, int N, cudaStream_t st);
template <typename R, int C, int S>
int launch_nudge(const ModelArgs<R>& A, const NudgeIO<R>& io, int N, cudaStream_t st);
// the adjoint window and nudging with the Matern noise (sch_adjoint_matern.cu): each
// precision's default solver
template <typename R, int C>
int launch_adjoint_matern(const ModelArgs<R>& A, const AdjointIO<R>& io, int N, cudaStream_t st);
template <typename R, int C>
int launch_nudge_matern(const ModelArgs<R>& A, const NudgeIO<R>& io, int N, cudaStream_t st);

// L-BFGS memory of the nudging optimiser
constexpr int LBFGS_M = 6;

// With the Matern noise the nudging optimiser keeps the window's drifts, increments and
// L-BFGS vectors in the particle's workspace after the adjoint's region of ws_adj
// elements of rsize bytes: 5 + 2 LBFGS_M vectors of NK doubles and 2 LBFGS_M doubles
// (8-byte aligned), then dW and lambda (NK elements each).  Elements per particle, even
// so that every particle's region stays 8-byte aligned.
inline size_t nudge_matern_ws_elems(size_t ws_adj, size_t NK, size_t rsize) {
    const size_t dbl = (ws_adj * rsize + 7) / 8 + (5 + 2 * (size_t)LBFGS_M) * NK + 2 * LBFGS_M;
    const size_t elems = (dbl * 8 + 2 * NK * rsize + rsize - 1) / rsize;
    return (elems + 1) / 2 * 2;
}
template <typename R, int C>
size_t adjoint_smem(int tp, int Ns, int K);
template <typename R, int C>
size_t nudge_smem(int tp, int Ns, int K);

template <typename R, int C, int S>
int launch_window(const ModelArgs<R>& A, const WindowIO<R>& io, int N, cudaStream_t st);
template <typename R, int C, int S>
int launch_jitter(const ModelArgs<R>& A, const JitterIO<R>& io, int N, cudaStream_t st);
template <typename R, int C>
int launch_helm(const ModelArgs<R>& A, const R* in, R* out, int mode, int N, cudaStream_t st);
template <typename R, int C>
int launch_prior(const ModelArgs<R>& A, const R* u_truth, uint64_t seed, R scale, R* m, R* u, int N,
                 cudaStream_t st, int mode, int particle0);
template <typename R, int C>
size_t jitter_smem(int tp, int Ns, int K);
// window and jitter kernels with the Matern noise, warp layout (sch_matern_warp.cu)
int launch_wwindow_matern(int cs, const ModelArgs<float>& A, const WArgs& W, const WindowIO<float>& io, int N,
                          cudaStream_t st);
int launch_wjitter_matern(int cs, const ModelArgs<float>& A, const WArgs& W, const JitterIO<float>& io, int N,
                          cudaStream_t st);
// window and jitter kernels with the Matern noise (sch_matern_{f32,f64}.cu): the
// default solver of each precision only
template <typename R, int C>
int launch_window_matern(const ModelArgs<R>& A, const WindowIO<R>& io, int N, cudaStream_t st);
template <typename R, int C>
int launch_jitter_matern(const ModelArgs<R>& A, const JitterIO<R>& io, int N, cudaStream_t st);
template <typename R>
int launch_draw(int N, int Ns, int K, R sqdt, uint64_t seed, uint64_t tag, uint64_t ctr, int particle0, int gen32,
                R* dW, cudaStream_t st);
template <typename R>
int launch_loglik(const ModelArgs<R>& A, int N, const R* u, const R* y, const R* dW, const R* lam, int Ns,
                  double* nll, double* logG, cudaStream_t st);
template <typename R, int C>
size_t window_smem(int tp, int Ns, int K);
template <typename R>
int launch_synth_obs(const ModelArgs<R>& A, const R* u, uint64_t seed, uint64_t ctr, R* y, cudaStream_t st);
template <typename R>
int launch_diag(const ModelArgs<R>& A, int N, const R* u, const R* u_truth, double* ws, double* out,
                cudaStream_t st);

// warp-per-particle kernels for float fields, n = 64 P cs with P = warp_streams(n)
// float-pair streams of two sub-chunks each (sch_window_warp.cu)
int warp_streams(int n);
int launch_wwindow(int cs, const ModelArgs<float>& A, const WArgs& W, const WindowIO<float>& io, int N,
                   cudaStream_t st);
int launch_wjitter(int cs, const ModelArgs<float>& A, const WArgs& W, const JitterIO<float>& io, int N,
                   cudaStream_t st);
size_t wwindow_smem(int cs, int Ns, int K);
size_t wjitter_smem(int cs, int Ns, int K);

// warp-group kernels for float fields (sch_window_group.cu): W warps per particle,
// each holding n / W nodes as 2 P sub-chunks of cs nodes per lane (n = 64 P cs W)
int launch_gwindow(int cs, int W, const ModelArgs<float>& A, const WArgs& Wa, const GArgs& G,
                   const WindowIO<float>& io, int N, cudaStream_t st);
int launch_gjitter(int cs, int W, const ModelArgs<float>& A, const WArgs& Wa, const GArgs& G,
                   const JitterIO<float>& io, int N, cudaStream_t st);
size_t gwindow_smem(int cs, int W, int Ns, int K);
size_t gjitter_smem(int cs, int W, int Ns, int K);

// MALA jitter (pf_mala.cu)
template <typename R>
int launch_mala_propose(int N, int Ns, int K, double theta, double h, double dt, const R* dW, const R* lam,
                        const R* gJ, uint64_t seed, uint64_t ctr, int particle0, R* dWp, cudaStream_t st);
template <typename R>
int launch_mala_accept(int N, int NK, double theta, double h, double dt, uint64_t seed, uint64_t ctr, int particle0,
                       R* dW, const R* dWp, const R* lam, double* J, const double* Jp, R* gJ, const R* gJp,
                       int32_t* accepts, cudaStream_t st);

// filter kernels (pf_filter.cu)
int launch_temper(int N, const double* nll, const double* logG, double theta, const double* theta_dev,
                  double ess_min, int halving, double* wbar,
                  double* out, cudaStream_t st);
int launch_resample_idx(int N, const double* wbar, uint64_t seed, uint64_t stage_ctr, const double* gate,
                        int32_t* idx, cudaStream_t st);
int launch_gather(int N, const int32_t* idx, const void* src, void* dst, size_t row_bytes, cudaStream_t st);
int launch_copy(const void* src, void* dst, size_t bytes, cudaStream_t st);
constexpr int GATHER_MAX_ARRAYS = 8;
int launch_gather_multi(int N, const int32_t* idx, int n, const void* const* src, void* const* dst,
                        const size_t* row_bytes, cudaStream_t st);

}  // namespace sch
