// Learned drift proposal on sm_103a: forward, backward and Adam of the small
// 1D convolutional network that maps a particle's window-start velocity and
// the innovation of the window's observations to nudging drifts lambda
// [Ns][K] (used in place of, or as the starting point of, the optimiser of
// Sec. 3.1.3; any drift keeps the weights consistent through Girsanov).
//
// Network (FP32 parameters and activations, FP32 accumulation):
//   x0[b] = (u_start, (y - u_start(x_obs)) / sigma scattered at the obs nodes)   2 x n
//   four circular convolutions, kernel 5, stride 2, padding 2, C channels, ReLU  -> C x n/16
//   Fourier-mode projection F[c][k] = (1/P) sum_q h[c][q] {sin,cos}(2 pi j q / P)
//   linear head lambda = Wh F + bh
// Every contraction runs through one tiled GEMM kernel with gather functors
// (implicit im2col for the convolutions), so no im2col buffer is formed: a SIMT
// FP32 kernel (NN_FP32, the check path), or a tensor-core kernel that rounds both
// operands to BF16 as it stages them in shared memory and accumulates in FP32
// with mma.sync m16n8k16 (NN_BF16).  Parameters, activations and gradients stay
// FP32 in memory in both (the FP32 master weights of Adam).
#include <cuda_bf16.h>

#include "sch_internal.h"

namespace sch {

struct NNDims {
    int n, K, Ns, C, M, prec;
    float sigma;
    int L[5];     // positions at layers 0..4: n, n/2, n/4, n/8, n/16
    int cin[4];   // input channels of conv l
    size_t off_w[4], off_b[4], off_wh, off_bh, nparam;
    size_t act_off[5], off_F, off_lam, act_total;   // per-sample activation offsets (floats)
};

static NNDims make_dims(const nn_shape* s) {
    NNDims d{};
    d.n = s->n; d.K = s->K; d.Ns = s->Ns; d.C = s->C; d.M = s->M; d.sigma = s->sigma; d.prec = s->precision;
    for (int l = 0; l <= 4; ++l) d.L[l] = s->n >> l;
    size_t o = 0;
    for (int l = 0; l < 4; ++l) {
        d.cin[l] = (l == 0) ? 2 : s->C;
        d.off_w[l] = o; o += (size_t)s->C * d.cin[l] * 5;
        d.off_b[l] = o; o += (size_t)s->C;
    }
    d.off_wh = o; o += (size_t)s->K * s->Ns * s->C * s->K;
    d.off_bh = o; o += (size_t)s->K * s->Ns;
    d.nparam = o;
    size_t a = 0;
    d.act_off[0] = a; a += 2 * (size_t)d.L[0];
    for (int l = 1; l <= 4; ++l) { d.act_off[l] = a; a += (size_t)s->C * d.L[l]; }
    d.off_F = a; a += (size_t)s->C * s->K;
    d.off_lam = a; a += (size_t)s->K * s->Ns;
    d.act_total = a;
    return d;
}

// --------------------------------------------------------------------------
// tiled SGEMM: C[m][n] (+)= sum_k A(m, k) B(k, n) over a batch index z.
// 64 x 64 tiles, k-chunks of 16, 256 threads, 4 x 4 outputs per thread.
// --------------------------------------------------------------------------
constexpr int TM = 64, TN = 64, TK = 16;

template <typename LA, typename LB, typename EP>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int Kd, int kchunk, LA la, LB lb, EP ep) {
    __shared__ float As[TK][TM + 4];
    __shared__ float Bs[TK][TN + 4];
    const int z = blockIdx.z;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int kbeg = (int)(blockIdx.z % (unsigned)max(1, (Kd + kchunk - 1) / kchunk)) * kchunk;
    const int zb = z / max(1, (Kd + kchunk - 1) / kchunk);
    const int kend = min(Kd, kbeg + kchunk);
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = kbeg; k0 < kend; k0 += TK) {
        for (int e = threadIdx.x; e < TK * TM; e += 256) {
            const int kk = e / TM, mm = e % TM;
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < kend) ? la(zb, gm, gk) : 0.f;
        }
        for (int e = threadIdx.x; e < TK * TN; e += 256) {
            const int kk = e / TN, nn = e % TN;
            const int gn = n0 + nn, gk = k0 + kk;
            Bs[kk][nn] = (gn < N && gk < kend) ? lb(zb, gk, gn) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
            if (gm < M && gn < N) ep(zb, gm, gn, acc[i][j]);
        }
}

// --------------------------------------------------------------------------
// BF16 tensor-core GEMM with the same gather functors: C[m][n] (+)= sum_k A(m, k)
// B(k, n), both operands rounded to BF16 (round to nearest) as they are staged in
// shared memory, products accumulated in FP32 by mma.sync.m16n8k16 (row.col).
// 64 x 64 tiles, k-chunks of 32, 128 threads: warp w computes the 32 x 32 quarter
// (w / 2, w % 2) as 2 x 4 fragments of 16 x 8.  Shared rows are padded by 8
// elements so that the 32-bit fragment loads of a warp fall in distinct banks.
// --------------------------------------------------------------------------
constexpr int HTM = 64, HTN = 64, HTK = 32, HPAD = 8;

// How a gather functor's operand lies in memory.  By default consecutive k are adjacent
// for an A operand and consecutive n for a B operand; a functor that declares
// `static constexpr bool transposed = true` has them the other way round (consecutive m
// adjacent as A, consecutive k as B).  The BF16 tile loaders walk the adjacent index
// fastest, so that a warp's loads are coalesced.
template <typename F, typename = void>
struct is_transposed {
    static constexpr bool value = false;
};
template <typename F>
struct is_transposed<F, decltype((void)F::transposed)> {
    static constexpr bool value = F::transposed;
};

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <typename LA, typename LB, typename EP>
__global__ void __launch_bounds__(128) hgemm_kernel(int M, int N, int Kd, int kchunk, LA la, LB lb, EP ep) {
    __shared__ __align__(16) __nv_bfloat16 As[HTM][HTK + HPAD];   // [m][k]
    __shared__ __align__(16) __nv_bfloat16 Bs[HTN][HTK + HPAD];   // [n][k]
    const int m0 = blockIdx.y * HTM, n0 = blockIdx.x * HTN;
    const int nkc = max(1, (Kd + kchunk - 1) / kchunk);
    const int kbeg = (int)(blockIdx.z % (unsigned)nkc) * kchunk;
    const int zb = blockIdx.z / nkc;
    const int kend = min(Kd, kbeg + kchunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gq = lane >> 2, tq = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    for (int k0 = kbeg; k0 < kend; k0 += HTK) {
        for (int e = threadIdx.x; e < HTK * HTM; e += 128) {
            const int mm = is_transposed<LA>::value ? e % HTM : e / HTK;
            const int kk = is_transposed<LA>::value ? e / HTM : e % HTK;
            const int gm = m0 + mm, gk = k0 + kk;
            As[mm][kk] = __float2bfloat16_rn((gm < M && gk < kend) ? la(zb, gm, gk) : 0.f);
        }
        for (int e = threadIdx.x; e < HTK * HTN; e += 128) {
            const int kk = is_transposed<LB>::value ? e % HTK : e / HTN;
            const int nn = is_transposed<LB>::value ? e / HTK : e % HTN;
            const int gn = n0 + nn, gk = k0 + kk;
            Bs[nn][kk] = __float2bfloat16_rn((gn < N && gk < kend) ? lb(zb, gk, gn) : 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < HTK; ks += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + 16 * i + gq;
                a[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tq]);
                a[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tq]);
                a[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tq + 8]);
                a[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tq + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + 8 * j + gq;
                b[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + 2 * tq]);
                b[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + 2 * tq + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16_16816(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    // fragment (i, j): rows wm + 16 i + gq (+ 8), columns wn + 8 j + 2 tq (+ 1)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int gm = m0 + wm + 16 * i + gq + ((e & 2) ? 8 : 0);
                const int gn = n0 + wn + 8 * j + 2 * tq + (e & 1);
                if (gm < M && gn < N) ep(zb, gm, gn, acc[i][j][e]);
            }
}

// k-splits for a reduction with few output tiles (weight gradients: the sum runs over
// batch x positions): about 8 CTAs per SM, chunks of at least 256 k-values
static int splitk_for(int M, int N, int Kd) {
    const int tiles = ((M + TM - 1) / TM) * ((N + TN - 1) / TN);
    return max(1, min(Kd / 256, 8 * device_sms() / tiles));
}

// k-chunks that sgemm launches for a split of splitk
static int splitk_chunks(int Kd, int splitk) {
    const int kchunk = (Kd + splitk - 1) / splitk;
    return (Kd + kchunk - 1) / kchunk;
}

// the GEMM in the network's precision: the FP32 SIMT kernel or the BF16 tensor-core kernel
// (same tile sizes, so the split-K chunks and the partial buffers are the same)
template <typename LA, typename LB, typename EP>
static void sgemm(int prec, int batch, int M, int N, int Kd, int splitk, LA la, LB lb, EP ep, cudaStream_t st) {
    const int kchunk = (Kd + splitk - 1) / splitk;
    const int nk = splitk_chunks(Kd, splitk);
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, batch * nk);
    if (prec == NN_BF16)
        hgemm_kernel<<<grid, 128, 0, st>>>(M, N, Kd, kchunk, la, lb, ep);
    else
        sgemm_kernel<<<grid, 256, 0, st>>>(M, N, Kd, kchunk, la, lb, ep);
}

// --------------------------------------------------------------------------
// functors
// --------------------------------------------------------------------------
struct ConvW {            // A(co, kk) = w[co][kk], kk = ci * 5 + j
    const float* w; int KK;
    __device__ float operator()(int, int m, int k) const { return w[(size_t)m * KK + k]; }
};
struct ConvX {            // B(kk, q) = x[b][ci][(2q + j - 2) mod L]
    const float* x; size_t bstride; int L;
    __device__ float operator()(int b, int k, int q) const {
        const int ci = k / 5, j = k % 5;
        int i = 2 * q + j - 2;
        i = (i + L) % L;
        return x[(size_t)b * bstride + (size_t)ci * L + i];
    }
};
struct StoreAct {         // out[b][co][q] = relu(acc + bias[co])
    float* out; size_t bstride; int Lo; const float* bias;
    __device__ void operator()(int b, int m, int n, float v) const {
        v += bias[m];
        out[(size_t)b * bstride + (size_t)m * Lo + n] = v > 0.f ? v : 0.f;
    }
};
// backward data: dx[b][ci][i] = sum_{co, j} w[co][ci][j] g[b][co][q], 2q + j - 2 = i (mod L)
struct WT {               // A(ci, kk') = w[co][ci][j], kk' = co * 5 + j
    const float* w; int Ci;
    __device__ float operator()(int, int m, int k) const {
        const int co = k / 5, j = k % 5;
        return w[((size_t)co * Ci + m) * 5 + j];
    }
};
struct GatherG {          // B(kk', i) = g[b][co][q] if 2q + j - 2 = i (mod L), else 0
    const float* g; size_t bstride; int L, Lo;
    __device__ float operator()(int b, int k, int i) const {
        const int co = k / 5, j = k % 5;
        int t = i - j + 2;
        t = ((t % L) + L) % L;
        if (t & 1) return 0.f;
        const int q = t >> 1;
        return g[(size_t)b * bstride + (size_t)co * Lo + q];
    }
};
struct StoreMasked {      // dx masked by the ReLU of the layer that produced x (x > 0)
    float* out; const float* x; size_t bstride; int L; int mask;
    __device__ void operator()(int b, int m, int n, float v) const {
        const size_t o = (size_t)b * bstride + (size_t)m * L + n;
        out[o] = (mask && !(x[o] > 0.f)) ? 0.f : v;
    }
};
// backward weights: dw[co][kk] = sum_{b, q} g[b][co][q] X(b, kk, q), batch folded into k
struct GRowsBQ {          // A(co, (b, q)) = g[b][co][q]
    const float* g; size_t bstride; int Lo;
    __device__ float operator()(int, int m, int k) const {
        const int b = k / Lo, q = k % Lo;
        return g[(size_t)b * bstride + (size_t)m * Lo + q];
    }
};
struct ConvXT {           // B((b, q), kk) = x[b][ci][(2q + j - 2) mod L]
    const float* x; size_t bstride; int L, Lo;
    __device__ float operator()(int, int k, int n) const {
        const int b = k / Lo, q = k % Lo;
        const int ci = n / 5, j = n % 5;
        int i = 2 * q + j - 2;
        i = (i + L) % L;
        return x[(size_t)b * bstride + (size_t)ci * L + i];
    }
};
// split-K partial of a batch-1 product: k-chunk blockIdx.z writes a slice of its own and
// the slices are summed afterwards in a fixed order, so the gradients are reproducible
struct StorePartial {
    float* out; int ld; size_t slice;
    __device__ void operator()(int, int m, int n, float v) const {
        out[(size_t)blockIdx.z * slice + (size_t)m * ld + n] = v;
    }
};
// generic row-major accessors
struct RowMajor {         // A(m, k) = p[z * bs + m * ld + k]
    const float* p; size_t bs; int ld;
    __device__ float operator()(int z, int m, int k) const { return p[(size_t)z * bs + (size_t)m * ld + k]; }
};
struct RowMajorT {        // A(m, k) = p[z * bs + k * ld + m]
    static constexpr bool transposed = true;
    const float* p; size_t bs; int ld;
    __device__ float operator()(int z, int m, int k) const { return p[(size_t)z * bs + (size_t)k * ld + m]; }
};
struct ModeS {            // S(q, k) = {sin, cos}(2 pi j q / P) / P
    int P;
    __device__ float operator()(int, int q, int k) const {
        const int j = k / 2 + 1;
        float s, c;
        sincospif(2.0f * (float)((j * q) % P) / (float)P, &s, &c);
        return ((k & 1) ? c : s) / (float)P;
    }
};
struct ModeST {           // S^T(k, q)
    int P;
    __device__ float operator()(int z, int k, int q) const { return ModeS{P}(z, q, k); }
};
struct Store {            // out[z * bs + m * ld + n] = v (+ bias[n] if bias)
    float* out; size_t bs; int ld; const float* bias;
    __device__ void operator()(int z, int m, int n, float v) const {
        out[(size_t)z * bs + (size_t)m * ld + n] = v + (bias ? bias[n] : 0.f);
    }
};
struct StoreBF16 {        // out[z * bs + m * ld + n] = v rounded to BF16
    __nv_bfloat16* out; size_t bs; int ld;
    __device__ void operator()(int z, int m, int n, float v) const {
        out[(size_t)z * bs + (size_t)m * ld + n] = __float2bfloat16_rn(v);
    }
};

// --------------------------------------------------------------------------
// element-wise kernels
// --------------------------------------------------------------------------
__global__ void features_kernel(int B, int n, int M, float sigma, const float* u, const float* y, int ystride,
                                float* x0, size_t bstride) {
    const size_t tot = (size_t)B * n;
    const int stride = n / M;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / n), i = (int)(e % n);
        const float ub = u[(size_t)b * n + i];
        float inn = 0.f;
        if (i % stride == 0) {
            const float yj = y[(size_t)b * ystride + i / stride];
            if (yj == yj) inn = (yj - ub) / sigma;   // NaN: not observed
        }
        x0[(size_t)b * bstride + i] = ub;
        x0[(size_t)b * bstride + n + i] = inn;
    }
}

// glam = (lam - target) / B, loss partials in double
__global__ void loss_kernel(int B, int O, const float* lam, size_t lstride, const float* target, float* glam,
                            double* loss) {
    const size_t tot = (size_t)B * O;
    double acc = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / O), o = (int)(e % O);
        const float d = lam[(size_t)b * lstride + o] - target[e];
        glam[e] = d / (float)B;
        acc += 0.5 * (double)d * (double)d / B;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// out[e] = sum of the nk slices part[s][e], in slice order
__global__ void sum_slices_kernel(size_t count, int nk, const float* __restrict__ part, float* __restrict__ out) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int s = 0; s < nk; ++s) acc += part[(size_t)s * count + e];
        out[e] = acc;
    }
}

// db[co] = sum over samples b and positions q of g[b][co][q].  Per-thread partial
// sums in FP32 (two interleaved accumulators; GB300's FP64 rate would make this
// the slowest step of the backward pass), the final reduction in FP64.  With
// L >= 32 positions the threads stride over q inside each sample; otherwise over
// the flattened (b, q).
__global__ void bias_grad_kernel(int B, int Co, int L, const float* g, size_t bstride, float* db) {
    const int co = blockIdx.x;
    float a0 = 0.f, a1 = 0.f;
    if (L >= 32) {
        const float* row = g + (size_t)co * L;
        for (int b = 0; b < B; b += 2) {
            for (int q = threadIdx.x; q < L; q += blockDim.x) {
                a0 += row[(size_t)b * bstride + q];
                if (b + 1 < B) a1 += row[(size_t)(b + 1) * bstride + q];
            }
        }
    } else {
        for (int e = threadIdx.x; e < B * L; e += blockDim.x)
            a0 += g[(size_t)(e / L) * bstride + (size_t)co * L + e % L];
    }
    double acc = warp_sum((double)a0 + (double)a1);
    __shared__ double sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        db[co] = (float)s;
    }
}

__global__ void zero_kernel(float* p, size_t nel, double* d) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nel; e += (size_t)gridDim.x * blockDim.x)
        p[e] = 0.f;
    if (d && blockIdx.x == 0 && threadIdx.x == 0) *d = 0.0;
}

__global__ void adam_kernel(size_t nel, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nel; e += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float mi = b1 * m[e] + (1.f - b1) * gi;
        const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
        m[e] = mi;
        v[e] = vi;
        p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void copy_rows_kernel(int B, int O, const float* src, size_t sstride, float* dst) {
    const size_t tot = (size_t)B * O;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x)
        dst[e] = src[(e / O) * sstride + e % O];
}

static int grid_elems(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > (size_t)device_sms() * 16) b = (size_t)device_sms() * 16;
    return (int)(b < 1 ? 1 : b);
}

// forward pass into the activation workspace (per-sample stride act_total)
static void nn_forward_impl(const NNDims& d, int B, const float* params, const float* u, const float* y, int ystride,
                            float* act, cudaStream_t st) {
    const size_t bs = d.act_total;
    features_kernel<<<grid_elems((size_t)B * d.n), 256, 0, st>>>(B, d.n, d.M, d.sigma, u, y, ystride,
                                                                 act + d.act_off[0], bs);
    for (int l = 0; l < 4; ++l) {
        const int Ci = d.cin[l], Lin = d.L[l], Lo = d.L[l + 1];
        sgemm(d.prec, B, d.C, Lo, Ci * 5, 1, ConvW{params + d.off_w[l], Ci * 5}, ConvX{act + d.act_off[l], bs, Lin},
              StoreAct{act + d.act_off[l + 1], bs, Lo, params + d.off_b[l]}, st);
    }
    const int P = d.L[4];
    // F[b][c][k] = sum_q h4[b][c][q] S[q][k]
    sgemm(d.prec, B, d.C, d.K, P, 1, RowMajor{act + d.act_off[4], bs, P}, ModeS{P},
          Store{act + d.off_F, bs, d.K, nullptr}, st);
    // lambda[b][o] = sum_f F[b][f] Wh[o][f] + bh[o]   (one GEMM over the batch: rows b)
    const int O = d.K * d.Ns, FF = d.C * d.K;
    sgemm(d.prec, 1, B, O, FF, 1, RowMajor{act + d.off_F, 0, (int)bs}, RowMajorT{params + d.off_wh, 0, FF},
          Store{act + d.off_lam, 0, (int)bs, params + d.off_bh}, st);
}

// --------------------------------------------------------------------------
// BF16 inference path with channels-last activations (nn_forward with NN_BF16 and
// C = 64): the activations of layers 1..4 are stored once as BF16, [b][position][c],
// so that a convolution's operand pairs (channel ci, ci + 1 at one input position)
// are adjacent and a tile's im2col is the input slab itself.  Layer 0 (two input
// channels, 10 taps) runs on the CUDA cores from the features; layers 1..3 on the
// tensor cores (conv_tc_kernel); the mode projection and the head through
// hgemm_kernel.  Values equal the BF16 path of nn_forward_impl (the same BF16
// rounding of every operand), accumulation orders aside.
// --------------------------------------------------------------------------
constexpr int CL_C = 64;                 // channels of the channels-last path
constexpr int CL_K = 5 * CL_C;           // reduction length of layers 1..3 (k = j C + ci)
constexpr int CL_WROW = CL_K + 8;        // shared weight row (bf16): 656 bytes, 16 mod 128
constexpr int CL_XROW = CL_C + 8;        // shared slab row (bf16): 144 bytes, 16 mod 128
constexpr int CL_TQ = 64;                // output positions per CTA
constexpr int CL_XPOS = 2 * CL_TQ + 3;   // input positions a tile reads
constexpr int CL_XEVEN = CL_TQ + 2;      // of which at even offsets from the slab's start

__host__ __device__ constexpr size_t cl_smem() {
    return ((size_t)CL_C * CL_WROW + 2 * (size_t)CL_XPOS * CL_XROW + (size_t)CL_TQ * (CL_C + 8)) *
           sizeof(__nv_bfloat16);
}

// the weights of conv layers 1..3 as BF16 [l][co][j C + ci] (k ordered tap-major)
__global__ void pack_conv_weights_kernel(const float* params, size_t off1, size_t off2, size_t off3,
                                         __nv_bfloat16* wb) {
    const int tot = 3 * CL_C * CL_K;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
        const int l = e / (CL_C * CL_K), r = e % (CL_C * CL_K);
        const int co = r / CL_K, k = r % CL_K, j = k / CL_C, ci = k % CL_C;
        const size_t off = (l == 0) ? off1 : (l == 1) ? off2 : off3;
        wb[e] = __float2bfloat16_rn(params[off + ((size_t)co * CL_C + ci) * 5 + j]);
    }
}

// Layer 0 on the tensor cores: out[b][q][co] = relu(b0[co] + sum_k X0[q][k] W0[co][k]) with
// k = 2 j + ci (ten taps x channels, padded to 16 with zero weights), X0[q][k] the feature
// of channel ci at input position 2q + j - 2.  A CTA takes 64 output positions of one
// sample: its threads form the features of the positions 2 q0 - 2 .. 2 q0 + 133 as BF16
// (u, innovation) pairs in shared memory, so that row q of X0 is 16 consecutive values
// starting at pair 2q; warp w then computes the 32 x 32 quarter (w / 2, w % 2) of the
// 64 x 64 output with one k-step of mma.sync m16n8k16.  Epilogue: bias, ReLU, BF16, the
// tile staged in shared memory and stored as 8 KB of contiguous rows.
constexpr int CL_OROW = CL_C + 8;         // staged output row (bf16): 144 bytes, rows in distinct banks

// a CTA's 64 x 64 output tile, staged in shared memory [64][CL_OROW], to the 64 consecutive
// channels-last rows from dst (8 KB contiguous): 16-byte stores, 128 threads
__device__ __forceinline__ void cl_store_tile(const __nv_bfloat16* Os, __nv_bfloat16* dst) {
    for (int e = threadIdx.x; e < 64 * (CL_C / 8); e += 128) {
        const int r = e / (CL_C / 8), c8 = e % (CL_C / 8);
        *reinterpret_cast<uint4*>(dst + (size_t)r * CL_C + 8 * c8) =
            *reinterpret_cast<const uint4*>(Os + r * CL_OROW + 8 * c8);
    }
}

constexpr int C0_TQ = 64;                 // output positions per CTA
constexpr int C0_XPOS = 2 * C0_TQ + 8;    // feature positions staged (rows read 8 positions)
constexpr int C0_WROW = 16 + 8;           // shared weight row (bf16)

__global__ void __launch_bounds__(128) conv0_cl_kernel(int n, int M, float sigma, const float* u, const float* y,
                                                       int ystride, const float* w0, const float* b0,
                                                       __nv_bfloat16* out, size_t out_bs) {
    __shared__ __align__(16) __nv_bfloat16 Xs[2 * C0_XPOS];      // (u, innovation) per position
    __shared__ __align__(16) __nv_bfloat16 Ws[CL_C * C0_WROW];   // [co][2 j + ci], zero for k >= 10
    __shared__ __align__(16) __nv_bfloat16 Os[C0_TQ * CL_OROW];  // the output tile
    const int b = blockIdx.y, q0 = blockIdx.x * C0_TQ, stride = n / M;
    for (int e = threadIdx.x; e < CL_C * 16; e += 128) {
        const int co = e / 16, k = e % 16, j = k >> 1, ci = k & 1;
        Ws[co * C0_WROW + k] = __float2bfloat16_rn(k < 10 ? w0[(co * 2 + ci) * 5 + j] : 0.f);
    }
    for (int r = threadIdx.x; r < C0_XPOS; r += 128) {
        const int i = (2 * q0 - 2 + r + n) % n;
        const float ub = u[(size_t)b * n + i];
        float inn = 0.f;
        if (i % stride == 0) {
            const float yj = y[(size_t)b * ystride + i / stride];
            if (yj == yj) inn = (yj - ub) / sigma;   // NaN: not observed
        }
        *reinterpret_cast<__nv_bfloat162*>(Xs + 2 * r) = __floats2bfloat162_rn(ub, inn);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wq = (warp >> 1) * 32, wc = (warp & 1) * 32;
    const int gq = lane >> 2, tq = lane & 3;
    uint32_t a[2][4], bf[4][2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int q = wq + 16 * i + gq;   // row q starts at pair 2q; k pair (2t, 2t+1) is pair 2q + t
        a[i][0] = *reinterpret_cast<const uint32_t*>(Xs + 2 * (2 * q + tq));
        a[i][1] = *reinterpret_cast<const uint32_t*>(Xs + 2 * (2 * (q + 8) + tq));
        a[i][2] = *reinterpret_cast<const uint32_t*>(Xs + 2 * (2 * q + tq + 4));
        a[i][3] = *reinterpret_cast<const uint32_t*>(Xs + 2 * (2 * (q + 8) + tq + 4));
    }
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
        const int c = wc + 8 * jj + gq;
        bf[jj][0] = *reinterpret_cast<const uint32_t*>(Ws + c * C0_WROW + 2 * tq);
        bf[jj][1] = *reinterpret_cast<const uint32_t*>(Ws + c * C0_WROW + 2 * tq + 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            mma_bf16_16816(acc, a[i], bf[jj]);
            const int co = wc + 8 * jj + 2 * tq;
            const float bb0 = b0[co], bb1 = b0[co + 1];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = wq + 16 * i + gq + 8 * h;
                const float v0 = acc[2 * h] + bb0, v1 = acc[2 * h + 1] + bb1;
                *reinterpret_cast<__nv_bfloat162*>(Os + q * CL_OROW + co) =
                    __floats2bfloat162_rn(v0 > 0.f ? v0 : 0.f, v1 > 0.f ? v1 : 0.f);
            }
        }
    __syncthreads();
    cl_store_tile(Os, out + (size_t)b * out_bs + (size_t)q0 * CL_C);
}

// 16-byte asynchronous copy global -> shared (cp.async, completion tracked by groups)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// four 8 x 8 BF16 matrices from shared memory (lane l gives the address of row l % 8 of
// matrix l / 8); register i receives matrix i in the mma fragment layout
__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void* smem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(sa));
}

// The input slab of tile (b, q0): positions 2 q0 - 2 + r, r = 0 .. 130 (mod Lin), 64 channels
// each, stored de-interleaved: offset r at row r / 2 when r is even, CL_XEVEN + r / 2 when odd,
// so that the rows 2q + j of the output positions q of a fragment are consecutive.
__device__ __forceinline__ int cl_slab_row(int r) { return (r & 1) ? CL_XEVEN + (r >> 1) : (r >> 1); }

__device__ __forceinline__ void cl_issue_slab(__nv_bfloat16* Xs, const __nv_bfloat16* in, size_t in_bs, int Lin,
                                              int b, int q0) {
    const __nv_bfloat16* inb = in + (size_t)b * in_bs;
    for (int e = threadIdx.x; e < CL_XPOS * (CL_C / 8); e += 128) {
        const int r = e / (CL_C / 8), c8 = e % (CL_C / 8);
        const int pos = (2 * q0 - 2 + r + Lin) % Lin;
        cp_async16(Xs + cl_slab_row(r) * CL_XROW + 8 * c8, inb + (size_t)pos * CL_C + 8 * c8);
    }
}

// Layers 1..3 on the tensor cores: D[q][co] = sum_k X[q][k] W[co][k], k = j C + ci and
// X[q][k] = in[b][(2q + j - 2) mod Lin][ci].  A persistent CTA stages the layer's weights
// [64][320] in shared memory once, then takes tiles of 64 output positions of one sample
// (all 64 output channels) in turn: the input slab of positions 2 q0 - 2 .. 2 q0 + 128
// (131 rows of 64 channels) is copied with cp.async into one of two buffers while the
// previous tile is computed.  Warp w computes the 32 x 32 quarter (w / 2, w % 2) of a
// tile with mma.sync m16n8k16, its A fragments loaded by ldmatrix straight from the slab
// (rows 2q + j, 16 channels), its B fragments from the weights.  Epilogue: bias, ReLU,
// BF16, the tile staged in shared memory and stored as 8 KB of contiguous rows.
__global__ void __launch_bounds__(128) conv_tc_kernel(int B, int Lin, const __nv_bfloat16* __restrict__ in,
                                                      size_t in_bs, const __nv_bfloat16* __restrict__ wb,
                                                      const float* __restrict__ bias, __nv_bfloat16* __restrict__ out,
                                                      size_t out_bs) {
    extern __shared__ __align__(16) unsigned char cl_raw[];
    __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(cl_raw);   // [64][CL_WROW]
    __nv_bfloat16* Xbuf = Ws + CL_C * CL_WROW;                       // [2][CL_XPOS][CL_XROW]
    __nv_bfloat16* Os = Xbuf + 2 * CL_XPOS * CL_XROW;                // [CL_TQ][CL_OROW] output tile
    const int tpb = (Lin / 2) / CL_TQ, ntiles = B * tpb;
    for (int e = threadIdx.x; e < CL_C * (CL_K / 8); e += 128) {
        const int r = e / (CL_K / 8), c8 = e % (CL_K / 8);
        *reinterpret_cast<uint4*>(Ws + r * CL_WROW + 8 * c8) = *reinterpret_cast<const uint4*>(wb + r * CL_K + 8 * c8);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the rows and column halves this lane addresses in ldmatrix: A (slab) matrices are
    // (rows 0-7, 8-15) x (columns 0-7, 8-15), B (weight) matrices (k 0-7, 8-15) x (n 0-7, 8-15)
    const int arow = (lane & 7) + 8 * ((lane >> 3) & 1), acol = 8 * (lane >> 4);
    const int brow = (lane & 7) + 8 * (lane >> 4), bcol = 8 * ((lane >> 3) & 1);
    const int wq = (warp >> 1) * 32, wc = (warp & 1) * 32;
    const int gq = lane >> 2, tq = lane & 3;
    int t = blockIdx.x;
    if (t < ntiles) cl_issue_slab(Xbuf, in, in_bs, Lin, t / tpb, (t % tpb) * CL_TQ);
    cp_async_commit();
    for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
        const int tn = t + gridDim.x;
        if (tn < ntiles)
            cl_issue_slab(Xbuf + ((it + 1) & 1) * CL_XPOS * CL_XROW, in, in_bs, Lin, tn / tpb, (tn % tpb) * CL_TQ);
        cp_async_commit();
        cp_async_wait1();   // this tile's slab (the group before the one just committed)
        __syncthreads();
        const __nv_bfloat16* Xs = Xbuf + (it & 1) * CL_XPOS * CL_XROW;
        const int b = t / tpb, q0 = (t % tpb) * CL_TQ;
        float acc[2][4][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[i][jj][e] = 0.f;
#pragma unroll 1
        for (int j = 0; j < 5; ++j) {
            // slab rows of tap j: offset 2q + j is row q + j/2 (even j) or CL_XEVEN + q + (j-1)/2
            const int jrow = (j & 1) ? CL_XEVEN + (j >> 1) : (j >> 1);
#pragma unroll
            for (int kc = 0; kc < CL_C; kc += 16) {
                uint32_t a[2][4], bf[4][2];
#pragma unroll
                for (int i = 0; i < 2; ++i)
                    ldmatrix_x4(a[i], Xs + (jrow + wq + 16 * i + arow) * CL_XROW + kc + acol);
#pragma unroll
                for (int jj = 0; jj < 4; jj += 2) {
                    uint32_t r4[4];
                    ldmatrix_x4(r4, Ws + (wc + 8 * jj + brow) * CL_WROW + j * CL_C + kc + bcol);
                    bf[jj][0] = r4[0];
                    bf[jj][1] = r4[1];
                    bf[jj + 1][0] = r4[2];
                    bf[jj + 1][1] = r4[3];
                }
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) mma_bf16_16816(acc[i][jj], a[i], bf[jj]);
            }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int co = wc + 8 * jj + 2 * tq;
                const float b0 = bias[co], b1 = bias[co + 1];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int q = wq + 16 * i + gq + 8 * h;
                    const float v0 = acc[i][jj][2 * h] + b0, v1 = acc[i][jj][2 * h + 1] + b1;
                    const __nv_bfloat162 pk = __floats2bfloat162_rn(v0 > 0.f ? v0 : 0.f, v1 > 0.f ? v1 : 0.f);
                    *reinterpret_cast<__nv_bfloat162*>(Os + q * CL_OROW + co) = pk;
                }
            }
        __syncthreads();
        cl_store_tile(Os, out + (size_t)b * out_bs + (size_t)q0 * CL_C);
        __syncthreads();   // every warp is done with this buffer and the output tile before reuse
    }
}

// BF16 weights of the head, Wh [K Ns][C K] in the parameters' layout
__global__ void pack_bf16_kernel(size_t count, const float* src, __nv_bfloat16* dst) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        dst[e] = __float2bfloat16_rn(src[e]);
}

// Dense GEMM with BF16 operands from memory and FP32 accumulation (the head of the
// channels-last path): C[m][n] = sum_k A[m][k] B[n][k] + bias[n], A [M][Kd] and B [N][Kd]
// row-major BF16, Kd a multiple of 32.  64 x 64 tiles, 128 threads (warp w: the 32 x 32
// quarter (w / 2, w % 2)), k-chunks of 32 double-buffered with cp.async, fragments by
// ldmatrix (80-byte shared rows: eight rows fall in distinct 16-byte bank groups).
constexpr int DG_T = 64, DG_BK = 32, DG_ROW = DG_BK + 8;

__global__ void __launch_bounds__(128) dense_bf16_gemm_kernel(int M, int N, int Kd,
                                                              const __nv_bfloat16* __restrict__ A,
                                                              const __nv_bfloat16* __restrict__ Bm,
                                                              const float* __restrict__ bias, float* __restrict__ C,
                                                              int ldc) {
    __shared__ __align__(16) __nv_bfloat16 As[2][DG_T][DG_ROW];
    __shared__ __align__(16) __nv_bfloat16 Bs[2][DG_T][DG_ROW];
    const int m0 = blockIdx.y * DG_T, n0 = blockIdx.x * DG_T;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gq = lane >> 2, tq = lane & 3;
    const int arow = (lane & 7) + 8 * ((lane >> 3) & 1), acol = 8 * (lane >> 4);
    const int brow = (lane & 7) + 8 * (lane >> 4), bcol = 8 * ((lane >> 3) & 1);
    auto issue = [&](int buf, int k0) {
        for (int e = threadIdx.x; e < DG_T * (DG_BK / 8); e += 128) {
            const int r = e / (DG_BK / 8), c8 = e % (DG_BK / 8);
            const int gm = min(m0 + r, M - 1), gn = min(n0 + r, N - 1);   // rows past the end: any row
            cp_async16(&As[buf][r][8 * c8], A + (size_t)gm * Kd + k0 + 8 * c8);
            cp_async16(&Bs[buf][r][8 * c8], Bm + (size_t)gn * Kd + k0 + 8 * c8);
        }
    };
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][jj][e] = 0.f;
    const int nk = Kd / DG_BK;
    issue(0, 0);
    cp_async_commit();
    for (int kt = 0; kt < nk; ++kt) {
        if (kt + 1 < nk) issue((kt + 1) & 1, (kt + 1) * DG_BK);
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const int b = kt & 1;
#pragma unroll
        for (int ks = 0; ks < DG_BK; ks += 16) {
            uint32_t a[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) ldmatrix_x4(a[i], &As[b][wm + 16 * i + arow][ks + acol]);
#pragma unroll
            for (int jj = 0; jj < 4; jj += 2) {
                uint32_t r4[4];
                ldmatrix_x4(r4, &Bs[b][wn + 8 * jj + brow][ks + bcol]);
                bf[jj][0] = r4[0];
                bf[jj][1] = r4[1];
                bf[jj + 1][0] = r4[2];
                bf[jj + 1][1] = r4[3];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) mma_bf16_16816(acc[i][jj], a[i], bf[jj]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int gm = m0 + wm + 16 * i + gq + ((e & 2) ? 8 : 0);
                const int gn = n0 + wn + 8 * jj + 2 * tq + (e & 1);
                if (gm < M && gn < N) C[(size_t)gm * ldc + gn] = acc[i][jj][e] + bias[gn];
            }
}

// A(c, q) = h[b][q][c] of a channels-last BF16 activation (the mode projection's operand)
struct CLRows {
    static constexpr bool transposed = true;
    const __nv_bfloat16* h; size_t bstride;
    __device__ float operator()(int b, int m, int k) const {
        return __bfloat162float(h[(size_t)b * bstride + (size_t)k * CL_C + m]);
    }
};

// bytes of the channels-last inference path's buffers per sample: layers 1..4 in BF16,
// the mode features F and lambda in FP32 (together below the FP32 path's act_total floats)
static size_t cl_act_elems(const NNDims& d) {
    return (size_t)CL_C * (d.L[1] + d.L[2] + d.L[3] + d.L[4]);
}

static bool cl_supported(const NNDims& d) {
    // 64 channels; every layer's output a whole number of 64-position tiles; the head's
    // reduction C K a multiple of the dense GEMM's k-chunk
    return d.prec == NN_BF16 && d.C == CL_C && d.L[4] % CL_TQ == 0 && (d.C * d.K) % DG_BK == 0;
}

static void nn_forward_cl(const NNDims& d, int B, const float* params, const float* u, const float* y, int ystride,
                          void* ws, float* lam_out, cudaStream_t st) {
    const size_t cs = cl_act_elems(d);
    __nv_bfloat16* act = reinterpret_cast<__nv_bfloat16*>(ws);
    const int P = d.L[4], FF = d.C * d.K, O = d.K * d.Ns;
    __nv_bfloat16* wb = act + (size_t)B * cs;                               // [3][64][320]
    __nv_bfloat16* whb = wb + 3 * CL_C * CL_K;                              // [O][FF]
    __nv_bfloat16* F = whb + (size_t)O * FF;                                // [B][C K]
    size_t off[5];
    off[1] = 0;
    for (int l = 1; l < 4; ++l) off[l + 1] = off[l] + (size_t)CL_C * d.L[l];
    pack_conv_weights_kernel<<<grid_elems(3 * CL_C * CL_K), 256, 0, st>>>(params, d.off_w[1], d.off_w[2], d.off_w[3],
                                                                           wb);
    conv0_cl_kernel<<<dim3(d.L[1] / C0_TQ, B), 128, 0, st>>>(d.n, d.M, d.sigma, u, y, ystride, params + d.off_w[0],
                                                            params + d.off_b[0], act + off[1], cs);
    const size_t sm = cl_smem();
    cudaFuncSetAttribute(conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    // persistent CTAs: as many as fit on the device at once (two per SM at 78 KB of shared memory)
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_tc_kernel, 128, sm);
    const int resident = max(1, nsm * max(1, per_sm));
    for (int l = 1; l < 4; ++l) {
        const int ntiles = B * (d.L[l + 1] / CL_TQ);
        conv_tc_kernel<<<min(ntiles, resident), 128, sm, st>>>(B, d.L[l], act + off[l], cs,
                                                               wb + (size_t)(l - 1) * CL_C * CL_K, params + d.off_b[l],
                                                               act + off[l + 1], cs);
    }
    // F = h4 S / P in BF16 (the head's operand), then lambda = F Wh^T + bh
    sgemm(NN_BF16, B, d.C, d.K, P, 1, CLRows{act + off[4], cs}, ModeS{P}, StoreBF16{F, (size_t)FF, d.K}, st);
    pack_bf16_kernel<<<grid_elems((size_t)O * FF), 256, 0, st>>>((size_t)O * FF, params + d.off_wh, whb);
    dim3 hg((O + DG_T - 1) / DG_T, (B + DG_T - 1) / DG_T);
    dense_bf16_gemm_kernel<<<hg, 128, 0, st>>>(B, O, FF, F, whb, params + d.off_bh, lam_out, O);
}

}  // namespace sch

using namespace sch;

extern "C" {

size_t nn_param_count(const nn_shape* s) {
    if (!s || s->n <= 0 || (s->n % 16) || s->K <= 0 || s->Ns <= 0 || s->C <= 0) return 0;
    if (s->precision != NN_FP32 && s->precision != NN_BF16) return 0;
    return make_dims(s).nparam;
}

// floats of the split-K partials of the largest weight-gradient product
static size_t partial_floats(const NNDims& d, int B) {
    const int O = d.K * d.Ns, FF = d.C * d.K;
    size_t m = (size_t)splitk_chunks(B, splitk_for(O, FF, B)) * O * FF;
    for (int l = 0; l < 4; ++l) {
        const int KK = d.cin[l] * 5, Kd = B * d.L[l + 1];
        m = max(m, (size_t)splitk_chunks(Kd, splitk_for(d.C, KK, Kd)) * d.C * KK);
    }
    return m;
}

size_t nn_workspace_bytes(const nn_shape* s, int B) {
    if (!s || B <= 0 || nn_param_count(s) == 0) return 0;
    const NNDims d = make_dims(s);
    // forward activations + two gradient buffers of one activation each + glam/gF + split-K partials
    return ((size_t)B * d.act_total * 3 + 2 * (size_t)d.C * d.K * B + (size_t)d.K * d.Ns * B +
            partial_floats(d, B)) * sizeof(float);
}

static int nn_check(const nn_shape* s, int B, const void* params, const void* u, const void* y, void* ws,
                    size_t ws_bytes) {
    if (!s || B <= 0 || !params || !u || !y || !ws) return SCH_ERR_ARG;
    if (nn_param_count(s) == 0 || s->M <= 0 || s->n % s->M || !(s->sigma > 0.f)) return SCH_ERR_ARG;
    if (ws_bytes < nn_workspace_bytes(s, B)) return SCH_ERR_WORKSPACE;
    return SCH_OK;
}

int nn_forward(const nn_shape* s, int B, const float* params, const float* u_start, const float* y, int y_stride,
               float* lam_out, void* ws, size_t ws_bytes, void* stream) {
    int rc = nn_check(s, B, params, u_start, y, ws, ws_bytes);
    if (rc != SCH_OK) return rc;
    if (!lam_out || y_stride < 0) return SCH_ERR_ARG;
    const NNDims d = make_dims(s);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cl_supported(d)) {
        nn_forward_cl(d, B, params, u_start, y, y_stride, ws, lam_out, st);
        return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
    }
    float* act = reinterpret_cast<float*>(ws);
    nn_forward_impl(d, B, params, u_start, y, y_stride, act, st);
    const int O = d.K * d.Ns;
    copy_rows_kernel<<<grid_elems((size_t)B * O), 256, 0, st>>>(B, O, act + d.off_lam, d.act_total, lam_out);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

int nn_backward(const nn_shape* s, int B, const float* params, const float* u_start, const float* y, int y_stride,
                const float* target, float* grads, double* loss, void* ws, size_t ws_bytes, void* stream) {
    int rc = nn_check(s, B, params, u_start, y, ws, ws_bytes);
    if (rc != SCH_OK) return rc;
    if (!target || !grads || !loss || y_stride < 0) return SCH_ERR_ARG;
    const NNDims d = make_dims(s);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    float* act = reinterpret_cast<float*>(ws);
    const size_t bs = d.act_total;
    float* gA = act + (size_t)B * bs;          // gradient of an activation (ping)
    float* gB = gA + (size_t)B * bs;           // (pong)
    float* gF = gB + (size_t)B * bs;           // [B][C K]
    float* glam = gF + (size_t)B * d.C * d.K;  // [B][O]
    float* part = glam + (size_t)B * d.K * d.Ns; // split-K partials [chunk][rows][cols]
    const int O = d.K * d.Ns, FF = d.C * d.K, P = d.L[4];
    nn_forward_impl(d, B, params, u_start, y, y_stride, act, st);
    zero_kernel<<<grid_elems(d.nparam), 256, 0, st>>>(grads, d.nparam, loss);
    loss_kernel<<<grid_elems((size_t)B * O), 256, 0, st>>>(B, O, act + d.off_lam, bs, target, glam, loss);
    // head: dWh[o][f] = sum_b glam[b][o] F[b][f]; dbh[o] = sum_b glam[b][o]; gF = glam Wh
    {
        const int sk = splitk_for(O, FF, B), nk = splitk_chunks(B, sk);
        sgemm(d.prec, 1, O, FF, B, sk, RowMajorT{glam, 0, O}, RowMajor{act + d.off_F, 0, (int)bs},
              StorePartial{part, FF, (size_t)O * FF}, st);
        sum_slices_kernel<<<grid_elems((size_t)O * FF), 256, 0, st>>>((size_t)O * FF, nk, part, grads + d.off_wh);
    }
    bias_grad_kernel<<<O, 256, 0, st>>>(B, O, 1, glam, (size_t)O, grads + d.off_bh);
    sgemm(d.prec, 1, B, FF, O, 1, RowMajor{glam, 0, O}, RowMajor{params + d.off_wh, 0, FF}, Store{gF, 0, FF, nullptr}, st);
    // dh4[b][c][q] = sum_k gF[b][c][k] S[q][k], masked by ReLU(h4 > 0)
    sgemm(d.prec, B, d.C, P, d.K, 1, RowMajor{gF, (size_t)FF, d.K}, ModeST{P}, StoreMasked{gA, act + d.act_off[4], bs, P, 1},
          st);
    // conv layers, last to first; gA holds dL/dz of layer l's output at offset act_off[l+1]
    float* gcur = gA;
    float* gnext = gB;
    for (int l = 3; l >= 0; --l) {
        const int Ci = d.cin[l], Lin = d.L[l], Lo = d.L[l + 1];
        const float* gz = gcur;
        // weights: dw[co][kk] = sum_{b,q} gz[b][co][q] X(b, kk, q)
        const int sk = splitk_for(d.C, Ci * 5, B * Lo), nk = splitk_chunks(B * Lo, sk);
        const size_t wcount = (size_t)d.C * Ci * 5;
        sgemm(d.prec, 1, d.C, Ci * 5, B * Lo, sk, GRowsBQ{gz, bs, Lo}, ConvXT{act + d.act_off[l], bs, Lin, Lo},
              StorePartial{part, Ci * 5, wcount}, st);
        sum_slices_kernel<<<grid_elems(wcount), 256, 0, st>>>(wcount, nk, part, grads + d.off_w[l]);
        bias_grad_kernel<<<d.C, 256, 0, st>>>(B, d.C, Lo, gz, bs, grads + d.off_b[l]);
        if (l > 0) {
            // data: dx[b][ci][i], masked by the ReLU of layer l-1's output
            sgemm(d.prec, B, Ci, Lin, d.C * 5, 1, WT{params + d.off_w[l], Ci}, GatherG{gz, bs, Lin, Lo},
                  StoreMasked{gnext, act + d.act_off[l], bs, Lin, 1}, st);
            float* t = gcur;
            gcur = gnext;
            gnext = t;
        }
    }
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

int nn_adam_step(size_t count, float* params, const float* grads, float* m, float* v, int t, float lr, float b1,
                 float b2, float eps, void* stream) {
    if (count == 0 || !params || !grads || !m || !v || t < 1 || !(lr > 0.f)) return SCH_ERR_ARG;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    adam_kernel<<<grid_elems(count), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(count, params, grads, m, v,
                                                                                         lr, b1, b2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

}  // extern "C"
