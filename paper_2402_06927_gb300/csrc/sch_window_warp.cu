// Instantiations of the warp-per-particle window and jitter kernels for float
// fields: (sub-chunk length CS, streams P) = (4, 1) for n = 256, (4, 2) for
// n = 512, (8, 2) for n = 1024 (n = 64 P CS).
#include "sch_warp.cuh"

namespace sch {

namespace {

template <int CS, int P>
size_t smem_of(int Ns, int K, int bufs) {
    return wsmem_base<CS, P>() + (size_t)bufs * Ns * K * sizeof(float);
}

template <typename Kern>
void prep(Kern k, size_t sm) {
    if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <int CS, int P, int PM, int HM>
int window_rm(const ModelArgs<float>& A, const WArgs& W, const WindowIO<float>& io, int N, cudaStream_t st) {
    const size_t sm = smem_of<CS, P>(io.Ns, A.K, 1);
    prep(wwindow_kernel<CS, P, PM, HM>, sm);
    wwindow_kernel<CS, P, PM, HM><<<N, 32, sm, st>>>(A, W, io);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

template <int CS, int P, int PM, int HM>
int jitter_rm(const ModelArgs<float>& A, const WArgs& W, const JitterIO<float>& io, int N, cudaStream_t st) {
    const size_t sm = smem_of<CS, P>(io.Ns, A.K, 3);
    prep(wjitter_kernel<CS, P, PM, HM>, sm);
    wjitter_kernel<CS, P, PM, HM><<<N, 32, sm, st>>>(A, W, io);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

// the kernels specialised to the two tables' reduced solves (diagonal or PCR)
template <int CS, int P>
int window(const ModelArgs<float>& A, const WArgs& W, const WindowIO<float>& io, int N, cudaStream_t st) {
    if (W.pic.diag)
        return W.hel.diag ? window_rm<CS, P, RED_DIAG, RED_DIAG>(A, W, io, N, st)
                          : window_rm<CS, P, RED_DIAG, RED_PCR>(A, W, io, N, st);
    return W.hel.diag ? window_rm<CS, P, RED_PCR, RED_DIAG>(A, W, io, N, st)
                      : window_rm<CS, P, RED_PCR, RED_PCR>(A, W, io, N, st);
}

template <int CS, int P>
int jitter(const ModelArgs<float>& A, const WArgs& W, const JitterIO<float>& io, int N, cudaStream_t st) {
    if (W.pic.diag)
        return W.hel.diag ? jitter_rm<CS, P, RED_DIAG, RED_DIAG>(A, W, io, N, st)
                          : jitter_rm<CS, P, RED_DIAG, RED_PCR>(A, W, io, N, st);
    return W.hel.diag ? jitter_rm<CS, P, RED_PCR, RED_DIAG>(A, W, io, N, st)
                      : jitter_rm<CS, P, RED_PCR, RED_PCR>(A, W, io, N, st);
}

}  // namespace

int warp_streams(int n) { return n == 256 ? 1 : 2; }

int launch_wwindow(int cs, const ModelArgs<float>& A, const WArgs& W, const WindowIO<float>& io, int N,
                   cudaStream_t st) {
    switch (A.n) {
        case 256: return cs == 4 ? window<4, 1>(A, W, io, N, st) : SCH_ERR_UNSUPPORTED;
        case 512: return cs == 4 ? window<4, 2>(A, W, io, N, st) : SCH_ERR_UNSUPPORTED;
        case 1024: return cs == 8 ? window<8, 2>(A, W, io, N, st) : SCH_ERR_UNSUPPORTED;
        default: return SCH_ERR_UNSUPPORTED;
    }
}

int launch_wjitter(int cs, const ModelArgs<float>& A, const WArgs& W, const JitterIO<float>& io, int N,
                   cudaStream_t st) {
    switch (A.n) {
        case 256: return cs == 4 ? jitter<4, 1>(A, W, io, N, st) : SCH_ERR_UNSUPPORTED;
        case 512: return cs == 4 ? jitter<4, 2>(A, W, io, N, st) : SCH_ERR_UNSUPPORTED;
        case 1024: return cs == 8 ? jitter<8, 2>(A, W, io, N, st) : SCH_ERR_UNSUPPORTED;
        default: return SCH_ERR_UNSUPPORTED;
    }
}

size_t wwindow_smem(int cs, int Ns, int K) {
    return (size_t)2 * cs * 32 * sizeof(float2) + (size_t)Ns * K * sizeof(float);
}

size_t wjitter_smem(int cs, int Ns, int K) {
    return (size_t)2 * cs * 32 * sizeof(float2) + (size_t)3 * Ns * K * sizeof(float);
}

}  // namespace sch
