// Instantiations of the warp-per-particle Matern window and jitter kernels (float
// fields): (sub-chunk length CS, streams P) = (4, 1) for n = 256, (4, 2) for n = 512,
// (8, 2) for n = 1024.
#include "sch_warp_matern.cuh"

namespace sch {

namespace {

template <typename Kern>
void prep(Kern k, size_t sm) {
    if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <int CS, int P, int PM, int HM, int MM>
int window_rm(const ModelArgs<float>& A, const WArgs& W, const WindowIO<float>& io, int N, cudaStream_t st) {
    const size_t sm = wsmem_base<CS, P>();
    prep(wmatern_window_kernel<CS, P, PM, HM, MM>, sm);
    wmatern_window_kernel<CS, P, PM, HM, MM><<<N, 32, sm, st>>>(A, W, io);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

template <int CS, int P, int PM, int HM, int MM>
int jitter_rm(const ModelArgs<float>& A, const WArgs& W, const JitterIO<float>& io, int N, cudaStream_t st) {
    const size_t sm = wmatern_smem<CS, P>();
    prep(wmatern_jitter_kernel<CS, P, PM, HM, MM>, sm);
    wmatern_jitter_kernel<CS, P, PM, HM, MM><<<N, 32, sm, st>>>(A, W, io);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

// Kernels specialised to the reduced solves of a diagonal Picard table and coupled
// Helmholtz and Matern tables (the usual case: small mu dt / h^2, alpha and 1/kappa
// many cells long); any other combination tests the flags at run time.
bool usual_tables(const WArgs& W) { return W.pic.diag && !W.hel.diag && !W.mat.diag; }

template <int CS, int P>
int window(const ModelArgs<float>& A, const WArgs& W, const WindowIO<float>& io, int N, cudaStream_t st) {
    return usual_tables(W) ? window_rm<CS, P, RED_DIAG, RED_PCR, RED_PCR>(A, W, io, N, st)
                           : window_rm<CS, P, RED_RUNTIME, RED_RUNTIME, RED_RUNTIME>(A, W, io, N, st);
}

template <int CS, int P>
int jitter(const ModelArgs<float>& A, const WArgs& W, const JitterIO<float>& io, int N, cudaStream_t st) {
    return usual_tables(W) ? jitter_rm<CS, P, RED_DIAG, RED_PCR, RED_PCR>(A, W, io, N, st)
                           : jitter_rm<CS, P, RED_RUNTIME, RED_RUNTIME, RED_RUNTIME>(A, W, io, N, st);
}

}  // namespace

int launch_wwindow_matern(int cs, const ModelArgs<float>& A, const WArgs& W, const WindowIO<float>& io, int N,
                          cudaStream_t st) {
    switch (A.n) {
        case 256: return cs == 4 ? window<4, 1>(A, W, io, N, st) : SCH_ERR_UNSUPPORTED;
        case 512: return cs == 4 ? window<4, 2>(A, W, io, N, st) : SCH_ERR_UNSUPPORTED;
        case 1024: return cs == 8 ? window<8, 2>(A, W, io, N, st) : SCH_ERR_UNSUPPORTED;
        default: return SCH_ERR_UNSUPPORTED;
    }
}

int launch_wjitter_matern(int cs, const ModelArgs<float>& A, const WArgs& W, const JitterIO<float>& io, int N,
                          cudaStream_t st) {
    switch (A.n) {
        case 256: return cs == 4 ? jitter<4, 1>(A, W, io, N, st) : SCH_ERR_UNSUPPORTED;
        case 512: return cs == 4 ? jitter<4, 2>(A, W, io, N, st) : SCH_ERR_UNSUPPORTED;
        case 1024: return cs == 8 ? jitter<8, 2>(A, W, io, N, st) : SCH_ERR_UNSUPPORTED;
        default: return SCH_ERR_UNSUPPORTED;
    }
}

}  // namespace sch
