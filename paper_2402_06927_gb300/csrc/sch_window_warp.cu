// Instantiations of the warp-per-particle window and jitter kernels for float
// fields with sub-chunks of CS = 4, 8, 16 nodes (n = 256, 512, 1024).
#include "sch_warp.cuh"

namespace sch {

namespace {

template <int CS>
size_t smem_of(int Ns, int K, int bufs) {
    return wsmem_base<CS>() + (size_t)bufs * Ns * K * sizeof(float);
}

template <typename Kern>
void prep(Kern k, size_t sm) {
    if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <int CS>
int window(const ModelArgs<float>& A, const WArgs& W, const WindowIO<float>& io, int N, cudaStream_t st) {
    const size_t sm = smem_of<CS>(io.Ns, A.K, 1);
    prep(wwindow_kernel<CS>, sm);
    wwindow_kernel<CS><<<N, 32, sm, st>>>(A, W, io);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

template <int CS>
int jitter(const ModelArgs<float>& A, const WArgs& W, const JitterIO<float>& io, int N, cudaStream_t st) {
    const size_t sm = smem_of<CS>(io.Ns, A.K, 3);
    prep(wjitter_kernel<CS>, sm);
    wjitter_kernel<CS><<<N, 32, sm, st>>>(A, W, io);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

}  // namespace

int launch_wwindow(int cs, const ModelArgs<float>& A, const WArgs& W, const WindowIO<float>& io, int N,
                   cudaStream_t st) {
    switch (cs) {
        case 4: return window<4>(A, W, io, N, st);
        case 8: return window<8>(A, W, io, N, st);
        case 16: return window<16>(A, W, io, N, st);
        default: return SCH_ERR_UNSUPPORTED;
    }
}

int launch_wjitter(int cs, const ModelArgs<float>& A, const WArgs& W, const JitterIO<float>& io, int N,
                   cudaStream_t st) {
    switch (cs) {
        case 4: return jitter<4>(A, W, io, N, st);
        case 8: return jitter<8>(A, W, io, N, st);
        case 16: return jitter<16>(A, W, io, N, st);
        default: return SCH_ERR_UNSUPPORTED;
    }
}

size_t wwindow_smem(int cs, int Ns, int K) {
    switch (cs) {
        case 4: return smem_of<4>(Ns, K, 1);
        case 8: return smem_of<8>(Ns, K, 1);
        case 16: return smem_of<16>(Ns, K, 1);
        default: return (size_t)-1;
    }
}

size_t wjitter_smem(int cs, int Ns, int K) {
    switch (cs) {
        case 4: return smem_of<4>(Ns, K, 3);
        case 8: return smem_of<8>(Ns, K, 3);
        case 16: return smem_of<16>(Ns, K, 3);
        default: return (size_t)-1;
    }
}

}  // namespace sch
