// Instantiations of the warp-group window and jitter kernels for float fields:
// W warps per particle, each lane holding 2 P = 4 sub-chunks of cs nodes
// (n = 64 P cs W): (cs, W) = (4, 2) for n = 1024, (8, 2) and (4, 4) for n = 2048,
// (8, 4) and (4, 8) for n = 4096.
#include "sch_group.cuh"

namespace sch {

namespace {

constexpr int GP = 2;   // float-pair streams per lane

template <int CS, int W>
size_t smem_of(int Ns, int K, int bufs) {
    return gsmem_base<CS, GP, W>() + (size_t)bufs * Ns * K * sizeof(float);
}

template <typename Kern>
void prep(Kern k, size_t sm) {
    if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <int CS, int W, int PD>
int window_pd(const ModelArgs<float>& A, const WArgs& Wa, const GArgs& G, const WindowIO<float>& io, int N,
              cudaStream_t st) {
    const size_t sm = smem_of<CS, W>(io.Ns, A.K, 1);
    prep(gwindow_kernel<CS, GP, W, PD>, sm);
    gwindow_kernel<CS, GP, W, PD><<<N, 32 * W, sm, st>>>(A, Wa, G, io);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

template <int CS, int W, int PD>
int jitter_pd(const ModelArgs<float>& A, const WArgs& Wa, const GArgs& G, const JitterIO<float>& io, int N,
              cudaStream_t st) {
    const size_t sm = smem_of<CS, W>(io.Ns, A.K, 3);
    prep(gjitter_kernel<CS, GP, W, PD>, sm);
    gjitter_kernel<CS, GP, W, PD><<<N, 32 * W, sm, st>>>(A, Wa, G, io);
    return cudaGetLastError() == cudaSuccess ? SCH_OK : SCH_ERR_CUDA;
}

// the kernels specialised to the Picard table's lane-level system (diagonal or not)
template <int CS, int W>
int window(const ModelArgs<float>& A, const WArgs& Wa, const GArgs& G, const WindowIO<float>& io, int N,
           cudaStream_t st) {
    return G.pic.ldiag ? window_pd<CS, W, 1>(A, Wa, G, io, N, st) : window_pd<CS, W, 0>(A, Wa, G, io, N, st);
}

template <int CS, int W>
int jitter(const ModelArgs<float>& A, const WArgs& Wa, const GArgs& G, const JitterIO<float>& io, int N,
           cudaStream_t st) {
    return G.pic.ldiag ? jitter_pd<CS, W, 1>(A, Wa, G, io, N, st) : jitter_pd<CS, W, 0>(A, Wa, G, io, N, st);
}

}  // namespace

int launch_gwindow(int cs, int W, const ModelArgs<float>& A, const WArgs& Wa, const GArgs& G,
                   const WindowIO<float>& io, int N, cudaStream_t st) {
    if (A.n != 64 * GP * cs * W) return SCH_ERR_UNSUPPORTED;
    if (cs == 4 && W == 2) return window<4, 2>(A, Wa, G, io, N, st);
    if (cs == 8 && W == 2) return window<8, 2>(A, Wa, G, io, N, st);
    if (cs == 4 && W == 4) return window<4, 4>(A, Wa, G, io, N, st);
    if (cs == 8 && W == 4) return window<8, 4>(A, Wa, G, io, N, st);
    if (cs == 4 && W == 8) return window<4, 8>(A, Wa, G, io, N, st);
    return SCH_ERR_UNSUPPORTED;
}

int launch_gjitter(int cs, int W, const ModelArgs<float>& A, const WArgs& Wa, const GArgs& G,
                   const JitterIO<float>& io, int N, cudaStream_t st) {
    if (A.n != 64 * GP * cs * W) return SCH_ERR_UNSUPPORTED;
    if (cs == 4 && W == 2) return jitter<4, 2>(A, Wa, G, io, N, st);
    if (cs == 8 && W == 2) return jitter<8, 2>(A, Wa, G, io, N, st);
    if (cs == 4 && W == 4) return jitter<4, 4>(A, Wa, G, io, N, st);
    if (cs == 8 && W == 4) return jitter<8, 4>(A, Wa, G, io, N, st);
    if (cs == 4 && W == 8) return jitter<4, 8>(A, Wa, G, io, N, st);
    return SCH_ERR_UNSUPPORTED;
}

size_t gwindow_smem(int cs, int W, int Ns, int K) {
    return (sizeof(GShared<GW_MAX>) + 15) / 16 * 16 + (size_t)3 * W * GP * cs * 32 * sizeof(float2) +
           (size_t)Ns * K * sizeof(float);
}

size_t gjitter_smem(int cs, int W, int Ns, int K) {
    return (sizeof(GShared<GW_MAX>) + 15) / 16 * 16 + (size_t)3 * W * GP * cs * 32 * sizeof(float2) +
           (size_t)3 * Ns * K * sizeof(float);
}

}  // namespace sch
