// Instantiations of the particle kernels for float fields, chunks of 8 nodes
// per thread and CTA sizes TP = 32 .. 512 (n = 8 TP): utilities, and the
// window and jitter kernels with the explicit-advection Picard solver.
#include "sch_kernels.cuh"

namespace sch {

#define SCH_TP_SWITCH(expr_tp, call)                      \
    switch (expr_tp) {                                    \
        case 32: return Launch<float, 8, 32>::call;     \
        case 64: return Launch<float, 8, 64>::call;     \
        case 128: return Launch<float, 8, 128>::call;   \
        case 256: return Launch<float, 8, 256>::call;   \
        case 512: return Launch<float, 8, 512>::call;   \
        default: return SCH_ERR_UNSUPPORTED;              \
    }

template <>
int launch_window<float, 8, SCH_SOLVER_EA>(const ModelArgs<float>& A, const WindowIO<float>& io, int N,
                                             cudaStream_t st) {
    SCH_TP_SWITCH(A.n / 8, template window<SCH_SOLVER_EA>(A, io, N, st))
}
template <>
int launch_jitter<float, 8, SCH_SOLVER_EA>(const ModelArgs<float>& A, const JitterIO<float>& io, int N,
                                             cudaStream_t st) {
    SCH_TP_SWITCH(A.n / 8, template jitter<SCH_SOLVER_EA>(A, io, N, st))
}
template <>
int launch_helm<float, 8>(const ModelArgs<float>& A, const float* in, float* out, int mode, int N, cudaStream_t st) {
    SCH_TP_SWITCH(A.n / 8, helm(A, in, out, mode, N, st))
}
template <>
int launch_prior<float, 8>(const ModelArgs<float>& A, const float* ut, uint64_t seed, float scale, float* m, float* u,
                            int N, cudaStream_t st, int mode, int particle0) {
    SCH_TP_SWITCH(A.n / 8, prior(A, ut, seed, scale, m, u, N, st, mode, particle0))
}

#define SCH_TP_SMEM(tp, bufs)                                          \
    switch (tp) {                                                      \
        case 32: return Launch<float, 8, 32>::smem(Ns, K, bufs);     \
        case 64: return Launch<float, 8, 64>::smem(Ns, K, bufs);     \
        case 128: return Launch<float, 8, 128>::smem(Ns, K, bufs);   \
        case 256: return Launch<float, 8, 256>::smem(Ns, K, bufs);   \
        case 512: return Launch<float, 8, 512>::smem(Ns, K, bufs);   \
        default: return (size_t)-1;                                    \
    }

template <>
size_t window_smem<float, 8>(int tp, int Ns, int K) { SCH_TP_SMEM(tp, 1) }
template <>
size_t jitter_smem<float, 8>(int tp, int Ns, int K) { SCH_TP_SMEM(tp, 3) }

}  // namespace sch
