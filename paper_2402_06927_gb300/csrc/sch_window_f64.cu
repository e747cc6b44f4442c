// Instantiations of the particle kernels for double fields, chunks of 4 nodes
// per thread and CTA sizes TP = 32 .. 512 (n = 4 TP): utilities, and the
// window and jitter kernels with the explicit-advection Picard solver.
#include "sch_kernels.cuh"

namespace sch {

#define SCH_TP_SWITCH(expr_tp, call)                      \
    switch (expr_tp) {                                    \
        case 32: return Launch<double, 4, 32>::call;     \
        case 64: return Launch<double, 4, 64>::call;     \
        case 128: return Launch<double, 4, 128>::call;   \
        case 256: return Launch<double, 4, 256>::call;   \
        case 512: return Launch<double, 4, 512>::call;   \
        default: return SCH_ERR_UNSUPPORTED;              \
    }

template <>
int launch_window<double, 4, SCH_SOLVER_EA>(const ModelArgs<double>& A, const WindowIO<double>& io, int N,
                                             cudaStream_t st) {
    SCH_TP_SWITCH(A.n / 4, template window<SCH_SOLVER_EA>(A, io, N, st))
}
template <>
int launch_jitter<double, 4, SCH_SOLVER_EA>(const ModelArgs<double>& A, const JitterIO<double>& io, int N,
                                             cudaStream_t st) {
    SCH_TP_SWITCH(A.n / 4, template jitter<SCH_SOLVER_EA>(A, io, N, st))
}
template <>
int launch_helm<double, 4>(const ModelArgs<double>& A, const double* in, double* out, int mode, int N, cudaStream_t st) {
    SCH_TP_SWITCH(A.n / 4, helm(A, in, out, mode, N, st))
}
template <>
int launch_prior<double, 4>(const ModelArgs<double>& A, const double* ut, uint64_t seed, double scale, double* m, double* u,
                            int N, cudaStream_t st, int mode, int particle0) {
    SCH_TP_SWITCH(A.n / 4, prior(A, ut, seed, scale, m, u, N, st, mode, particle0))
}

#define SCH_TP_SMEM(tp, bufs)                                          \
    switch (tp) {                                                      \
        case 32: return Launch<double, 4, 32>::smem(Ns, K, bufs);     \
        case 64: return Launch<double, 4, 64>::smem(Ns, K, bufs);     \
        case 128: return Launch<double, 4, 128>::smem(Ns, K, bufs);   \
        case 256: return Launch<double, 4, 256>::smem(Ns, K, bufs);   \
        case 512: return Launch<double, 4, 512>::smem(Ns, K, bufs);   \
        default: return (size_t)-1;                                    \
    }

template <>
size_t window_smem<double, 4>(int tp, int Ns, int K) { SCH_TP_SMEM(tp, 1) }
template <>
size_t jitter_smem<double, 4>(int tp, int Ns, int K) { SCH_TP_SMEM(tp, 3) }

}  // namespace sch
