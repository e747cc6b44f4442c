// Adjoint-window and nudging kernels for double fields (chunks of 4 nodes per
// thread, TP = 32 .. 512); the forward recomputation uses the default Picard
// solver of this precision (the other one returns SCH_ERR_UNSUPPORTED).
#include "sch_adjoint.cuh"

namespace sch {

#define SCH_ADJ_SWITCH(expr_tp, call)                        \
    switch (expr_tp) {                                       \
        case 32: return LaunchAdj<double, 4, 32>::call;     \
        case 64: return LaunchAdj<double, 4, 64>::call;     \
        case 128: return LaunchAdj<double, 4, 128>::call;   \
        case 256: return LaunchAdj<double, 4, 256>::call;   \
        case 512: return LaunchAdj<double, 4, 512>::call;   \
        default: return SCH_ERR_UNSUPPORTED;                 \
    }

template <>
int launch_adjoint<double, 4, SCH_SOLVER_LI>(const ModelArgs<double>& A, const AdjointIO<double>& io, int N,
                                              cudaStream_t st) {
    SCH_ADJ_SWITCH(A.n / 4, template adjoint<SCH_SOLVER_LI>(A, io, N, st))
}
template <>
int launch_adjoint<double, 4, SCH_SOLVER_EA>(const ModelArgs<double>& A, const AdjointIO<double>& io, int N,
                                              cudaStream_t st) {
    (void)A; (void)io; (void)N; (void)st;
    return SCH_ERR_UNSUPPORTED;   // only the default solver of this precision is compiled
}
template <>
int launch_nudge<double, 4, SCH_SOLVER_LI>(const ModelArgs<double>& A, const NudgeIO<double>& io, int N,
                                            cudaStream_t st) {
    SCH_ADJ_SWITCH(A.n / 4, template nudge<SCH_SOLVER_LI>(A, io, N, st))
}
template <>
int launch_nudge<double, 4, SCH_SOLVER_EA>(const ModelArgs<double>& A, const NudgeIO<double>& io, int N,
                                            cudaStream_t st) {
    (void)A; (void)io; (void)N; (void)st;
    return SCH_ERR_UNSUPPORTED;   // only the default solver of this precision is compiled
}

#define SCH_ADJ_SMEM(tp, fn)                                      \
    switch (tp) {                                                 \
        case 32: return LaunchAdj<double, 4, 32>::fn(Ns, K);     \
        case 64: return LaunchAdj<double, 4, 64>::fn(Ns, K);     \
        case 128: return LaunchAdj<double, 4, 128>::fn(Ns, K);   \
        case 256: return LaunchAdj<double, 4, 256>::fn(Ns, K);   \
        case 512: return LaunchAdj<double, 4, 512>::fn(Ns, K);   \
        default: return (size_t)-1;                               \
    }

template <>
size_t adjoint_smem<double, 4>(int tp, int Ns, int K) { SCH_ADJ_SMEM(tp, adj_smem) }
template <>
size_t nudge_smem<double, 4>(int tp, int Ns, int K) { SCH_ADJ_SMEM(tp, nudge_smem) }

}  // namespace sch
