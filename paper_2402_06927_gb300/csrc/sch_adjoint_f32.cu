// Adjoint-window and nudging kernels for float fields (chunks of 8 nodes per
// thread, TP = 32 .. 512); the forward recomputation uses the default Picard
// solver of this precision (the other one returns SCH_ERR_UNSUPPORTED).
#include "sch_adjoint.cuh"

namespace sch {

#define SCH_ADJ_SWITCH(expr_tp, call)                        \
    switch (expr_tp) {                                       \
        case 32: return LaunchAdj<float, 8, 32>::call;     \
        case 64: return LaunchAdj<float, 8, 64>::call;     \
        case 128: return LaunchAdj<float, 8, 128>::call;   \
        case 256: return LaunchAdj<float, 8, 256>::call;   \
        case 512: return LaunchAdj<float, 8, 512>::call;   \
        default: return SCH_ERR_UNSUPPORTED;                 \
    }

template <>
int launch_adjoint<float, 8, SCH_SOLVER_LI>(const ModelArgs<float>& A, const AdjointIO<float>& io, int N,
                                              cudaStream_t st) {
    (void)A; (void)io; (void)N; (void)st;
    return SCH_ERR_UNSUPPORTED;   // only the default solver of this precision is compiled
}
template <>
int launch_adjoint<float, 8, SCH_SOLVER_EA>(const ModelArgs<float>& A, const AdjointIO<float>& io, int N,
                                              cudaStream_t st) {
    SCH_ADJ_SWITCH(A.n / 8, template adjoint<SCH_SOLVER_EA>(A, io, N, st))
}
template <>
int launch_nudge<float, 8, SCH_SOLVER_LI>(const ModelArgs<float>& A, const NudgeIO<float>& io, int N,
                                            cudaStream_t st) {
    (void)A; (void)io; (void)N; (void)st;
    return SCH_ERR_UNSUPPORTED;   // only the default solver of this precision is compiled
}
template <>
int launch_nudge<float, 8, SCH_SOLVER_EA>(const ModelArgs<float>& A, const NudgeIO<float>& io, int N,
                                            cudaStream_t st) {
    SCH_ADJ_SWITCH(A.n / 8, template nudge<SCH_SOLVER_EA>(A, io, N, st))
}

#define SCH_ADJ_SMEM(tp, fn)                                      \
    switch (tp) {                                                 \
        case 32: return LaunchAdj<float, 8, 32>::fn(Ns, K);     \
        case 64: return LaunchAdj<float, 8, 64>::fn(Ns, K);     \
        case 128: return LaunchAdj<float, 8, 128>::fn(Ns, K);   \
        case 256: return LaunchAdj<float, 8, 256>::fn(Ns, K);   \
        case 512: return LaunchAdj<float, 8, 512>::fn(Ns, K);   \
        default: return (size_t)-1;                               \
    }

template <>
size_t adjoint_smem<float, 8>(int tp, int Ns, int K) { SCH_ADJ_SMEM(tp, adj_smem) }
template <>
size_t nudge_smem<float, 8>(int tp, int Ns, int K) { SCH_ADJ_SMEM(tp, nudge_smem) }

}  // namespace sch
