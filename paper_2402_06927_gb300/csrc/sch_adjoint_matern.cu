// Adjoint-window kernels with the paper's Matern SALT noise (Eq. noise_solve2) for both
// precisions, each with its default Picard solver: chunks of 4 (double) or 8 (float)
// nodes per thread, TP = 32 .. 512.
#include "sch_adjoint.cuh"

namespace sch {

#define SCH_ADJ_MATERN_SWITCH(R, C, S, expr_tp, fn)                                               \
    switch (expr_tp) {                                                                            \
        case 32: return LaunchAdj<R, C, 32>::template fn<S>(A, io, N, st);                      \
        case 64: return LaunchAdj<R, C, 64>::template fn<S>(A, io, N, st);                      \
        case 128: return LaunchAdj<R, C, 128>::template fn<S>(A, io, N, st);                    \
        case 256: return LaunchAdj<R, C, 256>::template fn<S>(A, io, N, st);                    \
        case 512: return LaunchAdj<R, C, 512>::template fn<S>(A, io, N, st);                    \
        default: return SCH_ERR_UNSUPPORTED;                                                      \
    }

template <>
int launch_adjoint_matern<double, 4>(const ModelArgs<double>& A, const AdjointIO<double>& io, int N,
                                     cudaStream_t st) {
    SCH_ADJ_MATERN_SWITCH(double, 4, SCH_SOLVER_LI, A.n / 4, adjoint_matern)
}

template <>
int launch_nudge_matern<double, 4>(const ModelArgs<double>& A, const NudgeIO<double>& io, int N, cudaStream_t st) {
    SCH_ADJ_MATERN_SWITCH(double, 4, SCH_SOLVER_LI, A.n / 4, nudge_matern)
}

template <>
int launch_adjoint_matern<float, 8>(const ModelArgs<float>& A, const AdjointIO<float>& io, int N, cudaStream_t st) {
    SCH_ADJ_MATERN_SWITCH(float, 8, SCH_SOLVER_EA, A.n / 8, adjoint_matern)
}

template <>
int launch_nudge_matern<float, 8>(const ModelArgs<float>& A, const NudgeIO<float>& io, int N, cudaStream_t st) {
    SCH_ADJ_MATERN_SWITCH(float, 8, SCH_SOLVER_EA, A.n / 8, nudge_matern)
}

}  // namespace sch
