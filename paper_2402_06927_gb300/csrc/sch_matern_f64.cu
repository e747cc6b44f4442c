// Window and jitter kernels with the paper's Matern SALT noise (Eq. noise_solve2) for
// double fields, chunks of 4 nodes per thread, TP = 32 .. 512 (n = 4 TP), with the
// linearly implicit Picard solver (the FP64 default).
#include "sch_matern.cuh"

namespace sch {

#define SCH_TP_SWITCH(expr_tp, ...)                       \
    switch (expr_tp) {                                    \
        case 32: return LaunchMatern<double, 4, 32>::__VA_ARGS__; \
        case 64: return LaunchMatern<double, 4, 64>::__VA_ARGS__; \
        case 128: return LaunchMatern<double, 4, 128>::__VA_ARGS__; \
        case 256: return LaunchMatern<double, 4, 256>::__VA_ARGS__; \
        case 512: return LaunchMatern<double, 4, 512>::__VA_ARGS__; \
        default: return SCH_ERR_UNSUPPORTED;              \
    }

template <>
int launch_window_matern<double, 4>(const ModelArgs<double>& A, const WindowIO<double>& io, int N, cudaStream_t st) {
    SCH_TP_SWITCH(A.n / 4, template window<SCH_SOLVER_LI>(A, io, N, st))
}
template <>
int launch_jitter_matern<double, 4>(const ModelArgs<double>& A, const JitterIO<double>& io, int N, cudaStream_t st) {
    SCH_TP_SWITCH(A.n / 4, template jitter<SCH_SOLVER_LI>(A, io, N, st))
}

}  // namespace sch
