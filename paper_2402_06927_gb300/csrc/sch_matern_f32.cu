// Window and jitter kernels with the paper's Matern SALT noise (Eq. noise_solve2) for
// float fields, chunks of 8 nodes per thread, TP = 32 .. 512 (n = 8 TP), with the
// explicit-advection Picard solver (the FP32 default).
#include "sch_matern.cuh"

namespace sch {

#define SCH_TP_SWITCH(expr_tp, ...)                       \
    switch (expr_tp) {                                    \
        case 32: return LaunchMatern<float, 8, 32>::__VA_ARGS__; \
        case 64: return LaunchMatern<float, 8, 64>::__VA_ARGS__; \
        case 128: return LaunchMatern<float, 8, 128>::__VA_ARGS__; \
        case 256: return LaunchMatern<float, 8, 256>::__VA_ARGS__; \
        case 512: return LaunchMatern<float, 8, 512>::__VA_ARGS__; \
        default: return SCH_ERR_UNSUPPORTED;              \
    }

template <>
int launch_window_matern<float, 8>(const ModelArgs<float>& A, const WindowIO<float>& io, int N, cudaStream_t st) {
    SCH_TP_SWITCH(A.n / 8, template window<SCH_SOLVER_EA>(A, io, N, st))
}
template <>
int launch_jitter_matern<float, 8>(const ModelArgs<float>& A, const JitterIO<float>& io, int N, cudaStream_t st) {
    SCH_TP_SWITCH(A.n / 8, template jitter<SCH_SOLVER_EA>(A, io, N, st))
}

}  // namespace sch
