// Window and jitter kernels for double fields with the linearly implicit Picard
// solver (chunks of 4 nodes per thread, TP = 32 .. 512).
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
int launch_window<double, 4, SCH_SOLVER_LI>(const ModelArgs<double>& A, const WindowIO<double>& io, int N,
                                             cudaStream_t st) {
    SCH_TP_SWITCH(A.n / 4, template window<SCH_SOLVER_LI>(A, io, N, st))
}
template <>
int launch_jitter<double, 4, SCH_SOLVER_LI>(const ModelArgs<double>& A, const JitterIO<double>& io, int N,
                                             cudaStream_t st) {
    SCH_TP_SWITCH(A.n / 4, template jitter<SCH_SOLVER_LI>(A, io, N, st))
}

}  // namespace sch
