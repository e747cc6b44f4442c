// Window and jitter kernels for float fields with the linearly implicit Picard
// solver (chunks of 8 nodes per thread, TP = 32 .. 512).
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
int launch_window<float, 8, SCH_SOLVER_LI>(const ModelArgs<float>& A, const WindowIO<float>& io, int N,
                                             cudaStream_t st) {
    SCH_TP_SWITCH(A.n / 8, template window<SCH_SOLVER_LI>(A, io, N, st))
}
template <>
int launch_jitter<float, 8, SCH_SOLVER_LI>(const ModelArgs<float>& A, const JitterIO<float>& io, int N,
                                             cudaStream_t st) {
    SCH_TP_SWITCH(A.n / 8, template jitter<SCH_SOLVER_LI>(A, io, N, st))
}

}  // namespace sch
