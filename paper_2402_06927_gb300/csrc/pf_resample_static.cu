// pf_resample_static: systematic resampling with in-place row gathers staged
// through a scratch buffer that the library itself holds, for callers that
// cannot allocate device memory (see include/sch.h for who they are).
//
// The scratch is a file-scope __device__ array of PF_RESAMPLE_STATIC_BYTES.
// Every GPU that loads this library keeps it until the process exits.  Host
// code cannot use the array's name as a device address, so the first call on
// each device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it; later calls on that device reuse the cached address.
#include <mutex>

#include "sch_internal.h"

namespace sch {

// the library-owned scratch (shared by every call on a device)
static __device__ __align__(256) unsigned char g_resample_scratch[PF_RESAMPLE_STATIC_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// device address of g_resample_scratch on the current device (set up once per device)
int static_scratch(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SCH_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SCH_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_resample_scratch);
        if (e != cudaSuccess || p == nullptr) return SCH_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SCH_OK;
}

}  // namespace
}  // namespace sch

extern "C" int pf_resample_static(int N, const double* wbar, uint64_t seed, uint64_t stage_ctr, int32_t* idx,
                                  int n_arrays, void* const* arrays, const size_t* row_bytes, void* stream) {
    using namespace sch;
    if (N <= 0 || N > 8192 || !wbar || !idx || n_arrays < 0) return SCH_ERR_ARG;
    for (int a = 0; a < n_arrays; ++a) {
        if (!arrays || !row_bytes || !arrays[a] || row_bytes[a] == 0 || row_bytes[a] % 16 != 0 ||
            ((uintptr_t)arrays[a] & 15))
            return SCH_ERR_ARG;
        // each array is staged whole in the scratch before it is copied back
        if ((size_t)N * row_bytes[a] > (size_t)PF_RESAMPLE_STATIC_BYTES) return SCH_ERR_WORKSPACE;
    }
    void* ws = nullptr;
    if (n_arrays > 0) {
        const int rc = static_scratch(&ws);
        if (rc != SCH_OK) return rc;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = launch_resample_idx(N, wbar, seed, stage_ctr, nullptr, idx, st);
    if (rc != SCH_OK) return rc;
    for (int a = 0; a < n_arrays; ++a) {
        rc = launch_gather(N, idx, arrays[a], ws, row_bytes[a], st);
        if (rc != SCH_OK) return rc;
        rc = launch_copy(ws, arrays[a], (size_t)N * row_bytes[a], st);
        if (rc != SCH_OK) return rc;
    }
    return SCH_OK;
}
