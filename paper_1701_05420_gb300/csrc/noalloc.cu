// cum_cumulants_noalloc: cum_cumulants with its workspace in a fixed device
// array owned by the library, for callers that cannot allocate device memory.
#include <mutex>

#include "cumgb.h"
#include "internal.h"

namespace cum {

// The workspace of every cum_cumulants_noalloc call.  Every GPU that loads the
// library holds these CUM_NOALLOC_WORKSPACE_BYTES until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_ws[CUM_NOALLOC_WORKSPACE_BYTES];

constexpr int kMaxDevices = 64;
static void* g_noalloc_ptr[kMaxDevices];
static std::mutex g_noalloc_mu;

// Device address of g_noalloc_ws on the current device.  In host code the
// array's name stands for a host-side shadow, so the address must come from
// cudaGetSymbolAddress, called with the device current, once per device.
static cudaError_t noalloc_ws(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_ws);
        if (e != cudaSuccess) return e;
        if (!p || ((uintptr_t)p % kWsAlign) != 0) return cudaErrorInvalidDevicePointer;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace cum

extern "C" int cum_cumulants_noalloc(const void* X, int dtype, int64_t t, int n, int64_t ldx, int d_max, int b,
                                     int prec, double* const* C_out, double* mean_out, void* stream)
{
    using namespace cum;
    if (!X || !C_out || (dtype != CUM_F32 && dtype != CUM_F64) || ldx < n) return CUM_EINVAL;
    if (d_max < 2 || d_max > kMaxOrder || !prec_is_valid(prec)) return CUM_EINVAL;
    for (int d = 2; d <= d_max; ++d)
        if (!C_out[d - 2]) return CUM_EINVAL;
    const size_t need = cum_workspace_size(t, n, d_max, b, prec);
    if (need == 0) return CUM_EINVAL;
    if (need > (size_t)CUM_NOALLOC_WORKSPACE_BYTES) return CUM_EUNSUPPORTED;  // request too large for the array
    void* ws = nullptr;
    cudaError_t e = noalloc_ws(&ws);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e);
    }
    // cum_cumulants clears the status word itself; every other workspace region
    // it reads was written earlier in the same call.
    return cum_cumulants(X, dtype, t, n, ldx, d_max, b, prec, C_out, mean_out, ws,
                         (size_t)CUM_NOALLOC_WORKSPACE_BYTES, stream);
}
