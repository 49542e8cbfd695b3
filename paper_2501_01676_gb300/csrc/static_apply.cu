// bddc_apply_static: the preconditioner apply without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// apply the preconditioner -- for example a host framework that hands out all
// device memory itself and forbids libraries from allocating behind its back,
// or code on a latency-critical path where an allocation call could
// synchronise the device.  bddc_apply itself allocates nothing per call, but
// it writes its two work vectors into buffers owned by the context; this
// variant writes them into one file-scope array instead.
//
// The array is a fixed 8 MiB (2^20 doubles) in device memory of every GPU on
// which the library is loaded, held until the process exits.  Every call,
// from every context on that GPU, shares it, and it keeps the contents of the
// last call; the kernels clear what has to start at zero.  Two calls that
// overlap on the GPU (different streams, no ordering between them) race on
// the array and give wrong results.  The context's device must be the current
// device: its address of the array is looked up with that device current.
#include <cuda_runtime.h>

#include <mutex>

#include "bddc_internal.h"

#define BDDC_STATIC_WORK_DOUBLES (1u << 20)

static __device__ __align__(256) double g_static_work[BDDC_STATIC_WORK_DOUBLES];

int bddc_apply_into(bddc_ctx* C, const double* r, double* z, int nrhs, double* work, size_t work_doubles);
int bddc_ctx_device(const bddc_ctx* C);

namespace {
constexpr int MAX_DEVICES = 256;
std::mutex g_mu;
double* g_addr[MAX_DEVICES] = {nullptr};

// Device address of the array on device `want`, which must be the current
// device; looked up once per device (host code only sees a host-side stand-in
// under the array's name).
int static_work_address(int want, double** out) {
    int dev = 0;
    BDDC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != want) {
        bddc_set_last_error("the context's device is not the current device", __FILE__, __LINE__);
        return BDDC_EINVAL;
    }
    if (dev < 0 || dev >= MAX_DEVICES) return BDDC_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_work);
        if (e != cudaSuccess) {
            bddc_set_last_error(cudaGetErrorString(e), __FILE__, __LINE__);
            return BDDC_ECUDA;
        }
        g_addr[dev] = (double*)p;
    }
    *out = g_addr[dev];
    return BDDC_OK;
}
}  // namespace

extern "C" int bddc_apply_static(bddc_ctx* ctx, const double* r_dev, double* z_dev, int nrhs) {
    if (!ctx || !r_dev || !z_dev || nrhs < 1) return BDDC_EINVAL;
    double* work = nullptr;
    BDDC_TRY(static_work_address(bddc_ctx_device(ctx), &work));
    return bddc_apply_into(ctx, r_dev, z_dev, nrhs, work, BDDC_STATIC_WORK_DOUBLES);
}
