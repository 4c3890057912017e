// A 1D stencil run that allocates no memory.
//
// Some callers cannot call cudaMalloc: code embedded in a framework whose own
// allocator owns all device memory, and real-time or pre-allocated
// deployments that must not touch the allocator after start-up.
// stencil_run needs a plan, and a plan allocates its scratch on first use, so
// such callers get this entry point instead.  Its intermediate grid lives in a
// file-scope device array of fixed size; the caller passes only the input and
// the output.
#include <algorithm>
#include <mutex>

#include "plan.h"

namespace {

// Largest intermediate grid the entry point accepts: 16 MiB, i.e. 4 Mi FP32
// or 2 Mi FP64 points.  Every GPU that loads this library keeps the array
// until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per device.
// In host code the array's name is only a host-side stand-in, so kernels must
// be given this address, never the name.
cudaError_t scratch_on_current_device(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" stencil_status_t stencil_run_1d_noalloc(const void *in, void *out, int64_t n, int radius,
                                                   const double *coeffs, int64_t T,
                                                   stencil_dtype_t dtype, stencil_stream_t stream)
{
    using namespace sg;
    if (!in || !out || !coeffs || n < 1 || T < 0 || radius < 1 ||
        (dtype != STENCIL_F32 && dtype != STENCIL_F64)) {
        set_error("stencil_run_1d_noalloc: bad argument");
        return STENCIL_ERR_INVALID_ARG;
    }
    if (n < 2 * radius + 1) {
        set_error("stencil_run_1d_noalloc: n below 2r+1");
        return STENCIL_ERR_INVALID_ARG;
    }
    const bool f64 = dtype == STENCIL_F64;
    if (!sweep1d_supported(radius, f64)) {
        set_error("stencil_run_1d_noalloc: no kernel for radius %d", radius);
        return STENCIL_ERR_UNSUPPORTED;
    }
    const size_t esz = f64 ? 8 : 4;
    const size_t bytes = esz * (size_t)n;
    if (bytes > kNoAllocScratchBytes) {
        set_error("stencil_run_1d_noalloc: grid of %zu bytes exceeds the fixed %zu-byte scratch",
                  bytes, kNoAllocScratchBytes);
        return STENCIL_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    void *scratch = nullptr;
    cudaError_t e = scratch_on_current_device(&scratch);
    if (e != cudaSuccess) return cuda_fail(e, "stencil_run_1d_noalloc scratch address");
    if (T == 0) {
        if (in == out) return STENCIL_OK;
        e = cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "stencil_run_1d_noalloc copy");
    }
    // Passes of up to 32 steps.  Each pass reads one buffer and writes the
    // other; the pass count is made to end on `out` and, when in == out, the
    // first pass writes the scratch so that no pass reads what it writes.
    const int bmax = 32;
    int64_t npass = (T + bmax - 1) / bmax;
    const bool first_to_scratch = (in == out) || (npass % 2 == 0);
    if ((in == out) && npass % 2 == 1) npass += 1;  // one more, shorter pass
    if (npass > T) {
        // T = 1 with in == out: two passes are impossible, go through the
        // scratch with a one-step pass and copy back
        Sweep1DArgs a;
        a.src = in;
        a.dst = scratch;
        a.n = n;
        a.tile = f64 ? 2048 : 4096;
        a.b = 1;
        for (int k = 0; k < 2 * radius + 1; ++k) a.c[k] = coeffs[k];
        e = launch_sweep1d(radius, f64, a, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, scratch, bytes, cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "stencil_run_1d_noalloc");
    }
    const void *src = in;
    bool to_scratch = first_to_scratch;
    int64_t left = T;
    for (int64_t i = 0; i < npass; ++i) {
        const int64_t passes_left = npass - i;
        const int b = (int)std::min<int64_t>(bmax, left - (passes_left - 1));
        Sweep1DArgs a;
        a.src = src;
        a.dst = to_scratch ? scratch : out;
        a.n = n;
        a.tile = f64 ? 2048 : 4096;
        a.b = b;
        for (int k = 0; k < 2 * radius + 1; ++k) a.c[k] = coeffs[k];
        e = launch_sweep1d(radius, f64, a, s);
        if (e != cudaSuccess) return cuda_fail(e, "stencil_run_1d_noalloc launch");
        src = a.dst;
        to_scratch = !to_scratch;
        left -= b;
    }
    return STENCIL_OK;
}
