// 1D stencil sweeps in FP32 or FP64, temporally blocked in shared memory.
//
// Each CTA owns `tile` consecutive outputs.  It loads them with a halo of
// H = b*R points per side (periodic indices, coalesced loads), runs b steps
// of the stencil between two shared-memory buffers on a region that shrinks
// by R per step, and writes its outputs.  A whole 2^20-point grid lives in
// L2, so one launch covers many steps (Section 3.4's time-loop fusion inside
// a tile; the redundant rim costs about b*R/tile extra work).
#include "device_common.cuh"
#include "internal.h"

namespace sg {
namespace {

constexpr int NT1 = 256;

template <typename T, int R>
__global__ void __launch_bounds__(NT1) k_sweep1d(const __grid_constant__ Sweep1DArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = a.b * R;
    const int L = a.tile + 2 * H;
    T *buf0 = reinterpret_cast<T *>(smem);
    T *buf1 = buf0 + L;
    const long long n = a.n;
    const long long x0 = (long long)blockIdx.x * a.tile - H;
    const T *__restrict__ src = static_cast<const T *>(a.src);
    T *__restrict__ dst = static_cast<T *>(a.dst);

    T w[2 * R + 1];
#pragma unroll
    for (int j = 0; j < 2 * R + 1; ++j) w[j] = static_cast<T>(a.c[j]);

    for (int k = threadIdx.x; k < L; k += NT1) {
        long long g = (x0 + k) % n;
        if (g < 0) g += n;
        buf0[k] = src[g];
    }
    __syncthreads();

    T *in = buf0, *out = buf1;
    for (int s = 0; s < a.b; ++s) {
        const int lo = (s + 1) * R, hi = L - (s + 1) * R;
        const bool last = (s == a.b - 1);
        for (int k = lo + threadIdx.x; k < hi; k += NT1) {
            T acc = 0;
#pragma unroll
            for (int j = 0; j < 2 * R + 1; ++j) acc = fma(w[j], in[k + j - R], acc);
            if (last) {
                const long long g = x0 + k;
                if (g < n) dst[g] = acc;
            } else {
                out[k] = acc;
            }
        }
        __syncthreads();
        T *t = in;
        in = out;
        out = t;
    }
}

template <typename T, int R>
cudaError_t launch_t(const Sweep1DArgs &a, cudaStream_t s)
{
    const cudaError_t e = smem_optin((const void *)k_sweep1d<T, R>);
    if (e != cudaSuccess) return e;
    const int H = a.b * R;
    const size_t smem = 2 * sizeof(T) * (size_t)(a.tile + 2 * H);
    const long long nt = (a.n + a.tile - 1) / a.tile;
    k_sweep1d<T, R><<<(unsigned)nt, NT1, smem, s>>>(a);
    return cudaGetLastError();
}

#define SG_SWEEP1D_LIST(X) X(1) X(2) X(3) X(4) X(6) X(8) X(12) X(16)

}  // namespace

bool sweep1d_supported(int R, bool f64)
{
    (void)f64;
#define SG_X(R_) \
    if (R == R_) return true;
    SG_SWEEP1D_LIST(SG_X)
#undef SG_X
    return false;
}

cudaError_t launch_sweep1d(int R, bool f64, const Sweep1DArgs &a, cudaStream_t s)
{
#define SG_X(R_)                                                       \
    if (R == R_) return f64 ? launch_t<double, R_>(a, s) : launch_t<float, R_>(a, s);
    SG_SWEEP1D_LIST(SG_X)
#undef SG_X
    return cudaErrorInvalidValue;
}

}  // namespace sg
