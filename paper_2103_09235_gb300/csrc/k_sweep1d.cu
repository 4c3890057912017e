// 1D stencil sweeps in FP32 or FP64, temporally blocked in shared memory.
//
// Each CTA owns `tile` consecutive outputs.  It loads them with a halo of
// H = b*R points per side (periodic indices, coalesced loads), runs b steps
// of the stencil between two shared-memory buffers on a region that shrinks
// by R per step, and writes its outputs.  A whole 2^20-point grid lives in
// L2, so one launch covers many steps (Section 3.4's time-loop fusion inside
// a tile; the redundant rim costs about b*R/tile extra work).
//
// FP32 steps of radius 4 and up work on strips of V = 8 consecutive outputs
// per thread: the
// strip and its 2R neighbours come in as 16-byte shared-memory loads (R
// rounded up to whole loads), and the 2R+1 taps of all eight outputs are
// summed from registers, so a step reads (8 + 2R)/8 values per output
// instead of 2R+1.  The buffers carry a pad before and after the tile so
// that a strip cut by the region's edge still loads whole 16-byte words; the
// outputs outside the region are computed from whatever the pad or the
// previous step left there and are never stored, nor read by the next step.
// FP64 steps, and FP32 steps of smaller radius, keep one output per thread
// (FP64 is bound by its FMA rate, not shared-memory traffic).
#include "device_common.cuh"
#include "internal.h"

namespace sg {
namespace {

constexpr int NT1 = 256;

// FP32 strip geometry for radius R: V outputs per thread, the halo rounded up
// to whole 16-byte loads, and the pad in front of element 0 of a buffer.
template <int R>
struct Strip1 {
    static constexpr int V = 8;
    static constexpr int RP = (R + 3) / 4 * 4;
    static constexpr int NSEG = V + 2 * RP;
    static constexpr int PAD = RP + V;
};

// Floats of one FP32 buffer for a tile of L = tile + 2H points.
template <int R>
__host__ __device__ constexpr int strip1_buf_floats(int L)
{
    return Strip1<R>::PAD + (L + Strip1<R>::V - 1) / Strip1<R>::V * Strip1<R>::V + Strip1<R>::PAD;
}

// FP32: b steps with 8-output strips.
template <int R>
__global__ void __launch_bounds__(NT1) k_sweep1d_f32(const __grid_constant__ Sweep1DArgs a)
{
    using S = Strip1<R>;
    constexpr int V = S::V, RP = S::RP, NSEG = S::NSEG, PAD = S::PAD;
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = a.b * R;
    const int L = a.tile + 2 * H;
    const int LB = strip1_buf_floats<R>(L);
    float *buf0 = reinterpret_cast<float *>(smem) + PAD;  // element 0 of each buffer
    float *buf1 = buf0 + LB;
    const long long n = a.n;
    const long long x0 = (long long)blockIdx.x * a.tile - H;
    const float *__restrict__ src = static_cast<const float *>(a.src);
    float *__restrict__ dst = static_cast<float *>(a.dst);

    float w[2 * R + 1];
#pragma unroll
    for (int j = 0; j < 2 * R + 1; ++j) w[j] = (float)a.c[j];

    for (int k = threadIdx.x; k < L; k += NT1) {
        long long g = (x0 + k) % n;
        if (g < 0) g += n;
        buf0[k] = src[g];
    }
    __syncthreads();

    float *in = buf0, *out = buf1;
    for (int s = 0; s < a.b; ++s) {
        const int lo = (s + 1) * R, hi = L - (s + 1) * R;
        const bool last = (s == a.b - 1);
        const int g0 = lo / V, g1 = (hi + V - 1) / V;
        for (int g = g0 + (int)threadIdx.x; g < g1; g += NT1) {
            const int k0 = g * V;
            float seg[NSEG];
            const float4 *rp = reinterpret_cast<const float4 *>(in + k0 - RP);
#pragma unroll
            for (int q = 0; q < NSEG / 4; ++q) {
                const float4 t = rp[q];
                seg[4 * q] = t.x;
                seg[4 * q + 1] = t.y;
                seg[4 * q + 2] = t.z;
                seg[4 * q + 3] = t.w;
            }
            float acc[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                float t = 0.f;
#pragma unroll
                for (int j = 0; j < 2 * R + 1; ++j) t = fmaf(w[j], seg[v + j - R + RP], t);
                acc[v] = t;
            }
            if (last) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int k = k0 + v;
                    const long long gg = x0 + k;
                    if (k >= lo && k < hi && gg < n) dst[gg] = acc[v];
                }
            } else {
                float4 *op = reinterpret_cast<float4 *>(out + k0);
#pragma unroll
                for (int q = 0; q < V / 4; ++q)
                    op[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
            }
        }
        __syncthreads();
        float *t = in;
        in = out;
        out = t;
    }
}

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
    const int H = a.b * R;
    const long long nt = (a.n + a.tile - 1) / a.tile;
    // strips from radius 4: below it the eight outputs of a strip leave too
    // little work per step between barriers (measured on GB300, 2^20 points,
    // b = 32: radius 1 at 818 GS/s with strips against 974 without; radius 6
    // at 2084 against 1793)
    if constexpr (sizeof(T) == 4 && R >= 4) {
        const cudaError_t e = smem_optin((const void *)k_sweep1d_f32<R>);
        if (e != cudaSuccess) return e;
        const size_t smem = 2 * sizeof(float) * (size_t)strip1_buf_floats<R>(a.tile + 2 * H);
        k_sweep1d_f32<R><<<(unsigned)nt, NT1, smem, s>>>(a);
    } else {
        const cudaError_t e = smem_optin((const void *)k_sweep1d<T, R>);
        if (e != cudaSuccess) return e;
        const size_t smem = 2 * sizeof(T) * (size_t)(a.tile + 2 * H);
        k_sweep1d<T, R><<<(unsigned)nt, NT1, smem, s>>>(a);
    }
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
