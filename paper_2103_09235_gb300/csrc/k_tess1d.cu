// 1D folded sweeps by exact tessellate tiling (Section 3.4): b steps of the
// (folded) stencil per pass with no point computed twice, in two launches.
//
// Stage 1 (k_tess_tri): one CTA per tile of W points loads its tile (no halo)
// into shared memory and runs the b steps of its shrinking triangle between
// two shared-memory arrays (level s in array s mod 2).  It writes the points
// that reached level b to the destination, and both arrays' values within
// (b+1)R of its edges to the two global Jacobi arrays par0 / par1.
// Stage 2 (k_tess_inv): one CTA per tile boundary loads the 2(b+1)R points
// around it from par0 / par1 and runs the b steps of the inverted triangle,
// step s advancing the points within s*R of the boundary; it writes the 2bR
// points around the boundary to the destination.
// The ranges come from tess1d.h, which the host-side profile function uses
// too.  Compared with the overlapped tiles of k_sweep1d.cu this removes the
// recomputed rim (about (b-1)R/W of the work) at the cost of a second launch
// and the edge values' round trip through L2.
#include <algorithm>

#include "../../include/stencil.h"
#include "device_common.cuh"
#include "internal.h"
#include "tess1d.h"

namespace sg {
namespace {

constexpr int NTT = 256;

template <typename T, int R>
__device__ __forceinline__ void load_weights(const Tess1DArgs &a, T (&w)[2 * R + 1])
{
#pragma unroll
    for (int j = 0; j < 2 * R + 1; ++j) w[j] = static_cast<T>(a.c[j]);
}

template <typename T, int R>
__global__ void __launch_bounds__(NTT) k_tess_tri(const __grid_constant__ Tess1DArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int j = blockIdx.x;
    const long long x0 = (long long)j * a.W;
    const int Wj = (j == a.ntiles - 1) ? (int)(a.n - x0) : a.W;
    T *buf0 = reinterpret_cast<T *>(smem);
    T *buf1 = buf0 + a.wmax;
    const T *__restrict__ src = static_cast<const T *>(a.src);
    T *__restrict__ dst = static_cast<T *>(a.dst);
    T *__restrict__ par0 = static_cast<T *>(a.par0);
    T *__restrict__ par1 = static_cast<T *>(a.par1);
    T w[2 * R + 1];
    load_weights<T, R>(a, w);

    for (int i = threadIdx.x; i < Wj; i += NTT) {
        const T v = src[x0 + i];
        buf0[i] = v;
        buf1[i] = v;  // level 0 in both arrays: never read as level 1, but defined
    }
    __syncthreads();
    for (int s = 1; s <= a.b; ++s) {
        const T *in = (s & 1) ? buf0 : buf1;
        T *out = (s & 1) ? buf1 : buf0;
        const int hi = tess::s1_hi(s, R, Wj);
        for (int i = tess::s1_lo(s, R) + threadIdx.x; i < hi; i += NTT) {
            T acc = 0;
#pragma unroll
            for (int k = 0; k < 2 * R + 1; ++k) acc = fma(w[k], in[i + k - R], acc);
            out[i] = acc;
        }
        __syncthreads();
    }
    const T *top = (a.b & 1) ? buf1 : buf0;
    const int E = tess::s2_half(a.b, R);
    for (int i = threadIdx.x; i < Wj; i += NTT) {
        if (i < E || i >= Wj - E) {
            par0[x0 + i] = buf0[i];
            par1[x0 + i] = buf1[i];
        }
        if (i >= tess::s1_lo(a.b, R) && i < tess::s1_hi(a.b, R, Wj)) dst[x0 + i] = top[i];
    }
}

// FP32 stage 1 for radius 4 and up: each thread advances strips of 8
// consecutive points from 16-byte shared-memory loads, as the overlapped
// kernel does (k_sweep1d.cu).  Both arrays carry a pad so that strips cut by
// the region's edge still load whole words; a strip writes only the points
// of its step's region, since the points outside keep the older levels that
// the export and stage 2 read.
template <int R>
struct TriStrip {
    static constexpr int V = 8;
    static constexpr int RP = (R + 3) / 4 * 4;
    static constexpr int NSEG = V + 2 * RP;
    static constexpr int PAD = RP + V;
};

template <int R>
__host__ __device__ constexpr int tri_buf_floats(int wmax)
{
    return TriStrip<R>::PAD + (wmax + TriStrip<R>::V - 1) / TriStrip<R>::V * TriStrip<R>::V +
           TriStrip<R>::PAD;
}

template <int R>
__global__ void __launch_bounds__(NTT) k_tess_tri_f32(const __grid_constant__ Tess1DArgs a)
{
    using S = TriStrip<R>;
    constexpr int V = S::V, RP = S::RP, NSEG = S::NSEG, PAD = S::PAD;
    extern __shared__ __align__(16) unsigned char smem[];
    const int j = blockIdx.x;
    const long long x0 = (long long)j * a.W;
    const int Wj = (j == a.ntiles - 1) ? (int)(a.n - x0) : a.W;
    float *buf0 = reinterpret_cast<float *>(smem) + PAD;  // element 0 of each array
    float *buf1 = buf0 + tri_buf_floats<R>(a.wmax);
    const float *__restrict__ src = static_cast<const float *>(a.src);
    float *__restrict__ dst = static_cast<float *>(a.dst);
    float *__restrict__ par0 = static_cast<float *>(a.par0);
    float *__restrict__ par1 = static_cast<float *>(a.par1);
    float w[2 * R + 1];
    load_weights<float, R>(a, w);

    for (int i = threadIdx.x; i < Wj; i += NTT) {
        const float v = src[x0 + i];
        buf0[i] = v;
        buf1[i] = v;  // level 0 in both arrays: never read as level 1, but defined
    }
    __syncthreads();
    for (int s = 1; s <= a.b; ++s) {
        const float *in = (s & 1) ? buf0 : buf1;
        float *out = (s & 1) ? buf1 : buf0;
        const int lo = tess::s1_lo(s, R), hi = tess::s1_hi(s, R, Wj);
        const int g0 = lo / V, g1 = (hi + V - 1) / V;
        for (int g = g0 + (int)threadIdx.x; g < g1; g += NTT) {
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
                for (int k = 0; k < 2 * R + 1; ++k) t = fmaf(w[k], seg[v + k - R + RP], t);
                acc[v] = t;
            }
            if (k0 >= lo && k0 + V <= hi) {
                float4 *op = reinterpret_cast<float4 *>(out + k0);
                op[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
                op[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (k0 + v >= lo && k0 + v < hi) out[k0 + v] = acc[v];
            }
        }
        __syncthreads();
    }
    const float *top = (a.b & 1) ? buf1 : buf0;
    const int E = tess::s2_half(a.b, R);
    for (int i = threadIdx.x; i < Wj; i += NTT) {
        if (i < E || i >= Wj - E) {
            par0[x0 + i] = buf0[i];
            par1[x0 + i] = buf1[i];
        }
        if (i >= tess::s1_lo(a.b, R) && i < tess::s1_hi(a.b, R, Wj)) dst[x0 + i] = top[i];
    }
}

template <typename T, int R>
__global__ void __launch_bounds__(NTT) k_tess_inv(const __grid_constant__ Tess1DArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const long long xb = (long long)blockIdx.x * a.W;  // the boundary left of tile blockIdx.x
    const int E = tess::s2_half(a.b, R);
    T *buf0 = reinterpret_cast<T *>(smem);
    T *buf1 = buf0 + 2 * E;
    const T *__restrict__ par0 = static_cast<const T *>(a.par0);
    const T *__restrict__ par1 = static_cast<const T *>(a.par1);
    T *__restrict__ dst = static_cast<T *>(a.dst);
    T w[2 * R + 1];
    load_weights<T, R>(a, w);
    const long long n = a.n;
    auto wrap = [n](long long g) {
        g %= n;
        return g < 0 ? g + n : g;
    };
    // window index u = t + E for the offset t from the boundary, t in [-E, E)
    for (int u = threadIdx.x; u < 2 * E; u += NTT) {
        const long long g = wrap(xb - E + u);
        buf0[u] = par0[g];
        buf1[u] = par1[g];
    }
    __syncthreads();
    for (int s = 1; s <= a.b; ++s) {
        const T *in = (s & 1) ? buf0 : buf1;
        T *out = (s & 1) ? buf1 : buf0;
        const int hi = tess::s2_hi(s, R) + E;
        for (int u = tess::s2_lo(s, R) + E + threadIdx.x; u < hi; u += NTT) {
            T acc = 0;
#pragma unroll
            for (int k = 0; k < 2 * R + 1; ++k) acc = fma(w[k], in[u + k - R], acc);
            out[u] = acc;
        }
        __syncthreads();
    }
    const T *top = (a.b & 1) ? buf1 : buf0;
    const int lo = tess::s2_lo(a.b, R) + E, hi = tess::s2_hi(a.b, R) + E;
    for (int u = lo + threadIdx.x; u < hi; u += NTT) dst[wrap(xb - E + u)] = top[u];
}

template <typename T, int R>
cudaError_t launch_t(const Tess1DArgs &a, cudaStream_t s)
{
    cudaError_t e;
    if constexpr (sizeof(T) == 4 && R >= 4) {  // strips, as in k_sweep1d.cu
        e = smem_optin((const void *)k_tess_tri_f32<R>);
        if (e != cudaSuccess) return e;
        k_tess_tri_f32<R><<<a.ntiles, NTT, 2 * sizeof(float) * (size_t)tri_buf_floats<R>(a.wmax),
                            s>>>(a);
    } else {
        e = smem_optin((const void *)k_tess_tri<T, R>);
        if (e != cudaSuccess) return e;
        k_tess_tri<T, R><<<a.ntiles, NTT, 2 * sizeof(T) * (size_t)a.wmax, s>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem2 = 4 * sizeof(T) * (size_t)tess::s2_half(a.b, R);
    k_tess_inv<T, R><<<a.ntiles, NTT, smem2, s>>>(a);
    return cudaGetLastError();
}

#define SG_TESS_LIST(X) X(1) X(2) X(3) X(4) X(6) X(8) X(12) X(16)

}  // namespace

bool tess1d_fits(long long n, int W, int b, int R)
{
    const long long ntiles = std::max<long long>(1, n / W);
    const long long wmax = n - (ntiles - 1) * W;
    return b >= 1 && W >= tess::min_width(b, R) && n >= 2LL * tess::s2_half(b, R) &&
           wmax <= 2LL * W && 2 * sizeof(double) * wmax <= 200 * 1024;
}

cudaError_t launch_tess1d(int R, bool f64, const Tess1DArgs &a, cudaStream_t s)
{
#define SG_X(R_) \
    if (R == R_) return f64 ? launch_t<double, R_>(a, s) : launch_t<float, R_>(a, s);
    SG_TESS_LIST(SG_X)
#undef SG_X
    return cudaErrorInvalidValue;
}

}  // namespace sg

namespace sg {
void set_error(const char *fmt, ...);
}

// Host-only profile of the two stages (the same ranges the kernels use).
extern "C" stencil_status_t stencil_tessellation_counts(int W, int b, int R, int *stage1,
                                                       int *stage2)
{
    using namespace sg;
    if (W < 1 || b < 1 || R < 1 || !stage1 || !stage2 || W < tess::min_width(b, R)) {
        set_error("stencil_tessellation_counts: need W >= 2*b*R >= 2 and output arrays");
        return STENCIL_ERR_INVALID_ARG;
    }
    for (int i = 0; i < W; ++i) {
        int c1 = 0, c2 = 0;
        for (int s = 1; s <= b; ++s) {
            if (i >= tess::s1_lo(s, R) && i < tess::s1_hi(s, R, W)) ++c1;
            const int tl = i, tr = i - W;  // offsets from the left and the right boundary
            if ((tl >= tess::s2_lo(s, R) && tl < tess::s2_hi(s, R)) ||
                (tr >= tess::s2_lo(s, R) && tr < tess::s2_hi(s, R)))
                ++c2;
        }
        stage1[i] = c1;
        stage2[i] = c2;
    }
    return STENCIL_OK;
}
