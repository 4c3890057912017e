// FP64 sweeps of 2D and 3D grids, plain or folded (Section 3.2 folding: one
// sweep of c^(m) advances m steps), the paper's own precision.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so these sweeps are
// bound by the FP64 pipe, not by memory: the kernel keeps the arithmetic
// plain and exact in order.  One CTA computes a TX x TY x TZ block of outputs
// from a shared-memory copy of the block plus a halo of R points per side,
// loaded with periodic indices straight from the source grid (rows and
// planes at the caller's strides); each thread walks the nonzero taps of the
// folded weights, which sit in shared memory too.
#include "device_common.cuh"
#include "internal.h"

namespace sg {
namespace {

constexpr int FX = 32, FY = 8;   // output block in x and y
constexpr int NTF = FX * FY;     // one thread per (x, y) column of the block

__device__ __forceinline__ long long wrapl(long long v, long long n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// One sweep: dst = c (*) src, c of radius R as (2R+1)^ndim doubles.
__global__ void __launch_bounds__(NTF) k_sweep_f64(const __grid_constant__ SweepF64Args a)
{
    extern __shared__ __align__(16) double smf[];
    const int R = a.R, W = 2 * R + 1;
    const int tz = a.ndim == 3 ? a.tz : 1;
    const int hz = a.ndim == 3 ? R : 0;
    const int SX = FX + 2 * R, SY = FY + 2 * R, SZ = tz + 2 * hz;
    double *tile = smf;                                              // SZ x SY x SX
    int *taps = reinterpret_cast<int *>(smf + (size_t)SZ * SY * SX);  // nonzero taps' offsets
    double *tw = reinterpret_cast<double *>(taps + ((a.nnz + 1) & ~1));  // and weights

    const int bx = blockIdx.x % a.bx, rest = blockIdx.x / a.bx;
    const int by = rest % a.by, bz = rest / a.by;
    const long long x0 = (long long)bx * FX, y0 = (long long)by * FY, z0 = (long long)bz * tz;

    // the nonzero taps, as offsets into the tile
    if (threadIdx.x == 0) {
        int k = 0;
        for (int i = 0; i < a.ntaps_dense; ++i) {
            const double w = a.c[i];
            if (w == 0.0) continue;
            const int dx = i % W - R, dy = (i / W) % W - R, dz = a.ndim == 3 ? i / (W * W) - R : 0;
            taps[k] = (dz * SY + dy) * SX + dx;
            tw[k] = w;
            ++k;
        }
    }
    const long long ntile = (long long)SZ * SY * SX;
    for (long long i = threadIdx.x; i < ntile; i += NTF) {
        const int lx = (int)(i % SX);
        const int ly = (int)((i / SX) % SY);
        const int lz = (int)(i / ((long long)SX * SY));
        const long long gx = wrapl(x0 + lx - R, a.nx), gy = wrapl(y0 + ly - R, a.ny);
        const long long gz = a.ndim == 3 ? wrapl(z0 + lz - hz, a.nz) : 0;
        tile[i] = a.src[gz * a.src_pz + gy * a.src_py + gx];
    }
    __syncthreads();
    const int tx = threadIdx.x % FX, ty = threadIdx.x / FX;
    const long long X = x0 + tx, Y = y0 + ty;
    if (X >= a.nx || Y >= a.ny) return;
    for (int lz = 0; lz < tz; ++lz) {
        const long long Z = z0 + lz;
        if (Z >= a.nz) break;
        const double *centre = tile + ((lz + hz) * SY + (ty + R)) * SX + (tx + R);
        double acc = 0.0;
        for (int k = 0; k < a.nnz; ++k) acc = fma(tw[k], centre[taps[k]], acc);
        a.dst[Z * a.dst_pz + Y * a.dst_py + X] = acc;
    }
}

}  // namespace

size_t sweep_f64_smem_bytes(int ndim, int R, int tz, int nnz)
{
    const int SZ = ndim == 3 ? tz + 2 * R : 1;
    return sizeof(double) * (size_t)SZ * (FY + 2 * R) * (FX + 2 * R) +
           sizeof(int) * (size_t)((nnz + 1) & ~1) + sizeof(double) * (size_t)nnz;
}

cudaError_t launch_sweep_f64(const SweepF64Args &a, cudaStream_t s)
{
    cudaError_t e = smem_optin((const void *)k_sweep_f64);
    if (e != cudaSuccess) return e;
    const long long nb = (long long)a.bx * a.by * (a.ndim == 3 ? (a.nz + a.tz - 1) / a.tz : 1);
    const size_t smem = sweep_f64_smem_bytes(a.ndim, a.R, a.tz, a.nnz);
    k_sweep_f64<<<(unsigned)nb, NTF, smem, s>>>(a);
    return cudaGetLastError();
}

int sweep_f64_block_x() { return FX; }
int sweep_f64_block_y() { return FY; }

}  // namespace sg
