// Centred storage of the FP32 CUDA-core runs.
//
// A run of T steps is linear, so it may advance x - mu instead of x and add
// mu * (sum c)^T back at the end, for any constant mu.  With mu the grid's
// mean, every FP32 sum of a sweep then rounds values near zero instead of
// values near mu: after diffusion the field is mu plus a small fluctuation,
// and rounding at the magnitude of mu (a few 1e-8 per operation) would
// otherwise act on that fluctuation sweep after sweep, with a bias that
// depends on the value and so accumulates.  The kernels here form the FP64
// sum of a grid (the mean's numerator) and add the final bias; the import
// kernels subtract mu.
#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace sg {
namespace {

__device__ __forceinline__ double warp_sum(double s)
{
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    return s;
}

// A lane's FP32 share of one row: 16-byte loads where the row allows them.
// The sum only fixes the centring constant, which is subtracted and added back
// unchanged, so the FP32 rounding of these partial sums does not reach the
// result; FP64 then gathers the rows.
__device__ __forceinline__ float row_share(const float *__restrict__ row, int nx, int lane)
{
    float fs = 0.f;
    int x0 = 0;
    if ((reinterpret_cast<uintptr_t>(row) & 15) == 0) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
        for (int i = lane; i < nx / 4; i += 32) {
            const float4 t = r4[i];
            fs += (t.x + t.y) + (t.z + t.w);
        }
        x0 = nx / 4 * 4;
    }
    for (int x = x0 + lane; x < nx; x += 32) fs += row[x];
    return fs;
}

// acc[0] += sum of the nx * ny * nz points (rows py, planes pz apart).
__global__ void k_sum_grid(const float *__restrict__ src, int nx, int ny, int nz, int64_t py,
                           int64_t pz, double *__restrict__ acc)
{
    double s = 0.0;
    const long long rows = (long long)ny * nz;
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows;
         r += nwarps)
        s += (double)row_share(src + (r / ny) * pz + (r % ny) * py, nx, lane);
    s = warp_sum(s);
    if (lane == 0) atomicAdd(acc, s);
}

__global__ void k_add_bias(float *__restrict__ dst, int nx, int ny, int nz, int64_t py, int64_t pz,
                           const double *__restrict__ mean_sum, double inv_n, double factor)
{
    const float mu = (float)(mean_sum[0] * inv_n);
    const float add = (float)((double)mu * factor);
    const long long rows = (long long)ny * nz;
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows;
         r += nwarps) {
        float *row = dst + (r / ny) * pz + (r % ny) * py;
        for (int x = lane; x < nx; x += 32) row[x] += add;
    }
}

// The job of a row of a batch's row space (the import's padded rows; only the
// interior rows y in [0, ny) are visited).
__device__ __forceinline__ int job_of(const ImportJob *__restrict__ jobs, int njobs, long long row)
{
    int lo = 0, hi = njobs - 1;  // last job with row0 <= row
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].row0 <= row) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_sum_batch(const ImportJob *__restrict__ jobs, int njobs, long long rows)
{
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long row = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); row < rows;
         row += nwarps) {
        const ImportJob &J = jobs[job_of(jobs, njobs, row)];
        const int y = (int)(row - J.row0) - J.gw;
        if (y < 0 || y >= J.ny || !J.mean_sum) continue;
        double s = (double)row_share(J.src + y * J.src_py, J.nx, lane);
        s = warp_sum(s);
        if (lane == 0) atomicAdd(J.mean_sum, s);
    }
}

__global__ void k_add_bias_batch(const ImportJob *__restrict__ jobs, int njobs, long long rows)
{
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long row = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); row < rows;
         row += nwarps) {
        const ImportJob &J = jobs[job_of(jobs, njobs, row)];
        const int y = (int)(row - J.row0) - J.gw;
        if (y < 0 || y >= J.ny || !J.mean_sum) continue;
        const float mu = (float)(J.mean_sum[0] * J.inv_n);
        const float add = (float)((double)mu * J.factor);
        float *orow = J.out + y * J.out_py;
        for (int x = lane; x < J.nx; x += 32) orow[x] += add;
    }
}

int grid_for_rows(long long rows)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (rows + 7) / 8;  // eight warps per CTA, one row each
    return (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * 8));
}

}  // namespace

cudaError_t launch_grid_sum(const float *src, int nx, int ny, int nz, int64_t py, int64_t pz,
                            double *acc, cudaStream_t s)
{
    k_sum_grid<<<grid_for_rows((long long)ny * nz), 256, 0, s>>>(src, nx, ny, nz, py, pz, acc);
    return cudaGetLastError();
}

cudaError_t launch_add_bias(float *dst, int nx, int ny, int nz, int64_t py, int64_t pz,
                            const double *mean_sum, double inv_n, double factor, cudaStream_t s)
{
    k_add_bias<<<grid_for_rows((long long)ny * nz), 256, 0, s>>>(dst, nx, ny, nz, py, pz,
                                                                mean_sum, inv_n, factor);
    return cudaGetLastError();
}

cudaError_t launch_grid_sum_batch(const ImportJob *d_jobs, int njobs, long long rows,
                                  cudaStream_t s)
{
    if (njobs == 0 || rows == 0) return cudaSuccess;
    k_sum_batch<<<grid_for_rows(rows), 256, 0, s>>>(d_jobs, njobs, rows);
    return cudaGetLastError();
}

cudaError_t launch_add_bias_batch(const ImportJob *d_jobs, int njobs, long long rows,
                                  cudaStream_t s)
{
    if (njobs == 0 || rows == 0) return cudaSuccess;
    k_add_bias_batch<<<grid_for_rows(rows), 256, 0, s>>>(d_jobs, njobs, rows);
    return cudaGetLastError();
}

}  // namespace sg
