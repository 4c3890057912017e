// Support kernels: dense <-> padded layout conversion, the FP64 folded-weight
// builder (the m-fold convolution power of Section 3.2), the FP64 relative-L2
// reduction, the grid mean used by the tensor-core path, and tensor-map
// encoding.
#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace sg {
namespace {

__device__ __forceinline__ int wrap_idx(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// dst (padded, ghost band gw) <- src (rows src_py, planes src_pz elements
// apart).  One CTA per padded row
// (z, y): the wrapped source row is found once, the interior is copied with
// 16-byte accesses when the rows allow it, and the 2*gwx ghost columns of the
// row are copied element by element.
__global__ void k_import(float *__restrict__ origin, int64_t py, int64_t pz, int nx, int ny,
                         int nz, int gwx, int gwy, int gwz, const float *__restrict__ src,
                         int64_t src_py, int64_t src_pz, int vec4,
                         const double *__restrict__ mean_sum, double inv_n)
{
    const int wy = ny + 2 * gwy, wz = nz + 2 * gwz;
    // centred storage: every value minus the grid mean, rounded to FP32 once
    const float mu = mean_sum ? (float)(mean_sum[0] * inv_n) : 0.f;
    for (long long row = blockIdx.x; row < (long long)wy * wz; row += gridDim.x) {
        const int y = (int)(row % wy) - gwy;
        const int z = (int)(row / wy) - gwz;
        const int sy = wrap_idx(y, ny), sz = wrap_idx(z, nz);
        const float *srow = src + sz * src_pz + sy * src_py;
        float *drow = origin + z * pz + y * py;
        if (vec4) {
            const float4 *s4 = reinterpret_cast<const float4 *>(srow);
            float4 *d4 = reinterpret_cast<float4 *>(drow);
            for (int i = threadIdx.x; i < nx / 4; i += blockDim.x) {
                const float4 v = s4[i];
                d4[i] = make_float4(v.x - mu, v.y - mu, v.z - mu, v.w - mu);
            }
        } else {
            for (int i = threadIdx.x; i < nx; i += blockDim.x) drow[i] = srow[i] - mu;
        }
        for (int i = threadIdx.x; i < 2 * gwx; i += blockDim.x) {
            const int x = i < gwx ? i - gwx : nx + (i - gwx);
            drow[x] = srow[wrap_idx(x, nx)] - mu;
        }
    }
}

// The imports of a whole batch of 2D grids in one launch: one warp per padded
// row, the row's grid found by binary search over the jobs' first rows.
__global__ void k_import_batch(const ImportJob *__restrict__ jobs, int njobs, long long rows)
{
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long row = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); row < rows;
         row += nwarps) {
        int lo = 0, hi = njobs - 1;  // last job with row0 <= row
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].row0 <= row) lo = mid;
            else hi = mid - 1;
        }
        const ImportJob &J = jobs[lo];
        const int y = (int)(row - J.row0) - J.gw;
        const float *srow = J.src + wrap_idx(y, J.ny) * J.src_py;
        float *drow = J.origin + y * J.py;
        const float mu = J.mean_sum ? (float)(J.mean_sum[0] * J.inv_n) : 0.f;
        if (J.vec4) {
            const float4 *s4 = reinterpret_cast<const float4 *>(srow);
            float4 *d4 = reinterpret_cast<float4 *>(drow);
            for (int i = lane; i < J.nx / 4; i += 32) {
                const float4 v = s4[i];
                d4[i] = make_float4(v.x - mu, v.y - mu, v.z - mu, v.w - mu);
            }
        } else {
            for (int i = lane; i < J.nx; i += 32) drow[i] = srow[i] - mu;
        }
        for (int i = lane; i < 2 * J.gw; i += 32) {
            const int x = i < J.gw ? i - J.gw : J.nx + (i - J.gw);
            drow[x] = srow[wrap_idx(x, J.nx)] - mu;
        }
    }
}

__global__ void k_export(const float *__restrict__ origin, int64_t py, int64_t pz, int nx, int ny,
                         int nz, float *__restrict__ dst)
{
    const long long total = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long r = i / nx;
        const int y = (int)(r % ny);
        const int z = (int)(r / ny);
        dst[i] = origin[z * pz + y * py + x];
    }
}

// out = c^(m): starting from c, m-1 full convolutions with c, all in FP64.
// One CTA; the intermediate arrays live in `work`.
__global__ void k_fold_power(int ndim, int r, int m, const double *__restrict__ c,
                             double *__restrict__ out, double *__restrict__ work)
{
    const int wc = 2 * r + 1;
    const int wmax = 2 * m * r + 1;
    int wlen = 1;
    for (int d = 0; d < ndim; ++d) wlen *= wmax;
    double *cur = work, *nxt = work + wlen;
    // cur <- c (width wc)
    int ncur = 1;
    for (int d = 0; d < ndim; ++d) ncur *= wc;
    for (int i = threadIdx.x; i < ncur; i += blockDim.x) cur[i] = c[i];
    __syncthreads();
    int wcur = wc;
    for (int step = 1; step < m; ++step) {
        const int wn = wcur + wc - 1;
        int nn = 1;
        for (int d = 0; d < ndim; ++d) nn *= wn;
        for (int i = threadIdx.x; i < nn; i += blockDim.x) {
            // output index p (offsets from the corner) = q + s, q in c, s in cur
            int p[3] = {0, 0, 0};
            int t = i;
            for (int d = ndim - 1; d >= 0; --d) { p[d] = t % wn; t /= wn; }
            double acc = 0.0;
            int nq = 1;
            for (int d = 0; d < ndim; ++d) nq *= wc;
            for (int q = 0; q < nq; ++q) {
                int qi[3] = {0, 0, 0};
                int tq = q;
                for (int d = ndim - 1; d >= 0; --d) { qi[d] = tq % wc; tq /= wc; }
                int sidx = 0;
                bool ok = true;
                for (int d = 0; d < ndim; ++d) {
                    const int s = p[d] - qi[d];
                    if (s < 0 || s >= wcur) { ok = false; break; }
                    sidx = sidx * wcur + s;
                }
                if (ok) acc += c[q] * cur[sidx];
            }
            nxt[i] = acc;
        }
        __syncthreads();
        double *tmp = cur; cur = nxt; nxt = tmp;
        wcur = wn;
    }
    int nout = 1;
    for (int d = 0; d < ndim; ++d) nout *= wcur;
    for (int i = threadIdx.x; i < nout; i += blockDim.x) out[i] = cur[i];
}

template <typename T>
__global__ void k_rel_l2(const T *__restrict__ y, const double *__restrict__ ref, long long n,
                         double *__restrict__ acc)
{
    double e2 = 0.0, r2 = 0.0, sy = 0.0, sr = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double yv = (double)y[i], rv = ref[i], d = yv - rv;
        e2 += d * d;
        r2 += rv * rv;
        sy += yv;
        sr += rv;
    }
    __shared__ double red[4][32];
    double v[4] = {e2, r2, sy, sr};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double t = v[k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = t;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double t = threadIdx.x < nw ? red[k][threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (threadIdx.x == 0) atomicAdd(&acc[k], t);
        }
    }
}

__global__ void k_grid_sum(const float *__restrict__ origin, int nx, int ny, int64_t py,
                           double *__restrict__ acc)
{
    double s = 0.0;
    const long long total = (long long)nx * ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), yy = (int)(i / nx);
        s += (double)origin[yy * py + x];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

cudaError_t launch_import(const Padded &P, const float *src, int gw, cudaStream_t s,
                          int64_t src_py, int64_t src_pz, const double *mean_sum, double inv_n)
{
    const int gwx = gw, gwy = P.ndim >= 2 ? gw : 0, gwz = P.ndim >= 3 ? gw : 0;
    if (src_py <= 0) src_py = P.nx;
    if (src_pz <= 0) src_pz = src_py * P.ny;
    // 16-byte interior copies need 16-byte aligned rows on both sides
    const int vec4 = (P.nx % 4 == 0) && ((uintptr_t)src % 16 == 0) && (P.py % 4 == 0) &&
                     ((uintptr_t)P.origin % 16 == 0) && (src_py % 4 == 0) &&
                     (P.ndim < 3 || src_pz % 4 == 0);
    const long long rows = (long long)(P.ny + 2 * gwy) * (P.nz + 2 * gwz);
    const int grid = (int)std::min<long long>(rows, (long long)sm_count() * 16);
    k_import<<<grid, 256, 0, s>>>(P.origin, P.py, P.pz, P.nx, P.ny, P.nz, gwx, gwy, gwz, src,
                                  src_py, src_pz, vec4, mean_sum, inv_n);
    return cudaGetLastError();
}

ImportJob make_import_job(const Padded &P, const float *src, int gw, long long row0,
                          int64_t src_py)
{
    ImportJob j;
    j.origin = P.origin;
    j.py = P.py;
    j.src = src;
    j.src_py = src_py > 0 ? src_py : P.nx;
    j.mean_sum = nullptr;
    j.inv_n = 0.0;
    j.out = nullptr;
    j.out_py = 0;
    j.factor = 1.0;
    j.row0 = row0;
    j.nx = P.nx;
    j.ny = P.ny;
    j.gw = gw;
    j.vec4 = (P.nx % 4 == 0) && ((uintptr_t)src % 16 == 0) && (P.py % 4 == 0) &&
             ((uintptr_t)P.origin % 16 == 0) && (j.src_py % 4 == 0);
    return j;
}

cudaError_t launch_import_batch(const ImportJob *d_jobs, int njobs, long long rows, cudaStream_t s)
{
    if (njobs == 0 || rows == 0) return cudaSuccess;
    const int grid = (int)std::min<long long>((rows + 7) / 8, (long long)sm_count() * 16);
    k_import_batch<<<grid, 256, 0, s>>>(d_jobs, njobs, rows);
    return cudaGetLastError();
}

cudaError_t launch_export(const Padded &P, float *dst, cudaStream_t s)
{
    k_export<<<sm_count() * 8, 256, 0, s>>>(P.origin, P.py, P.pz, P.nx, P.ny, P.nz, dst);
    return cudaGetLastError();
}

cudaError_t launch_fold_power(int ndim, int r, int m, const double *d_c, double *d_out,
                              double *d_work, cudaStream_t s)
{
    k_fold_power<<<1, 256, 0, s>>>(ndim, r, m, d_c, d_out, d_work);
    return cudaGetLastError();
}

cudaError_t launch_rel_l2(const void *y, bool y_f64, const double *ref, long long n, double *acc,
                          cudaStream_t s)
{
    const int grid = sm_count() * 4;
    if (y_f64)
        k_rel_l2<double><<<grid, 256, 0, s>>>(static_cast<const double *>(y), ref, n, acc);
    else
        k_rel_l2<float><<<grid, 256, 0, s>>>(static_cast<const float *>(y), ref, n, acc);
    return cudaGetLastError();
}

cudaError_t launch_grid_mean(const float *origin, int nx, int ny, int64_t py, double *acc,
                             cudaStream_t s)
{
    k_grid_sum<<<sm_count() * 4, 256, 0, s>>>(origin, nx, ny, py, acc);
    return cudaGetLastError();
}

// ---- tensor maps ---------------------------------------------------------

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}
}  // namespace

bool encode_store_map_2d(CUtensorMap *map, float *base, int nx, int ny, int64_t pitch, int box_x,
                         int box_y)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    if (((uintptr_t)base % 16) != 0 || (pitch * 4) % 16 != 0) return false;
    cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
    cuuint32_t bx[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y}, es[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, bx, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_padded_map(CUtensorMap *map, const Padded &P, const int *box)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3], strides[2];
    cuuint32_t bx[3], es[3] = {1, 1, 1};
    const int rank = P.ndim;
    dims[0] = (cuuint64_t)P.py;
    bx[0] = (cuuint32_t)box[0];
    if (rank >= 2) {
        dims[1] = (cuuint64_t)(P.ny + 2 * P.gy);
        strides[0] = (cuuint64_t)P.py * 4;
        bx[1] = (cuuint32_t)box[1];
    }
    if (rank >= 3) {
        dims[2] = (cuuint64_t)(P.nz + 2 * P.gz);
        strides[1] = (cuuint64_t)P.pz * 4;
        bx[2] = (cuuint32_t)box[2];
    }
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, P.alloc, dims, strides,
                    bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace sg
