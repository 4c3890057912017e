// Time-loop driver of FP64 2D and 3D grids: floor(T/m) sweeps of the FP64
// folded weights c^(m) (Section 3.2) then T mod m plain sweeps, alternating
// between two plan-owned buffers in the caller's layout; the last sweep
// writes `out`.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "plan.h"

namespace sg {

stencil_status_t run_f64nd(stencil_plan_s *p, const double *in, double *out, int64_t T, int m,
                           cudaStream_t s)
{
    if (m == 0) {
        if (p->tuned_m == 0 && p->autotune) {
            stencil_status_t st = autotune2d(p, s);
            if (st != STENCIL_OK) return st;
        }
        m = p->tuned_m > 0 ? p->tuned_m : 1;
    }
    const int R = m * p->r;
    const int rmax = p->ndim == 3 ? kMaxRF64_3D : kMaxRF64_2D;
    const int nmin = std::min(p->nx, p->ndim == 3 ? std::min(p->ny, p->nz) : p->ny);
    if (2 * R + 1 > nmin) {
        set_error("FP64 sweep: folded width %d exceeds the grid", 2 * R + 1);
        return STENCIL_ERR_INVALID_ARG;
    }
    if (R > rmax) {
        set_error("FP64 sweep: folded radius %d above %d", R, rmax);
        return STENCIL_ERR_UNSUPPORTED;
    }
    const std::vector<double> *cm = nullptr, *c1 = nullptr;
    stencil_status_t st = plan_folded(p, m, &cm);
    if (st == STENCIL_OK) st = plan_folded(p, 1, &c1);
    if (st != STENCIL_OK) return st;
    const size_t bytes = sizeof(double) * grid_extent(p);
    if (!p->d1a) {
        cudaError_t e = cudaMalloc(&p->d1a, bytes);
        if (e == cudaSuccess) e = cudaMalloc(&p->d1b, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "FP64 scratch");
        p->scratch_bytes += 2 * bytes;
    }
    ensure_device_facts(p);
    std::vector<int> ms;  // fold of each sweep
    for (int64_t i = 0; i < T / m; ++i) ms.push_back(m);
    for (int64_t i = 0; i < T % m; ++i) ms.push_back(1);

    auto args_for = [&](int mm, const double *src, double *dst) {
        SweepF64Args a;
        const std::vector<double> &c = mm == m ? *cm : *c1;
        a.src = src;
        a.dst = dst;
        a.nx = p->nx;
        a.ny = p->ny;
        a.nz = p->nz;
        a.src_py = a.dst_py = p->pitch_y;
        a.src_pz = a.dst_pz = p->pitch_z;
        a.ndim = p->ndim;
        a.R = mm * p->r;
        a.tz = p->ndim == 3 ? 4 : 1;
        a.bx = ceil_div(p->nx, sweep_f64_block_x());
        a.by = ceil_div(p->ny, sweep_f64_block_y());
        a.ntaps_dense = (int)c.size();
        a.nnz = 0;
        for (size_t k = 0; k < c.size(); ++k) {
            a.c[k] = c[k];
            a.nnz += c[k] != 0.0;
        }
        return a;
    };
    auto enqueue = [&](cudaStream_t st_, int *nl) -> stencil_status_t {
        const double *src = in;
        if (in == out && ms.size() == 1) {
            // one sweep cannot read and write the same grid: go through a buffer
            cudaError_t e = copy_grid(p, p->d1b, in, cudaMemcpyDeviceToDevice, st_);
            if (e != cudaSuccess) return cuda_fail(e, "FP64 alias copy");
            src = static_cast<const double *>(p->d1b);
        }
        double *bufs[2] = {static_cast<double *>(p->d1a), static_cast<double *>(p->d1b)};
        int nb = 0;
        for (size_t i = 0; i < ms.size(); ++i) {
            const bool last = i + 1 == ms.size();
            double *dst = last ? out : bufs[nb];
            if (!last && dst == src) dst = bufs[nb ^ 1];
            const SweepF64Args a = args_for(ms[i], src, dst);
            cudaError_t e = launch_sweep_f64(a, st_);
            if (e != cudaSuccess) return cuda_fail(e, "FP64 sweep launch");
            *nl += 1;
            src = dst;
            nb ^= 1;
        }
        return STENCIL_OK;
    };
    std::vector<int64_t> key = {6, (int64_t)(uintptr_t)in, (int64_t)(uintptr_t)out, T, m};
    st = run_maybe_graph(p, key, s, enqueue);
    p->last_m = m;
    p->last_b = 1;
    p->last_engine = 0;
    return st;
}

}  // namespace sg
