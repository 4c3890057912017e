// Time-loop driver of the 3D tensor-core path: floor(T/m) folded sweeps of a
// 3D stencil on tcgen05 (k_tc3d.cu, BF16 hi/lo split, FP32 accumulation),
// then T mod m plain CUDA-core steps, ping-ponging between the plan's padded
// grids and ending in `out`.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "plan.h"

namespace sg {

static stencil_status_t tc3d_panels(stencil_plan_s *p, int m, const uint16_t **out, double *sum)
{
    const int key = m + 256;  // the 2D kernels' panels use keys below 256
    auto it = p->panels.find(key);
    if (it == p->panels.end()) {
        const std::vector<double> *cm = nullptr;
        stencil_status_t st = plan_folded(p, m, &cm);
        if (st != STENCIL_OK) return st;
        const int R = m * p->r;
        std::vector<uint16_t> host(tc3d_panel_elems(R));
        const double wsum = tc3d_build_panels(cm->data(), R, host.data());
        uint16_t *d = nullptr;
        cudaError_t e = cudaMalloc(&d, host.size() * sizeof(uint16_t));
        if (e == cudaSuccess)
            e = cudaMemcpy(d, host.data(), host.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (d) cudaFree(d);
            return cuda_fail(e, "3D tensor-core panels");
        }
        p->scratch_bytes += host.size() * sizeof(uint16_t);
        it = p->panels.emplace(key, d).first;
        p->panel_sum[key] = wsum;
    }
    *out = it->second;
    *sum = p->panel_sum[key];
    return STENCIL_OK;
}

static stencil_status_t launch_tc3d_pass(stencil_plan_s *p, const Padded &src, int m,
                                         const uint16_t *panels, double sum_c, float *dst,
                                         int64_t dst_py, int64_t dst_pz, int dst_gw, bool dst_vec4,
                                         cudaStream_t s)
{
    const int R = m * p->r;
    TC3DArgs a3;
    memset(&a3, 0, sizeof(a3));
    TC2DArgs &a = a3.t;
    a.nx = p->nx;
    a.ny = p->ny;
    a.tiles_x = ceil_div(p->nx, kTcN);
    a3.tiles_y = ceil_div(p->ny, kTcM);
    a3.nz = p->nz;
    a.ntiles = a.tiles_x * a3.tiles_y * p->nz;
    a.R = R;
    tc3d_geometry(R, &a.rows, &a.rows_p, &a.box_w, &a.halo_x);
    a.terms = p->precision == STENCIL_PREC_BF16X1 ? 1 : 3;
    a.map_x0 = src.gx;
    a.map_y0 = src.gy;
    a3.map_z0 = src.gz;
    a.mean_sum = p->tc_center ? p->d_acc : nullptr;
    a.inv_n = 1.0 / ((double)p->nx * p->ny * p->nz);
    a.sum_c = (float)sum_c;
    a.panels = panels;
    a.dst = dst;
    a.dst_py = dst_py;
    a3.dst_pz = dst_pz;
    a.dst_gw = dst_gw;
    a.dst_vec4 = dst_vec4 ? 1 : 0;
    a.status = p->d_status;
    a.wait_ns = (unsigned long long)p->wait_ms * 1000000ull;
    a.fault_withhold_mma = p->fault_withhold_mma;
    const int box[3] = {a.box_w, a.rows, 1};
    const CUtensorMap *map = plan_map(p, src, box);
    if (!map) return STENCIL_ERR_CUDA;
    const int grid = std::min(a.ntiles, p->sm_count);
    cudaError_t e = launch_tc3d(*map, a3, grid, tc3d_smem_bytes(R), s);
    if (e != cudaSuccess) return cuda_fail(e, "3D tensor-core sweep launch");
    return STENCIL_OK;
}

stencil_status_t run3d_tc(stencil_plan_s *p, const float *in, float *out, int64_t T, int m,
                          cudaStream_t s)
{
    const int R = m * p->r;
    const int nmin = std::min(p->nx, std::min(p->ny, p->nz));
    if (2 * R + 1 > nmin || R > kGhost) {
        set_error("3D tensor-core sweep: folded width %d exceeds the grid", 2 * R + 1);
        return STENCIL_ERR_INVALID_ARG;
    }
    if (!tc3d_supported(R) || !sweep3d_supported(p->r, 1, p->pattern)) {
        set_error("3D tensor-core sweep: folded radius %d unsupported (1..%d)", R, kTc3MaxR);
        return STENCIL_ERR_UNSUPPORTED;
    }
    ensure_device_facts(p);
    if (tc3d_smem_bytes(R) > (size_t)p->max_smem) {
        set_error("3D tensor-core sweep: shared memory");
        return STENCIL_ERR_UNSUPPORTED;
    }
    const uint16_t *panels = nullptr;
    double sum_c = 0.0;
    const std::vector<double> *c1 = nullptr;
    stencil_status_t st = tc3d_panels(p, m, &panels, &sum_c);
    if (st == STENCIL_OK) st = plan_folded(p, 1, &c1);
    if (st == STENCIL_OK) st = ensure_padded(p);
    if (st != STENCIL_OK) return st;
    const int64_t q = T / m, rem = T % m;
    int gw = q ? R : 0;
    if (rem) gw = std::max(gw, p->r);
    const bool out_vec4 = grid_vec4(p, out);
    const int64_t npass = q + rem;  // the remainder runs as single plain sweeps

    auto enqueue = [&](cudaStream_t st_, int *nl) -> stencil_status_t {
        cudaError_t e = launch_import(p->A, in, gw, st_, p->pitch_y, p->pitch_z);
        if (e != cudaSuccess) return cuda_fail(e, "import launch");
        *nl += 1;
        if (p->tc_center && q > 0) {
            e = cudaMemsetAsync(p->d_acc, 0, sizeof(double), st_);
            if (e == cudaSuccess)
                e = launch_grid_sum(p->A.origin, p->nx, p->ny, p->nz, p->A.py, p->A.pz, p->d_acc,
                                    st_);
            if (e != cudaSuccess) return cuda_fail(e, "grid mean");
            *nl += 1;
        }
        const Padded *cur = &p->A, *oth = &p->B;
        for (int64_t i = 0; i < npass; ++i) {
            const bool last = i + 1 == npass;
            float *dst = last ? out : oth->origin;
            const int64_t dpy = last ? p->pitch_y : oth->py;
            const int64_t dpz = last ? p->pitch_z : oth->pz;
            stencil_status_t r =
                i < q ? launch_tc3d_pass(p, *cur, m, panels, sum_c, dst, dpy, dpz, last ? 0 : gw,
                                         last ? out_vec4 : true, st_)
                      : launch_pass3d(p, *cur, 1, 1, *c1, dst, dpy, dpz, last ? 0 : gw,
                                      last ? out_vec4 : true, st_);
            if (r != STENCIL_OK) return r;
            *nl += 1;
            std::swap(cur, oth);
        }
        return STENCIL_OK;
    };
    std::vector<int64_t> key = {7, (int64_t)(uintptr_t)in, (int64_t)(uintptr_t)out, T, m,
                                p->precision, p->tc_center, p->wait_ms, p->fault_withhold_mma};
    st = run_maybe_graph(p, key, s, enqueue);
    p->last_m = m;
    p->last_b = 1;
    p->last_engine = 1;
    p->last_tc_form = 1;
    return st;
}

}  // namespace sg
