// Time-loop driver of the tensor-core path: floor(T/m) folded sweeps of a 2D
// box stencil on tcgen05 (BF16 hi/lo split, FP32 accumulation), then T mod m
// plain CUDA-core steps (Section 3.4: the skipped intermediate steps).
#include <cuda_runtime.h>

#include <string.h>

#include <algorithm>
#include <vector>

#include "plan.h"

namespace sg {

// Toeplitz panels of c^(m) for the per-offset or the grouped tensor-core
// kernel, built once per plan.
static stencil_status_t tc_panels(stencil_plan_s *p, int m, bool grouped, bool tf32,
                                  const uint16_t **out, double *sum)
{
    const int key = grouped ? m + 64 : (tf32 ? m + 128 : m);
    auto it = p->panels.find(key);
    if (it == p->panels.end()) {
        const std::vector<double> *cm = nullptr;
        stencil_status_t st = plan_folded(p, m, &cm);
        if (st != STENCIL_OK) return st;
        const int R = m * p->r;
        std::vector<uint16_t> host(grouped ? tc2dg_panel_elems(R) : tc2d_panel_bytes(R, tf32) / 2);
        const double wsum = grouped ? tc2dg_build_panels(cm->data(), R, host.data())
                                    : tc2d_build_panels(cm->data(), R, host.data(), tf32);
        uint16_t *d = nullptr;
        cudaError_t e = cudaMalloc(&d, host.size() * sizeof(uint16_t));
        if (e == cudaSuccess)
            e = cudaMemcpy(d, host.data(), host.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (d) cudaFree(d);
            return cuda_fail(e, "tensor-core panels");
        }
        p->scratch_bytes += host.size() * sizeof(uint16_t);
        it = p->panels.emplace(key, d).first;
        p->panel_sum[key] = wsum;
    }
    *out = it->second;
    *sum = p->panel_sum[key];
    return STENCIL_OK;
}

// One pass of the grouped tensor-core kernel (k_tc2d_grouped.cu).
static stencil_status_t launch_tc_grouped_pass(stencil_plan_s *p, const Padded &src, int m,
                                               const uint16_t *panels, double sum_c, float *dst,
                                               int64_t dst_py, int dst_gw, bool dst_vec4,
                                               cudaStream_t s)
{
    const int R = m * p->r;
    TC2DArgs a;
    memset(&a, 0, sizeof(a));
    a.nx = p->nx;
    a.ny = p->ny;
    a.tiles_x = ceil_div(p->nx, kTcN);
    a.ntiles = a.tiles_x * ceil_div(p->ny, kTcOutRows);
    a.R = R;
    tc2dg_geometry(R, &a.rows, &a.rows_p, &a.box_w, &a.halo_x);
    a.terms = p->precision == STENCIL_PREC_BF16X1 ? 1 : 3;
    a.map_x0 = src.gx;
    a.map_y0 = src.gy;
    a.mean_sum = p->tc_center ? p->d_acc : nullptr;
    a.inv_n = 1.0 / ((double)p->nx * p->ny);
    a.sum_c = (float)sum_c;
    a.panels = panels;
    a.dst = dst;
    a.dst_py = dst_py;
    a.dst_gw = dst_gw;
    a.dst_vec4 = dst_vec4 ? 1 : 0;
    a.status = p->d_status;
    a.wait_ns = (unsigned long long)p->wait_ms * 1000000ull;
    a.fault_withhold_mma = p->fault_withhold_mma;
    const int box[2] = {a.box_w, a.rows};
    const CUtensorMap *map = plan_map(p, src, box);
    if (!map) return STENCIL_ERR_CUDA;
    // two FP32 staging slots when they fit, else one: the converters empty a
    // slot long before the tile's MMAs finish
    a.nstage = tc2dg_smem_bytes(R, 2) <= (size_t)p->max_smem ? 2 : 1;
    const int grid = std::min(a.ntiles, p->sm_count);
    cudaError_t e = launch_tc2dg(*map, a, grid, tc2dg_smem_bytes(R, a.nstage), s);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core sweep launch");
    return STENCIL_OK;
}

static stencil_status_t launch_tc_pass(stencil_plan_s *p, const Padded &src, int m,
                                       const uint16_t *panels, double sum_c, float *dst,
                                       int64_t dst_py, int dst_gw, bool dst_vec4, cudaStream_t s)
{
    const int R = m * p->r;
    TC2DArgs a;
    memset(&a, 0, sizeof(a));
    a.nx = p->nx;
    a.ny = p->ny;
    a.tiles_x = ceil_div(p->nx, kTcN);
    a.tiles_y = ceil_div(p->ny, kTcM);
    a.ntiles = a.tiles_x * a.tiles_y;
    a.nplanes = 1;
    a.R = R;
    a.halo_x = round_up(R, 4);
    a.rows = kTcM + 2 * R;
    a.rows_p = a.rows | 1;
    a.box_w = round_up(kTcK + a.halo_x - R, 4);
    a.terms = p->precision == STENCIL_PREC_BF16X1 ? 1 : 3;
    a.map_x0 = src.gx;
    a.map_y0 = src.gy;
    a.mean_sum = p->tc_center ? p->d_acc : nullptr;
    a.inv_n = 1.0 / ((double)p->nx * p->ny);
    a.sum_c = (float)sum_c;
    a.panels = panels;
    a.dst = dst;
    a.dst_py = dst_py;
    a.dst_gw = dst_gw;
    a.dst_vec4 = dst_vec4 ? 1 : 0;
    a.status = p->d_status;
    a.wait_ns = (unsigned long long)p->wait_ms * 1000000ull;
    a.fault_withhold_mma = p->fault_withhold_mma;
    const bool tf32 = p->precision == STENCIL_PREC_TF32X3;
    const int box[2] = {a.box_w, a.rows};
    const CUtensorMap *map = plan_map(p, src, box);
    if (!map) return STENCIL_ERR_CUDA;
    // the output leaves by TMA store when the tile buffer fits and the
    // destination rows are 16-byte aligned; otherwise by direct stores
    CUtensorMap dmap;
    memset(&dmap, 0, sizeof(dmap));
    a.tma_store = 0;
    if (p->tc_tma_store && tc2d_smem_bytes(R, true, tf32) <= (size_t)p->max_smem &&
        encode_store_map_2d(&dmap, dst, p->nx, p->ny, dst_py, kTcN, kTcM))
        a.tma_store = 1;
    const size_t smem = tc2d_smem_bytes(R, a.tma_store != 0, tf32);
    const int grid = std::min(a.ntiles, p->sm_count);
    cudaError_t e = launch_tc2d(*map, dmap, a, grid, smem, s, tf32);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core sweep launch");
    return STENCIL_OK;
}

// ---- 3D: the folded weights plane by plane (Section 3.3 treats a 3D grid as
// a stack of 2D slices).  c^(m) splits into its 2R+1 plane slices c_dz, and
// one folded sweep is
//   out[z] = sum_dz S_dz(in[z + dz]),
// S_dz the 2D folded sweep with the weights c_dz.  Each term is one launch of
// the per-offset tensor-core kernel over every plane at once (the padded 3D
// grid seen as one tall 2D array), each tile reading the plane dz away from
// the plane it writes; the first term stores and the others add.  The terms
// carry centred values; the last adds mu * sum(c^(m)) once.

// Toeplitz panels of the plane slices of c^(m), built once per plan; sums[i]
// is the FP64 sum of slice i.
static stencil_status_t tc_panels_3d(stencil_plan_s *p, int m, bool tf32,
                                     std::vector<const uint16_t *> &panels,
                                     std::vector<double> &sums)
{
    const std::vector<double> *cm = nullptr;
    stencil_status_t st = plan_folded(p, m, &cm);
    if (st != STENCIL_OK) return st;
    const int R = m * p->r, W = 2 * R + 1;
    panels.assign(W, nullptr);
    sums.assign(W, 0.0);
    for (int i = 0; i < W; ++i) {
        const int key = 4096 + (tf32 ? 2048 : 0) + m * 64 + i;
        auto it = p->panels.find(key);
        if (it == p->panels.end()) {
            std::vector<uint16_t> host(tc2d_panel_bytes(R, tf32) / 2);
            const double wsum =
                tc2d_build_panels(cm->data() + (size_t)i * W * W, R, host.data(), tf32);
            uint16_t *d = nullptr;
            cudaError_t e = cudaMalloc(&d, host.size() * sizeof(uint16_t));
            if (e == cudaSuccess)
                e = cudaMemcpy(d, host.data(), host.size() * sizeof(uint16_t),
                               cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                if (d) cudaFree(d);
                return cuda_fail(e, "tensor-core panels");
            }
            p->scratch_bytes += host.size() * sizeof(uint16_t);
            it = p->panels.emplace(key, d).first;
            p->panel_sum[key] = wsum;
        }
        panels[i] = it->second;
        sums[i] = p->panel_sum[key];
    }
    return STENCIL_OK;
}

// One term (plane offset dz) of a 3D tensor-core sweep from the padded grid
// src into the caller-layout grid dst.  sum_c: mu * sum_c is added (the last
// term passes the whole sum of c^(m), the others 0).
static stencil_status_t launch_tc3d_term(stencil_plan_s *p, const Padded &src, int m, int dz,
                                         const uint16_t *panels, double sum_c, bool accumulate,
                                         float *dst, bool dst_vec4, cudaStream_t s)
{
    const int R = m * p->r;
    TC2DArgs a;
    memset(&a, 0, sizeof(a));
    a.nx = p->nx;
    a.ny = p->ny;
    a.tiles_x = ceil_div(p->nx, kTcN);
    a.tiles_y = ceil_div(p->ny, kTcM);
    a.nplanes = p->nz;
    a.ntiles = a.tiles_x * a.tiles_y * a.nplanes;
    a.R = R;
    a.halo_x = round_up(R, 4);
    a.rows = kTcM + 2 * R;
    a.rows_p = a.rows | 1;
    a.box_w = round_up(kTcK + a.halo_x - R, 4);
    a.terms = p->precision == STENCIL_PREC_BF16X1 ? 1 : 3;
    // the padded grid as one 2D array of (nz + 2g)(ny + 2g) rows
    Padded flat = src;
    flat.ndim = 2;
    flat.ny = (src.nz + 2 * src.gz) * (src.ny + 2 * src.gy);
    flat.gy = 0;
    flat.nz = 1;
    flat.gz = 0;
    a.src_plane_rows = src.ny + 2 * src.gy;
    a.map_x0 = src.gx;
    a.map_y0 = (int)(src.gz * a.src_plane_rows + src.gy);
    a.dz = dz;
    a.mean_sum = p->tc_center ? p->d_acc : nullptr;
    a.inv_n = 1.0 / ((double)p->nx * p->ny * p->nz);
    a.sum_c = (float)sum_c;
    a.panels = panels;
    a.dst = dst;
    a.dst_py = p->pitch_y;
    a.dst_pz = p->pitch_z;
    a.dst_gw = 0;
    a.dst_vec4 = dst_vec4 ? 1 : 0;
    a.accumulate = accumulate ? 1 : 0;
    a.tma_store = 0;
    a.status = p->d_status;
    a.wait_ns = (unsigned long long)p->wait_ms * 1000000ull;
    a.fault_withhold_mma = p->fault_withhold_mma;
    const bool tf32 = p->precision == STENCIL_PREC_TF32X3;
    const int box[2] = {a.box_w, a.rows};
    const CUtensorMap *map = plan_map(p, flat, box);
    if (!map) return STENCIL_ERR_CUDA;
    CUtensorMap dmap;
    memset(&dmap, 0, sizeof(dmap));
    const size_t smem = tc2d_smem_bytes(R, false, tf32);
    const int grid = std::min(a.ntiles, p->sm_count);
    cudaError_t e = launch_tc2d(*map, dmap, a, grid, smem, s, tf32);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core 3D sweep launch");
    return STENCIL_OK;
}

stencil_status_t run3d_tc(stencil_plan_s *p, const float *in, float *out, int64_t T, int m,
                          cudaStream_t s)
{
    const int R = m * p->r;
    const int nmin = std::min(p->nx, std::min(p->ny, p->nz));
    if (2 * R + 1 > nmin || R > kGhost) {
        set_error("tensor-core 3D sweep: folded width %d exceeds the grid", 2 * R + 1);
        return STENCIL_ERR_INVALID_ARG;
    }
    const bool tf32 = p->precision == STENCIL_PREC_TF32X3;
    if (!(tf32 ? tc2d_tf32_supported(R) : tc2d_supported(R)) ||
        !sweep3d_supported(p->r, 1, p->pattern)) {
        set_error("tensor-core 3D sweep: folded radius %d unsupported (1..%d)", R,
                  tf32 ? kTcMaxRTf32 : kTcMaxR);
        return STENCIL_ERR_UNSUPPORTED;
    }
    ensure_device_facts(p);
    if (tc2d_smem_bytes(R, false, tf32) > (size_t)p->max_smem) {
        set_error("tensor-core 3D sweep: shared memory");
        return STENCIL_ERR_UNSUPPORTED;
    }
    std::vector<const uint16_t *> panels;
    std::vector<double> sums;
    const std::vector<double> *c1 = nullptr;
    stencil_status_t st = tc_panels_3d(p, m, tf32, panels, sums);
    if (st == STENCIL_OK) st = plan_folded(p, 1, &c1);
    if (st == STENCIL_OK) st = ensure_padded(p);
    if (st != STENCIL_OK) return st;
    double total = 0.0;
    for (double v : sums) total += v;
    const int64_t q = T / m, rem = T % m;
    // the T mod m plain steps: fused pairs where the kernel has them
    std::vector<int> plain;
    const int b1 = (sweep3d_tb_supported(p->r, 1, p->pattern) && 2 * p->r <= std::min(kGhost, nmin))
                       ? 2 : 1;
    for (int64_t d = 0; d < rem; d += b1) plain.push_back((int)std::min<int64_t>(b1, rem - d));
    int gw = std::max(p->r, q ? R : 0);
    for (int b : plain) gw = std::max(gw, b * p->r);
    const bool out_vec4 = grid_vec4(p, out);
    const int64_t npass = q + (int64_t)plain.size();
    auto enqueue = [&](cudaStream_t st_, int *nl) -> stencil_status_t {
        cudaError_t e = cudaSuccess;
        if (p->tc_center && q > 0) {
            e = cudaMemsetAsync(p->d_acc, 0, sizeof(double), st_);
            if (e == cudaSuccess)
                e = launch_grid_sum(in, p->nx, p->ny, p->nz, p->pitch_y, p->pitch_z, p->d_acc, st_);
            if (e != cudaSuccess) return cuda_fail(e, "grid sum launch");
            *nl += 1;
        }
        e = launch_import(p->A, in, gw, st_, p->pitch_y, p->pitch_z);
        if (e != cudaSuccess) return cuda_fail(e, "import launch");
        *nl += 1;
        const Padded *cur = &p->A, *oth = &p->B;
        int64_t done = 0;
        for (int64_t i = 0; i < q; ++i, ++done) {
            // the terms build the sweep's result in the caller's output grid,
            // which the next pass (if any) re-imports with its ghost band
            for (int dz = -R; dz <= R; ++dz) {
                stencil_status_t r =
                    launch_tc3d_term(p, *cur, m, dz, panels[dz + R], dz == R ? total : 0.0,
                                     dz > -R, out, out_vec4, st_);
                if (r != STENCIL_OK) return r;
                *nl += 1;
            }
            if (done + 1 < npass) {
                e = launch_import(*oth, out, gw, st_, p->pitch_y, p->pitch_z);
                if (e != cudaSuccess) return cuda_fail(e, "import launch");
                *nl += 1;
                std::swap(cur, oth);
            }
        }
        for (int b : plain) {
            const bool last = done + 1 == npass;
            stencil_status_t r = launch_pass3d(p, *cur, 1, b, *c1, last ? out : oth->origin,
                                               last ? p->pitch_y : oth->py,
                                               last ? p->pitch_z : oth->pz, last ? 0 : gw,
                                               last ? out_vec4 : true, st_);
            if (r != STENCIL_OK) return r;
            *nl += 1;
            ++done;
            std::swap(cur, oth);
        }
        return STENCIL_OK;
    };
    std::vector<int64_t> key = {6, (int64_t)(uintptr_t)in, (int64_t)(uintptr_t)out, T, m,
                                p->precision, p->tc_center, p->wait_ms, p->fault_withhold_mma};
    st = run_maybe_graph(p, key, s, enqueue);
    p->last_m = m;
    p->last_b = 1;
    p->last_engine = 1;
    p->last_tc_form = 1;
    return st;
}

stencil_status_t run2d_tc(stencil_plan_s *p, const float *in, float *out, int64_t T, int m,
                          cudaStream_t s)
{
    const int R = m * p->r;
    const int nmin = std::min(p->nx, p->ny);
    if (2 * R + 1 > nmin) {
        set_error("tensor-core sweep: folded width %d exceeds the grid", 2 * R + 1);
        return STENCIL_ERR_INVALID_ARG;
    }
    const bool tf32 = p->precision == STENCIL_PREC_TF32X3;
    if (!(tf32 ? tc2d_tf32_supported(R) : tc2d_supported(R)) ||
        !sweep2d_supported(p->r, 1, p->pattern)) {
        set_error("tensor-core sweep: folded radius %d unsupported (1..%d)", R,
                  tf32 ? kTcMaxRTf32 : kTcMaxR);
        return STENCIL_ERR_UNSUPPORTED;
    }
    ensure_device_facts(p);
    // the grouped form issues about a quarter of the MMAs but pays a fixed
    // epilogue per tile: it wins for wide folds (measured on GB300: 1318 vs
    // 1002 GS/s at R = 8, 783 vs 853 at R = 4, 394 vs 643 at R = 2)
    // TF32 operands run in the per-offset kernel only
    const bool grouped = !tf32 && (p->tc_form == 2 || (p->tc_form == 0 && R >= kTcGroupedMinR));
    if (grouped ? tc2dg_smem_bytes(R, 1) > (size_t)p->max_smem
                : tc2d_smem_bytes(R, false, tf32) > (size_t)p->max_smem) {
        set_error("tensor-core sweep: shared memory");
        return STENCIL_ERR_UNSUPPORTED;
    }
    const uint16_t *panels = nullptr;
    double sum_c = 0.0;
    const std::vector<double> *c1 = nullptr;
    stencil_status_t st = tc_panels(p, m, grouped, tf32, &panels, &sum_c);
    if (st == STENCIL_OK) st = plan_folded(p, 1, &c1);
    if (st == STENCIL_OK) st = ensure_padded(p);
    if (st != STENCIL_OK) return st;
    const int64_t q = T / m, rem = T % m;
    const int max_halo = std::min(kGhost, nmin);
    const int bplain = std::max(1, max_halo / p->r);
    std::vector<int> plain;  // fused plain steps per remainder pass
    for (int64_t d = 0; d < rem; d += bplain) plain.push_back((int)std::min<int64_t>(bplain, rem - d));
    int gw = q ? R : 0;
    for (int b : plain) gw = std::max(gw, b * p->r);
    for (int b : plain) {
        stencil_plan_s::PassCfg cfg;
        st = pass2d_config(p, 1, b, &cfg);
        if (st != STENCIL_OK) return st;
    }
    const bool out_vec4 = grid_vec4(p, out);
    const int64_t npass = q + (int64_t)plain.size();

    auto enqueue = [&](cudaStream_t st_, int *nl) -> stencil_status_t {
        cudaError_t e = launch_import(p->A, in, gw, st_, p->pitch_y);
        if (e != cudaSuccess) return cuda_fail(e, "import launch");
        *nl += 1;
        if (p->tc_center && q > 0) {
            e = cudaMemsetAsync(p->d_acc, 0, sizeof(double), st_);
            if (e == cudaSuccess) e = launch_grid_mean(p->A.origin, p->nx, p->ny, p->A.py, p->d_acc, st_);
            if (e != cudaSuccess) return cuda_fail(e, "grid mean");
            *nl += 1;
        }
        const Padded *cur = &p->A, *oth = &p->B;
        int64_t done = 0;
        for (int64_t i = 0; i < q; ++i, ++done) {
            const bool last = done + 1 == npass;
            float *dst = last ? out : oth->origin;
            const int64_t dpy = last ? p->pitch_y : oth->py;
            stencil_status_t r =
                grouped ? launch_tc_grouped_pass(p, *cur, m, panels, sum_c, dst, dpy, last ? 0 : gw,
                                                 last ? out_vec4 : true, st_)
                        : launch_tc_pass(p, *cur, m, panels, sum_c, dst, dpy, last ? 0 : gw,
                                         last ? out_vec4 : true, st_);
            if (r != STENCIL_OK) return r;
            *nl += 1;
            std::swap(cur, oth);
        }
        for (int b : plain) {
            const bool last = done + 1 == npass;
            stencil_status_t r = launch_pass2d(p, *cur, 1, b, *c1, last ? out : oth->origin,
                                               last ? p->pitch_y : oth->py, last ? 0 : gw,
                                               last ? out_vec4 : true, st_);
            if (r != STENCIL_OK) return r;
            *nl += 1;
            ++done;
            std::swap(cur, oth);
        }
        return STENCIL_OK;
    };
    std::vector<int64_t> key = {3, (int64_t)(uintptr_t)in, (int64_t)(uintptr_t)out, T, m,
                                p->precision, p->tc_center, p->wait_ms, grouped ? 1 : 0,
                                p->fault_withhold_mma};
    st = run_maybe_graph(p, key, s, enqueue);
    p->last_m = m;
    p->last_b = 1;
    p->last_engine = 1;
    p->last_tc_form = grouped ? 2 : 1;
    return st;
}

}  // namespace sg
