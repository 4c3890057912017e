// Time-loop driver of 3D runs: floor(T/m) folded sweeps and T mod m plain
// steps, one z-streaming CUDA-core sweep per launch, ping-ponging between the
// plan's padded grids (Section 3.3's two arrays) and ending in `out`.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "plan.h"

namespace sg {

namespace {
constexpr int kTX3 = 64, kTY3 = 16;
}

// One 3D pass of b (1 or 2) fused sweeps of c = c^(m).
stencil_status_t launch_pass3d(stencil_plan_s *p, const Padded &src, int m, int b,
                                      const std::vector<double> &c, float *dst, int64_t dst_py,
                                      int64_t dst_pz, int dst_gw, bool dst_vec4, cudaStream_t s)
{
    const int R = m * p->r;
    Sweep3DArgs a;
    a.nx = p->nx;
    a.ny = p->ny;
    a.nz = p->nz;
    a.tiles_x = ceil_div(p->nx, kTX3);
    a.tiles_y = ceil_div(p->ny, kTY3);
    a.ntiles_xy = a.tiles_x * a.tiles_y;
    // z chunks of 16 planes for a single radius-1 sweep and 32 otherwise (each
    // chunk re-reads 2bR planes of halo): many short CTAs balance the SMs and
    // bound the tail; measured on GB300 at 512^3 and 256^3
    int zc = (b == 1 && R <= 1) ? 16 : 32;
    while (zc > 8 && (int64_t)a.ntiles_xy * ceil_div(p->nz, zc) < 4 * p->sm_count) zc /= 2;
    if (p->z_chunk > 0) zc = p->z_chunk;  // the plan's option
    a.zchunk = zc;
    a.zchunks = ceil_div(p->nz, zc);
    a.ntiles = a.ntiles_xy * a.zchunks;
    a.fault_withhold_copy = p->fault_withhold_copy;
    a.tile_y = kTY3;
    a.halo_x = b == 2 ? sweep3d_tb_halo_x() : round_up(R, 4);
    a.map_x0 = src.gx;
    a.map_y0 = src.gy;
    a.map_z0 = src.gz;
    int bf = 0;
    // ring stages of a single sweep: the plan's option (2 or 3), else 2 --
    // measured on GB300, two stages let a fourth CTA onto each SM (shared
    // memory held three) and were never slower: 256^3 box 377 vs 349 GS/s,
    // 384^3 box 509 vs 476, 512^3 star m = 2 1003 vs 955, plain star equal
    a.nst = (p->stages == 2 || p->stages == 3) ? p->stages : 2;
    const size_t smem = b == 2 ? sweep3d_tb_smem_bytes(R, &bf)
                               : sweep3d_smem_bytes(kTY3, R, &bf, a.nst);
    a.buf_floats = bf;
    a.dst = dst;
    a.dst_py = dst_py;
    a.dst_pz = dst_pz;
    a.dst_gw = dst_gw;
    a.dst_vec4 = dst_vec4 ? 1 : 0;
    a.status = p->d_status;
    a.wait_ns = (unsigned long long)p->wait_ms * 1000000ull;
    round_f32_mass(c.data(), c.size(), c.size() / 2, a.c);
    // one 3D box per stage: 64+2HX columns, 16+2bR rows, 4 planes
    const int box[3] = {kTX3 + 2 * a.halo_x, kTY3 + 2 * b * R, 4};
    const CUtensorMap *map = plan_map(p, src, box);
    if (!map) return STENCIL_ERR_CUDA;
    cudaError_t e = b == 2 ? launch_sweep3d_tb(p->r, m, p->pattern, *map, a, a.ntiles, smem, s)
                           : launch_sweep3d(p->r, m, p->pattern, *map, a, a.ntiles, smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "3D sweep launch");
    return STENCIL_OK;
}

stencil_status_t run3d(stencil_plan_s *p, const float *in, float *out, int64_t T, int m,
                       cudaStream_t s)
{
    // an explicit fold with a BF16 or TF32 precision runs on the tensor cores
    if (m > 1 && p->precision != STENCIL_PREC_FP32) return run3d_tc(p, in, out, T, m, s);
    int b = p->block_b;
    if (m == 0) {
        if (p->tuned_m == 0 && p->autotune) {
            stencil_status_t st = autotune2d(p, s);
            if (st != STENCIL_OK) return st;
        }
        m = p->tuned_m > 0 ? p->tuned_m : 1;
        if (b == 0) b = p->tuned_b;
    }
    if (b <= 0) b = 1;
    if (b > 2) {
        set_error("3D sweep: at most 2 fused sweeps per pass (block_b = %d)", b);
        return STENCIL_ERR_UNSUPPORTED;
    }
    const int R = m * p->r;
    const int nmin = std::min(p->nx, std::min(p->ny, p->nz));
    if (2 * R + 1 > nmin || R > kGhost) {
        set_error("3D sweep: folded width %d exceeds the grid", 2 * R + 1);
        return STENCIL_ERR_INVALID_ARG;
    }
    if (!sweep3d_supported(p->r, m, p->pattern) || !sweep3d_supported(p->r, 1, p->pattern)) {
        set_error("3D sweep: no kernel for r=%d m=%d", p->r, m);
        return STENCIL_ERR_UNSUPPORTED;
    }
    if (b == 2 && (!sweep3d_tb_supported(p->r, m, p->pattern) || 2 * R > std::min(kGhost, nmin))) {
        set_error("3D sweep: no fused pair of sweeps for r=%d m=%d on this grid", p->r, m);
        return STENCIL_ERR_UNSUPPORTED;
    }
    const std::vector<double> *cm = nullptr, *c1 = nullptr;
    stencil_status_t st = plan_folded(p, m, &cm);
    if (st == STENCIL_OK) st = plan_folded(p, 1, &c1);
    if (st == STENCIL_OK) st = ensure_padded(p);
    if (st != STENCIL_OK) return st;
    ensure_device_facts(p);
    // passes as (m, fused sweeps): floor(T/m) folded sweeps in groups of b,
    // then the T mod m plain steps, paired too when a fused plain pair exists
    std::vector<std::pair<int, int>> passes;
    const int64_t q = T / m, rem = T % m;
    for (int64_t d = 0; d < q; d += b) passes.push_back({m, (int)std::min<int64_t>(b, q - d)});
    const int b1 = (b == 2 && sweep3d_tb_supported(p->r, 1, p->pattern)) ? 2 : 1;
    for (int64_t d = 0; d < rem; d += b1) passes.push_back({1, (int)std::min<int64_t>(b1, rem - d)});
    // ghost band: the widest halo any pass reads
    int gw = p->r;
    for (auto &x : passes) gw = std::max(gw, x.first * x.second * p->r);
    const bool out_vec4 = grid_vec4(p, out);
    const CentredRun cr = centred_run(p, T);
    auto enqueue = [&](cudaStream_t st_, int *nl) -> stencil_status_t {
        cudaError_t e = cudaSuccess;
        if (cr.on) {
            e = cudaMemsetAsync(cr.sum, 0, sizeof(double), st_);
            if (e == cudaSuccess)
                e = launch_grid_sum(in, p->nx, p->ny, p->nz, p->pitch_y, p->pitch_z, cr.sum, st_);
            if (e != cudaSuccess) return cuda_fail(e, "grid sum launch");
            *nl += 1;
        }
        e = launch_import(p->A, in, gw, st_, p->pitch_y, p->pitch_z, cr.on ? cr.sum : nullptr,
                          cr.inv_n);
        if (e != cudaSuccess) return cuda_fail(e, "import launch");
        *nl += 1;
        const Padded *cur = &p->A, *oth = &p->B;
        for (size_t i = 0; i < passes.size(); ++i) {
            const bool last = i + 1 == passes.size();
            const int mm = passes[i].first, bb = passes[i].second;
            stencil_status_t r = launch_pass3d(
                p, *cur, mm, bb, mm == m ? *cm : *c1, last ? out : oth->origin,
                last ? p->pitch_y : oth->py, last ? p->pitch_z : oth->pz,
                last ? 0 : gw, last ? out_vec4 : true, st_);
            if (r != STENCIL_OK) return r;
            *nl += 1;
            std::swap(cur, oth);
        }
        if (cr.on) {
            e = launch_add_bias(out, p->nx, p->ny, p->nz, p->pitch_y, p->pitch_z, cr.sum,
                                cr.inv_n, cr.factor, st_);
            if (e != cudaSuccess) return cuda_fail(e, "bias launch");
            *nl += 1;
        }
        return STENCIL_OK;
    };
    std::vector<int64_t> key = {4, (int64_t)(uintptr_t)in, (int64_t)(uintptr_t)out, T, m, b,
                                p->wait_ms, p->fault_withhold_copy, cr.on ? 1 : 0};
    st = run_maybe_graph(p, key, s, enqueue);
    p->last_m = m;
    p->last_b = b;
    p->last_engine = 0;
    return st;
}

}  // namespace sg
