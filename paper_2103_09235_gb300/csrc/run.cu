// Time-loop drivers of stencil_run (T steps = floor(T/m) folded sweeps plus
// T mod m plain steps, Section 3.4; two alternating arrays, Section 3.3):
// they split the sweeps into passes of b fused sweeps, pick tile shapes,
// encode tensor maps and launch the sweep kernels in stream order, replaying
// a captured CUDA graph for repeated runs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "plan.h"

namespace sg {

namespace {

struct Pass {
    int m;  // fold factor of this pass's stencil
    int b;  // sweeps fused in this pass
};

// floor(T/m) folded sweeps in passes of at most b, then T mod m plain steps
// in passes whose halo fits max_halo.
std::vector<Pass> make_passes(int64_t T, int m, int b, int r, int max_halo)
{
    std::vector<Pass> v;
    const int64_t q = T / m, rem = T % m;
    for (int64_t done = 0; done < q; done += b) v.push_back({m, (int)std::min<int64_t>(b, q - done)});
    const int bmax_plain = std::max(1, max_halo / r);
    for (int64_t done = 0; done < rem; done += bmax_plain)
        v.push_back({1, (int)std::min<int64_t>(bmax_plain, rem - done)});
    return v;
}

}  // namespace

void ensure_device_facts(stencil_plan_s *p)
{
    if (p->sm_count) return;
    cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    cudaDeviceGetAttribute(&p->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    cudaDeviceGetAttribute(&p->max_smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, p->device);
    if (p->sm_count <= 0) p->sm_count = 1;
}

CentredRun centred_run(stencil_plan_s *p, int64_t T)
{
    CentredRun c;
    c.on = p->center != 0;
    c.sum = p->d_acc + 1;  // d_acc[0] belongs to the tensor-core path's own centring
    c.inv_n = 1.0 / ((double)p->nx * p->ny * p->nz);
    double sc = 0.0;
    for (double v : p->coeffs) sc += v;
    c.factor = pow(sc, (double)T);  // the mean's gain over T steps: (sum c)^T
    return c;
}

void clear_graphs(stencil_plan_s *p)
{
    for (auto &kv : p->graphs) cudaGraphExecDestroy(kv.second.exec);
    p->graphs.clear();
}

stencil_status_t run1d(stencil_plan_s *p, const void *in, void *out, int64_t T, int m,
                       cudaStream_t s)
{
    const int saved_b = p->block_b;
    struct RestoreB {
        stencil_plan_s *p;
        int b;
        ~RestoreB() { p->block_b = b; }
    } restore_b{p, saved_b};
    const bool auto_fold = m == 0;
    if (m == 0) {
        if (p->tuned_m == 0 && p->autotune) {
            stencil_status_t st = autotune2d(p, s, T);
            if (st != STENCIL_OK) return st;
        }
        m = p->tuned_m > 0 ? p->tuned_m : 1;
        if (p->block_b == 0 && p->tuned_b > 0) p->block_b = p->tuned_b;
    }
    const bool use_tess = auto_fold ? p->tuned_tess != 0 : p->tessellate != 0;
    const bool f64 = p->dtype == STENCIL_F64;
    const size_t esz = f64 ? 8 : 4;
    const int R = m * p->r;
    if (2 * R + 1 > p->nx) {
        set_error("1D sweep: folded width %d exceeds the grid", 2 * R + 1);
        return STENCIL_ERR_INVALID_ARG;
    }
    if (!sweep1d_supported(R, f64) || !sweep1d_supported(p->r, f64)) {
        set_error("1D sweep: no kernel for folded radius %d", R);
        return STENCIL_ERR_UNSUPPORTED;
    }
    const std::vector<double> *cm = nullptr, *c1 = nullptr;
    stencil_status_t st = plan_folded(p, m, &cm);
    if (st == STENCIL_OK) st = plan_folded(p, 1, &c1);
    if (st != STENCIL_OK) return st;

    // points per CTA tile: the plan's option, else the tuned size of an
    // automatic fold, else by form and radius -- measured on GB300, 2^20
    // points, T = 100: overlapped tiles of 1024 points up to radius 6 (FP32
    // m = 1 1176 against 993 GS/s with 4096, m = 4 3293 against 2624; FP64
    // m = 1 156 against 138 with 2048) and 4096 above (m = 8: 2129 against
    // 1859); tessellated FP32 4096 (m = 6: 2492 against 2174 with 1024),
    // tessellated FP64 1024 (m = 4: 199 against 181 with 2048)
    const int tile = p->tile_1d > 0                    ? p->tile_1d
                     : (auto_fold && p->tuned_ty > 0) ? p->tuned_ty
                     : use_tess                        ? (f64 ? 1024 : 4096)
                     : (R <= 6 ? 1024 : 4096);
    const int bsteps = p->block_b > 0 ? p->block_b : 32;  // sweeps per launch
    const size_t bytes = esz * (size_t)p->nx;
    if (!p->d1a) {
        cudaError_t e = cudaMalloc(&p->d1a, bytes);
        if (e == cudaSuccess) e = cudaMalloc(&p->d1b, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "1D scratch");
        p->scratch_bytes += 2 * bytes;
    }
    const int64_t q = T / m, rem = T % m;
    std::vector<Pass> passes;
    for (int64_t d = 0; d < q; d += bsteps) passes.push_back({m, (int)std::min<int64_t>(bsteps, q - d)});
    for (int64_t d = 0; d < rem; d += bsteps) passes.push_back({1, (int)std::min<int64_t>(bsteps, rem - d)});
    // passes that tessellate exactly (Section 3.4) where their b steps fit the tile
    std::vector<char> tess_pass(passes.size(), 0);
    bool any_tess = false;
    for (size_t i = 0; i < passes.size(); ++i) {
        tess_pass[i] = use_tess && tess1d_fits(p->nx, tile, passes[i].b, passes[i].m * p->r);
        any_tess = any_tess || tess_pass[i];
    }
    if (any_tess && !p->d1p0) {
        cudaError_t e = cudaMalloc(&p->d1p0, bytes);
        if (e == cudaSuccess) e = cudaMalloc(&p->d1p1, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "1D tessellation scratch");
        p->scratch_bytes += 2 * bytes;
    }

    auto enqueue = [&](cudaStream_t st_, int *nl) -> stencil_status_t {
        const void *src = in;
        if (in == out && passes.size() == 1) {
            cudaError_t e = cudaMemcpyAsync(p->d1b, in, bytes, cudaMemcpyDeviceToDevice, st_);
            if (e != cudaSuccess) return cuda_fail(e, "1D alias copy");
            src = p->d1b;
        }
        void *bufs[2] = {p->d1a, p->d1b};
        int nb = 0;
        for (size_t i = 0; i < passes.size(); ++i) {
            const Pass &ps = passes[i];
            const bool last = i + 1 == passes.size();
            void *dst = last ? out : bufs[nb];
            if (!last && dst == src) dst = bufs[nb ^ 1];
            const std::vector<double> &c = ps.m == m ? *cm : *c1;
            double wts[2 * kMaxR1D + 1];
            if (f64) {
                for (size_t k = 0; k < c.size(); ++k) wts[k] = c[k];
            } else {
                float w[2 * kMaxR1D + 1];
                round_f32_mass(c.data(), c.size(), c.size() / 2, w);
                for (size_t k = 0; k < c.size(); ++k) wts[k] = (double)w[k];
            }
            cudaError_t e;
            if (tess_pass[i]) {
                Tess1DArgs t;
                t.src = src;
                t.dst = dst;
                t.par0 = p->d1p0;
                t.par1 = p->d1p1;
                t.n = p->nx;
                t.W = tile;
                t.ntiles = (int)std::max<int64_t>(1, p->nx / tile);
                t.wmax = (int)(p->nx - (int64_t)(t.ntiles - 1) * tile);
                t.b = ps.b;
                for (size_t k = 0; k < c.size(); ++k) t.c[k] = wts[k];
                e = launch_tess1d(ps.m * p->r, f64, t, st_);
                *nl += 2;
            } else {
                Sweep1DArgs a;
                a.src = src;
                a.dst = dst;
                a.n = p->nx;
                a.tile = tile;
                a.b = ps.b;
                for (size_t k = 0; k < c.size(); ++k) a.c[k] = wts[k];
                e = launch_sweep1d(ps.m * p->r, f64, a, st_);
                *nl += 1;
            }
            if (e != cudaSuccess) return cuda_fail(e, "1D sweep launch");
            src = dst;
            nb ^= 1;
        }
        return STENCIL_OK;
    };
    std::vector<int64_t> key = {1, (int64_t)(uintptr_t)in, (int64_t)(uintptr_t)out, T, m, bsteps,
                                any_tess ? 1 : 0, tile};
    st = run_maybe_graph(p, key, s, enqueue);
    p->last_m = m;
    p->last_b = bsteps;
    p->last_engine = 0;
    p->last_tess = (!passes.empty() && tess_pass[0]) ? 1 : 0;
    p->last_ty = tile;
    return st;
}

// Tile shape, shared memory and grid of a 2D CUDA-core pass (cached per plan).
stencil_status_t pass2d_config(stencil_plan_s *p, int m, int b,
                                      stencil_plan_s::PassCfg *cfg, int cpk)
{
    auto key = std::make_tuple(m, b,
                               ((p->tile_y * 8 + p->stages) * 1024 + p->cta_threads) * 4 + cpk);
    auto it = p->pass_cfg.find(key);
    if (it != p->pass_cfg.end()) {
        *cfg = it->second;
        return STENCIL_OK;
    }
    ensure_device_facts(p);
    const int R = m * p->r;
    const int H = b * R;
    // single sweeps and temporally blocked passes alike: 64-row tiles, two
    // stages (measured on GB300 for plain sweeps against 32-row tiles with
    // four stages: 8192^2 box 670 vs 654 GS/s, star 697 vs 630; 4096^2 box
    // 847 vs 677, star 877 vs 773 -- half the shared memory per CTA lets
    // twice the CTAs onto an SM); counterpart passes refill their stage
    // after the first vertical fold: one stage and the tallest tile that fits
    int ty = p->tile_y > 0 ? p->tile_y : (cpk ? 160 : 64);
    int ns = p->stages > 0 ? p->stages : (cpk ? 1 : 2);
    int bf = 0;
    size_t smem = sweep2d_smem_bytes(ty, b, R, &bf, ns, cpk);
    // a blocked pass refills its stage right after a tile's first sweep, so
    // one stage still overlaps the copy with the other sweeps: drop the
    // second stage before shrinking the tile
    if (p->stages <= 0 && b >= 2 && smem > (size_t)p->max_smem) {
        ns = 1;
        smem = sweep2d_smem_bytes(ty, b, R, &bf, ns, cpk);
    }
    while ((smem > (size_t)p->max_smem || ty + 2 * H > 256) && ty > 16) {
        ty -= 8;
        smem = sweep2d_smem_bytes(ty, b, R, &bf, ns, cpk);
    }
    if (smem > (size_t)p->max_smem) {
        set_error("2D sweep: halo %d needs too much shared memory", H);
        return STENCIL_ERR_UNSUPPORTED;
    }
    const int ntiles = ceil_div(p->nx, kTileX2D) * ceil_div(p->ny, ty);
    // counterpart instances are (1, R, PAT_CPk)
    const int occ = std::max(1, cpk ? sweep2d_ctas_per_sm(1, R, PAT_CP1 + cpk - 1, smem, p->cta_threads)
                                    : sweep2d_ctas_per_sm(p->r, m, p->pattern, smem, p->cta_threads));
    cfg->threads = p->cta_threads;
    cfg->ty = ty;
    cfg->nstages = ns;
    cfg->bf = bf;
    cfg->smem = smem;
    cfg->grid = std::min(ntiles, occ * p->sm_count);
    p->pass_cfg[key] = *cfg;
    return STENCIL_OK;
}

// One CUDA-core 2D pass from padded grid `src` to `dst` (padded origin or dense).
stencil_status_t launch_pass2d(stencil_plan_s *p, const Padded &src, int m, int b,
                                      const std::vector<double> &c, float *dst, int64_t dst_py,
                                      int dst_gw, bool dst_vec4, cudaStream_t s,
                                      const CpFactor *cp)
{
    const int cpk = cp ? cp->k : 0;
    stencil_plan_s::PassCfg cfg;
    stencil_status_t st = pass2d_config(p, m, b, &cfg, cpk);
    if (st != STENCIL_OK) return st;
    const int R = m * p->r;
    const int H = b * R, HX = round_up(H, 4);
    Sweep2DArgs a;
    a.nx = p->nx;
    a.ny = p->ny;
    a.tiles_x = ceil_div(p->nx, kTileX2D);
    a.ntiles = a.tiles_x * ceil_div(p->ny, cfg.ty);
    a.tile_y = cfg.ty;
    a.b = b;
    a.halo = H;
    a.halo_x = HX;
    a.map_x0 = src.gx;
    a.map_y0 = src.gy;
    a.buf_floats = cfg.bf;
    a.nstages = cfg.nstages;
    a.dst = dst;
    a.dst_py = dst_py;
    a.dst_gw = dst_gw;
    a.dst_vec4 = dst_vec4 ? 1 : 0;
    a.status = p->d_status;
    a.wait_ns = (unsigned long long)p->wait_ms * 1000000ull;
    a.fault_withhold_copy = p->fault_withhold_copy;
    if (cpk) {
        // u_0 .. u_{K-1}, then v_0 .. v_{K-1}
        // each factor keeps its own sum, so every separable term keeps its mass
        const int W = 2 * R + 1;
        for (int k = 0; k < cpk; ++k) {
            round_f32_mass(cp->u.data() + k * W, W, W / 2, a.c + k * W);
            round_f32_mass(cp->v.data() + k * W, W, W / 2, a.c + cpk * W + k * W);
        }
    } else {
        round_f32_mass(c.data(), c.size(), c.size() / 2, a.c);
    }
    const int box[2] = {kTileX2D + 2 * HX, cfg.ty + 2 * H};
    const CUtensorMap *map = plan_map(p, src, box);
    if (!map) return STENCIL_ERR_CUDA;
    cudaError_t e = cpk ? launch_sweep2d(1, R, PAT_CP1 + cpk - 1, *map, a, cfg.grid, cfg.smem,
                                         cfg.threads, s)
                        : launch_sweep2d(p->r, m, p->pattern, *map, a, cfg.grid, cfg.smem,
                                         cfg.threads, s);
    if (e != cudaSuccess) return cuda_fail(e, "2D sweep launch");
    return STENCIL_OK;
}

stencil_status_t run2d_tc(stencil_plan_s *p, const float *in, float *out, int64_t T, int m,
                          cudaStream_t s);

stencil_status_t run2d(stencil_plan_s *p, const float *in, float *out, int64_t T, int m,
                       cudaStream_t s)
{
    int b = p->block_b;
    struct Restore {
        stencil_plan_s *p;
        int ty, thr, ns;
        ~Restore()
        {
            p->tile_y = ty;
            p->cta_threads = thr;
            p->stages = ns;
        }
    } restore{p, p->tile_y, p->cta_threads, p->stages};
    bool cuda_core_only = false;
    if (m == 0) {
        if (p->tuned_m == 0 && p->autotune) {
            stencil_status_t st = autotune2d(p, s);
            if (st != STENCIL_OK) return st;
        }
        if (p->tuned_m == 0) {
            p->tuned_m = 1;
            p->tuned_b = 1;
        }
        m = p->tuned_m;
        if (b == 0) b = p->tuned_b;
        if (p->tile_y == 0) p->tile_y = p->tuned_ty;
        if (p->cta_threads == 0) p->cta_threads = p->tuned_thr;
        if (p->stages == 0) p->stages = p->tuned_ns;
        cuda_core_only = p->tuned_engine == 0;
    }

    // any folded 2D stencil fits the Toeplitz contraction (a star's folded
    // diamond just leaves zero weights in the panels)
    if (m > 1 && p->precision != STENCIL_PREC_FP32 && !cuda_core_only)
        return run2d_tc(p, in, out, T, m, s);
    const int R = m * p->r;
    const int nmin = std::min(p->nx, p->ny);
    if (2 * R + 1 > nmin || R > kGhost) {
        set_error("2D sweep: folded width %d exceeds the grid or the ghost band", 2 * R + 1);
        return STENCIL_ERR_INVALID_ARG;
    }
    // the counterpart form of the folded (and, when forced, the plain) passes
    const CpFactor *cpm = nullptr, *cp1 = nullptr;
    stencil_status_t st = plan_counterparts(p, m, &cpm);
    if (st == STENCIL_OK) st = plan_counterparts(p, 1, &cp1);
    if (st != STENCIL_OK) return st;
    if ((!cpm->k && !sweep2d_supported(p->r, m, p->pattern)) ||
        (!cp1->k && !sweep2d_supported(p->r, 1, p->pattern))) {
        set_error("2D sweep: no CUDA-core kernel for r=%d m=%d", p->r, m);
        return STENCIL_ERR_UNSUPPORTED;
    }
    if (b == 0) b = m == 1 ? 1 : std::max(1, 8 / R);
    const int max_halo = std::min(kGhost, nmin);
    while (b > 1 && b * R > max_halo) --b;

    const std::vector<double> *cm = nullptr, *c1 = nullptr;
    st = plan_folded(p, m, &cm);
    if (st == STENCIL_OK) st = plan_folded(p, 1, &c1);
    if (st == STENCIL_OK) st = ensure_padded(p);
    if (st != STENCIL_OK) return st;
    const std::vector<Pass> passes = make_passes(T, m, b, p->r, max_halo);
    auto cp_of = [&](const Pass &ps) { return ps.m == m ? cpm : cp1; };
    int gw = 0;
    for (const Pass &ps : passes) gw = std::max(gw, ps.b * ps.m * p->r);
    // resolve every pass configuration before any capture starts
    int first_ty = 0, first_thr = 0, first_ns = 0;
    for (const Pass &ps : passes) {
        stencil_plan_s::PassCfg cfg;
        st = pass2d_config(p, ps.m, ps.b, &cfg, cp_of(ps)->k);
        if (st != STENCIL_OK) return st;
        if (!first_ty) {
            const int cpk = cp_of(ps)->k;
            first_ty = cfg.ty;
            first_ns = cfg.nstages;
            first_thr = cpk ? sweep2d_block_threads(1, ps.m * p->r, PAT_CP1 + cpk - 1, cfg.threads)
                            : sweep2d_block_threads(p->r, ps.m, p->pattern, cfg.threads);
        }
    }
    const bool out_vec4 = grid_vec4(p, out);
    const CentredRun cr = centred_run(p, T);

    auto enqueue = [&](cudaStream_t st_, int *nl) -> stencil_status_t {
        cudaError_t e = cudaSuccess;
        if (cr.on) {
            e = cudaMemsetAsync(cr.sum, 0, sizeof(double), st_);
            if (e == cudaSuccess)
                e = launch_grid_sum(in, p->nx, p->ny, 1, p->pitch_y, p->pitch_z, cr.sum, st_);
            if (e != cudaSuccess) return cuda_fail(e, "grid sum launch");
            *nl += 1;
        }
        e = launch_import(p->A, in, gw, st_, p->pitch_y, 0, cr.on ? cr.sum : nullptr, cr.inv_n);
        if (e != cudaSuccess) return cuda_fail(e, "import launch");
        *nl += 1;
        const Padded *cur = &p->A, *oth = &p->B;
        for (size_t i = 0; i < passes.size(); ++i) {
            const bool last = i + 1 == passes.size();
            const Pass &ps = passes[i];
            stencil_status_t r = launch_pass2d(p, *cur, ps.m, ps.b, ps.m == m ? *cm : *c1,
                                               last ? out : oth->origin,
                                               last ? p->pitch_y : oth->py, last ? 0 : gw,
                                               last ? out_vec4 : true, st_,
                                               cp_of(ps)->k ? cp_of(ps) : nullptr);
            if (r != STENCIL_OK) return r;
            *nl += 1;
            std::swap(cur, oth);
        }
        if (cr.on) {
            e = launch_add_bias(out, p->nx, p->ny, 1, p->pitch_y, p->pitch_z, cr.sum, cr.inv_n,
                                cr.factor, st_);
            if (e != cudaSuccess) return cuda_fail(e, "bias launch");
            *nl += 1;
        }
        return STENCIL_OK;
    };
    std::vector<int64_t> key = {2, (int64_t)(uintptr_t)in, (int64_t)(uintptr_t)out, T, m, b,
                                p->tile_y, p->wait_ms, p->fault_withhold_copy, cpm->k, cp1->k,
                                cr.on ? 1 : 0, p->cta_threads, p->stages};
    st = run_maybe_graph(p, key, s, enqueue);
    p->last_m = m;
    p->last_b = b;
    p->last_ty = first_ty;
    p->last_threads = first_thr;
    p->last_stages = first_ns;
    p->last_cp = cpm->k;
    p->last_engine = 0;
    return st;
}

}  // namespace sg
