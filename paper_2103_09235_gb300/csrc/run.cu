// Time-loop drivers of stencil_run (T steps = floor(T/m) folded sweeps plus
// T mod m plain steps, Section 3.4; two alternating arrays, Section 3.3):
// they split the sweeps into passes of b fused sweeps, pick tile shapes,
// encode tensor maps and launch the sweep kernels in stream order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "plan.h"

namespace sg {

namespace {

int device_attr(cudaDeviceAttr a)
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, a, dev);
    return v;
}

struct Pass {
    int m;  // fold factor of this pass's stencil
    int b;  // sweeps fused in this pass
};

// floor(T/m) folded sweeps in passes of at most b, then T mod m plain steps
// in passes whose halo fits the ghost band.
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

stencil_status_t run1d(stencil_plan_s *p, const void *in, void *out, int64_t T, int m,
                       cudaStream_t s)
{
    if (m == 0) m = 1;
    const bool f64 = p->dtype == STENCIL_F64;
    const size_t esz = f64 ? 8 : 4;
    const int R = m * p->r;
    if (!sweep1d_supported(R, f64) || !sweep1d_supported(p->r, f64)) {
        set_error("1D sweep: no kernel for folded radius %d", R);
        return STENCIL_ERR_UNSUPPORTED;
    }
    if (2 * R + 1 > p->nx) {
        set_error("1D sweep: folded width %d exceeds the grid", 2 * R + 1);
        return STENCIL_ERR_INVALID_ARG;
    }
    const std::vector<double> *cm = nullptr, *c1 = nullptr;
    stencil_status_t st = plan_folded(p, m, &cm);
    if (st == STENCIL_OK) st = plan_folded(p, 1, &c1);
    if (st != STENCIL_OK) return st;

    const int tile = f64 ? 2048 : 4096;
    const int bsteps = p->block_b > 0 ? p->block_b : 32;  // sweeps per launch
    const size_t bytes = esz * (size_t)p->nx;
    cudaError_t e;
    if (!p->d1a) {
        e = cudaMalloc(&p->d1a, bytes);
        if (e == cudaSuccess) e = cudaMalloc(&p->d1b, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "1D scratch");
        p->scratch_bytes += 2 * bytes;
    }
    const int64_t q = T / m, rem = T % m;
    std::vector<Pass> passes;
    for (int64_t d = 0; d < q; d += bsteps) passes.push_back({m, (int)std::min<int64_t>(bsteps, q - d)});
    for (int64_t d = 0; d < rem; d += bsteps) passes.push_back({1, (int)std::min<int64_t>(bsteps, rem - d)});

    const void *src = in;
    if (in == out && passes.size() == 1) {
        e = cudaMemcpyAsync(p->d1b, in, bytes, cudaMemcpyDeviceToDevice, s);
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
        Sweep1DArgs a;
        a.src = src;
        a.dst = dst;
        a.n = p->nx;
        a.tile = tile;
        a.b = ps.b;
        const std::vector<double> &c = ps.m == m ? *cm : *c1;
        for (size_t k = 0; k < c.size(); ++k) a.c[k] = c[k];
        e = launch_sweep1d(ps.m * p->r, f64, a, s);
        if (e != cudaSuccess) return cuda_fail(e, "1D sweep launch");
        p->launches += 1;
        src = dst;
        nb ^= 1;
    }
    p->last_m = m;
    p->last_b = bsteps;
    p->last_engine = 0;
    return STENCIL_OK;
}

// One CUDA-core 2D pass from padded grid `src` to `dst_origin`.
static stencil_status_t launch_pass2d(stencil_plan_s *p, const Padded &src, int m, int b,
                                      const std::vector<double> &c, float *dst, int64_t dst_py,
                                      int dst_gw, bool dst_vec4, cudaStream_t s)
{
    const int R = m * p->r;
    const int H = b * R, HX = round_up(H, 4);
    const int max_smem = device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin);
    int ty = p->tile_y > 0 ? p->tile_y : 64;
    int bf = 0;
    size_t smem = sweep2d_smem_bytes(ty, b, R, &bf);
    while ((smem > (size_t)max_smem || ty + 2 * H > 256) && ty > 16) {
        ty -= 8;
        smem = sweep2d_smem_bytes(ty, b, R, &bf);
    }
    if (smem > (size_t)max_smem) {
        set_error("2D sweep: halo %d needs too much shared memory", H);
        return STENCIL_ERR_UNSUPPORTED;
    }
    Sweep2DArgs a;
    a.nx = p->nx;
    a.ny = p->ny;
    a.tiles_x = ceil_div(p->nx, kTileX2D);
    const int tiles_y = ceil_div(p->ny, ty);
    a.ntiles = a.tiles_x * tiles_y;
    a.tile_y = ty;
    a.b = b;
    a.halo = H;
    a.halo_x = HX;
    a.map_x0 = src.gx;
    a.map_y0 = src.gy;
    a.buf_floats = bf;
    a.dst = dst;
    a.dst_py = dst_py;
    a.dst_gw = dst_gw;
    a.dst_vec4 = dst_vec4 ? 1 : 0;
    a.status = p->d_status;
    a.wait_ns = (unsigned long long)p->wait_ms * 1000000ull;
    for (size_t k = 0; k < c.size(); ++k) a.c[k] = (float)c[k];
    const int box[2] = {kTileX2D + 2 * HX, ty + 2 * H};
    const CUtensorMap *map = plan_map(p, src, box);
    if (!map) return STENCIL_ERR_CUDA;
    const int occ = std::max(1, sweep2d_ctas_per_sm(p->r, m, p->pattern, smem));
    const int grid = std::min(a.ntiles, occ * device_attr(cudaDevAttrMultiProcessorCount));
    cudaError_t e = launch_sweep2d(p->r, m, p->pattern, *map, a, grid, smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "2D sweep launch");
    p->launches += 1;
    return STENCIL_OK;
}

stencil_status_t run2d_tc(stencil_plan_s *p, const float *in, float *out, int64_t T, int m,
                          cudaStream_t s);

stencil_status_t run2d(stencil_plan_s *p, const float *in, float *out, int64_t T, int m,
                       cudaStream_t s)
{
    int b = p->block_b;
    int ty_saved = p->tile_y;
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
    }
    if (m > 1 && p->pattern == PAT_BOX && p->precision != STENCIL_PREC_FP32) {
        p->tile_y = ty_saved;
        return run2d_tc(p, in, out, T, m, s);
    }
    const int R = m * p->r;
    const int nmin = std::min(p->nx, p->ny);
    if (2 * R + 1 > nmin || R > kGhost) {
        p->tile_y = ty_saved;
        set_error("2D sweep: folded width %d exceeds the grid or the ghost band", 2 * R + 1);
        return STENCIL_ERR_INVALID_ARG;
    }
    if (!sweep2d_supported(p->r, m, p->pattern) || !sweep2d_supported(p->r, 1, p->pattern)) {
        p->tile_y = ty_saved;
        set_error("2D sweep: no CUDA-core kernel for r=%d m=%d", p->r, m);
        return STENCIL_ERR_UNSUPPORTED;
    }
    if (b == 0) b = m == 1 ? 1 : std::max(1, 8 / R);
    const int max_halo = std::min(kGhost, nmin);
    while (b > 1 && b * R > max_halo) --b;

    const std::vector<double> *cm = nullptr, *c1 = nullptr;
    stencil_status_t st = plan_folded(p, m, &cm);
    if (st == STENCIL_OK) st = plan_folded(p, 1, &c1);
    if (st == STENCIL_OK) st = ensure_padded(p);
    if (st != STENCIL_OK) {
        p->tile_y = ty_saved;
        return st;
    }
    std::vector<Pass> passes = make_passes(T, m, b, p->r, max_halo);
    int gw = 0;
    for (const Pass &ps : passes) gw = std::max(gw, ps.b * ps.m * p->r);

    cudaError_t e = launch_import(p->A, in, gw, s);
    if (e != cudaSuccess) {
        p->tile_y = ty_saved;
        return cuda_fail(e, "import launch");
    }
    p->launches += 1;
    const Padded *cur = &p->A, *oth = &p->B;
    const bool out_vec4 = (p->nx % 4 == 0) && ((uintptr_t)out % 16 == 0);
    for (size_t i = 0; i < passes.size() && st == STENCIL_OK; ++i) {
        const bool last = i + 1 == passes.size();
        const Pass &ps = passes[i];
        st = launch_pass2d(p, *cur, ps.m, ps.b, ps.m == m ? *cm : *c1,
                           last ? out : oth->origin, last ? (int64_t)p->nx : oth->py,
                           last ? 0 : gw, last ? out_vec4 : true, s);
        std::swap(cur, oth);
    }
    p->tile_y = ty_saved;
    p->last_m = m;
    p->last_b = b;
    p->last_engine = 0;
    return st;
}

}  // namespace sg
