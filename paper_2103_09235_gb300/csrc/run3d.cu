// Time-loop driver of 3D runs: floor(T/m) folded sweeps and T mod m plain
// steps, one z-streaming CUDA-core sweep per launch, ping-ponging between the
// plan's padded grids (Section 3.3's two arrays) and ending in `out`.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "plan.h"

namespace sg {

namespace {
constexpr int kTX3 = 64, kTY3 = 16;
}

// Planes per z chunk of a 3D pass of b fused sweeps of folded radius R: 16
// for a single radius-1 sweep and 32 otherwise (each chunk re-reads 2bR
// planes of halo), halved down to 8 while the grid has fewer than 4 CTAs per
// SM (many short CTAs balance the SMs and bound the tail; measured on GB300
// at 512^3 and 256^3); the plan's z_chunk option overrides it.
int zchunk3d(const stencil_plan_s *p, int R, int b)
{
    const int ntiles_xy = ceil_div(p->nx, kTX3) * ceil_div(p->ny, kTY3);
    int zc = (b == 1 && R <= 1) ? 16 : 32;
    while (zc > 8 && (int64_t)ntiles_xy * ceil_div(p->nz, zc) < 4 * p->sm_count) zc /= 2;
    if (p->z_chunk > 0) zc = p->z_chunk;
    return zc;
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
    const int zc = zchunk3d(p, R, b);
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

namespace {

// The pieces' pass counters and neighbour lists for a multi-pass sweep of
// folded radius R with z chunks of zc planes (built and uploaded once per
// plan and configuration), or null if a neighbour list is too long or the
// axes have too many tiles for the host tables.
int *q3_memory(stencil_plan_s *p, int R, int zc, int HX)
{
    const auto key = std::make_tuple(R, zc, HX);
    auto it = p->q3_mem.find(key);
    if (it != p->q3_mem.end()) return it->second;
    const int tx = ceil_div(p->nx, kTX3), ty = ceil_div(p->ny, kTY3), tz = ceil_div(p->nz, zc);
    if (std::max(tx, std::max(ty, tz)) > 4096) return nullptr;
    const size_t ntiles = (size_t)tx * ty * tz;
    std::vector<int> dep((size_t)(tx + ty + tz) * kDep3);
    // x: the staged box spans 64 + 2 HX columns; y: 16 + 2R rows; z: the
    // chunk's planes and R on either side, read four planes at a time
    const bool ok =
        axis_deps(p->nx, kTX3, tx, [&](int t) { return std::make_pair(t * kTX3 - HX, t * kTX3 + kTX3 + HX); },
                  dep.data()) &&
        axis_deps(p->ny, kTY3, ty, [&](int t) { return std::make_pair(t * kTY3 - R, t * kTY3 + kTY3 + R); },
                  dep.data() + (size_t)tx * kDep3) &&
        axis_deps(p->nz, zc, tz,
                  [&](int t) {
                      const int z0 = t * zc, z1 = std::min(p->nz, z0 + zc);
                      return std::make_pair(z0 - R, z0 - R + round_up(z1 - z0 + 2 * R, 4));
                  },
                  dep.data() + (size_t)(tx + ty) * kDep3);
    if (!ok) return nullptr;
    int *mem = nullptr;
    const size_t bytes = (ntiles + dep.size()) * sizeof(int);
    if (cudaMalloc(&mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaMemcpy(mem + ntiles, dep.data(), dep.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(mem);
        cudaGetLastError();
        return nullptr;
    }
    p->scratch_bytes += bytes;
    p->q3_mem[key] = mem;
    return mem;
}

// npass single sweeps of c = c^(m) in one persistent launch (k_sweep3d_q):
// pass t reads `cur` (t even) or `oth` (t odd) and writes the other grid,
// except the last pass, which writes dst.
stencil_status_t launch_passes3d_q(stencil_plan_s *p, const Padded &cur, const Padded &oth, int m,
                                   int npass, int gw, const std::vector<double> &c, float *dst,
                                   int64_t dst_py, int64_t dst_pz, int dst_gw, bool dst_vec4,
                                   int *qmem, cudaStream_t s)
{
    const int R = m * p->r;
    Sweep3DArgs a;
    a.nx = p->nx;
    a.ny = p->ny;
    a.nz = p->nz;
    a.tiles_x = ceil_div(p->nx, kTX3);
    a.tiles_y = ceil_div(p->ny, kTY3);
    a.ntiles_xy = a.tiles_x * a.tiles_y;
    a.zchunk = zchunk3d(p, R, 1);
    a.zchunks = ceil_div(p->nz, a.zchunk);
    a.ntiles = a.ntiles_xy * a.zchunks;
    a.fault_withhold_copy = p->fault_withhold_copy;
    a.tile_y = kTY3;
    a.halo_x = round_up(R, 4);
    a.map_x0 = cur.gx;
    a.map_y0 = cur.gy;
    a.map_z0 = cur.gz;
    a.nst = (p->stages == 2 || p->stages == 3) ? p->stages : 2;
    int bf = 0;
    const size_t smem = sweep3d_smem_bytes(kTY3, R, &bf, a.nst);
    a.buf_floats = bf;
    a.dst = dst;
    a.dst_py = dst_py;
    a.dst_pz = dst_pz;
    a.dst_gw = dst_gw;
    a.dst_vec4 = dst_vec4 ? 1 : 0;
    a.status = p->d_status;
    a.wait_ns = (unsigned long long)p->wait_ms * 1000000ull;
    round_f32_mass(c.data(), c.size(), c.size() / 2, a.c);
    Sweep3DQueue q;
    memset(&q, 0, sizeof(q));
    q.npass = npass;
    q.done = qmem;
    q.dep = qmem + a.ntiles;
    q.dep_y = a.tiles_x * kDep3;
    q.dep_z = (a.tiles_x + a.tiles_y) * kDep3;
    q.dst[0] = oth.origin;  // even passes read cur
    q.dst[1] = cur.origin;
    q.py = cur.py;
    q.pz = cur.pz;
    q.gw = gw;
    q.fault_withhold_dep = p->fault_withhold_dep;
    const int box[3] = {kTX3 + 2 * a.halo_x, kTY3 + 2 * R, 4};
    const CUtensorMap *map_e = plan_map(p, cur, box);
    const CUtensorMap *map_o = map_e ? plan_map(p, oth, box) : nullptr;
    if (!map_o) return STENCIL_ERR_CUDA;
    const int occ = std::max(1, sweep3d_q_ctas_per_sm(p->r, m, p->pattern, smem));
    const int64_t nitems = (int64_t)npass * a.ntiles;
    const int grid = (int)std::min<int64_t>(nitems, (int64_t)occ * p->sm_count);
    cudaError_t e = cudaMemsetAsync(qmem, 0, sizeof(int) * a.ntiles, s);
    if (e == cudaSuccess)
        e = launch_sweep3d_q(p->r, m, p->pattern, *map_e, *map_o, a, q, grid, smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "3D multi-pass sweep launch");
    return STENCIL_OK;
}

}  // namespace

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
    // each run of consecutive single sweeps of one stencil may become one
    // multi-pass launch (at most 2^30 items each): always with the persistent
    // option 1; with -1 when a pass has more than one and at most 3.5 waves of
    // pieces.  Measured on GB300 (one launch per pass -> persistent, waves):
    // 192^3 box 283 -> 361 GS/s (1.4), 256^3 box 378 -> 448 (1.7), folded
    // m = 2 276 -> 299 (1.7), 256^3 star 423 -> 543 (1.7), 288^3 box 399 ->
    // 432 (2.7), 320^3 box 456 -> 468 (3.3); but 384^3 box 515 -> 448 (5.7)
    // and 512^3 star 710 -> 498 (13.5), where the per-pass launches' four
    // CTAs per SM and better L2 reuse win, and 128^3 box 153 -> 133 (0.4),
    // where a pass has fewer pieces than CTAs and items wait on their
    // neighbours.  The counters and neighbour lists are set up here, before
    // any capture.
    std::vector<int> group(passes.size(), 1);
    std::vector<int *> gmem(passes.size(), nullptr);
    if (p->persistent != 0) {
        for (size_t i = 0; i < passes.size();) {
            size_t j = i;
            while (j < passes.size() && passes[j] == passes[i]) ++j;
            const int mm = passes[i].first, R = mm * p->r, zc = zchunk3d(p, R, 1);
            const int64_t ntiles = (int64_t)ceil_div(p->nx, kTX3) * ceil_div(p->ny, kTY3) *
                                   ceil_div(p->nz, zc);
            bool want = p->persistent == 1;
            if (!want && passes[i].second == 1 && sweep3d_supported(p->r, mm, p->pattern)) {
                const int nst = (p->stages == 2 || p->stages == 3) ? p->stages : 2;
                const int occ = sweep3d_ctas_per_sm(p->r, mm, p->pattern,
                                                    sweep3d_smem_bytes(kTY3, R, nullptr, nst));
                const int64_t slots = (int64_t)occ * p->sm_count;
                want = occ > 0 && ntiles > slots && 2 * ntiles <= 7 * slots;
            }
            int *qm = (want && passes[i].second == 1 && sweep3d_q_supported(p->r, mm, p->pattern) &&
                       j - i >= 2)
                          ? q3_memory(p, R, zc, round_up(R, 4))
                          : nullptr;
            if (qm) {
                const size_t cap = (size_t)std::max<int64_t>(1, (1ll << 30) / ntiles);
                for (size_t k = i; k < j; k += cap) {
                    group[k] = (int)std::min(cap, j - k);
                    gmem[k] = qm;
                }
            }
            i = j;
        }
    }
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
            if (gmem[i] && group[i] >= 2) {
                // passes i .. i+n-1 in one launch; the last of them writes
                // `out` if it ends the run, else the grid it would write
                const int n = group[i], mm = passes[i].first;
                const bool last = i + n == passes.size();
                const Padded *fin = (n % 2) ? oth : cur;
                stencil_status_t r = launch_passes3d_q(
                    p, *cur, *oth, mm, n, gw, mm == m ? *cm : *c1, last ? out : fin->origin,
                    last ? p->pitch_y : fin->py, last ? p->pitch_z : fin->pz, last ? 0 : gw,
                    last ? out_vec4 : true, gmem[i], st_);
                if (r != STENCIL_OK) return r;
                *nl += 1;
                if (n % 2) std::swap(cur, oth);
                i += n - 1;
                continue;
            }
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
                                p->wait_ms, p->fault_withhold_copy, cr.on ? 1 : 0,
                                p->persistent, p->fault_withhold_dep, p->z_chunk, p->stages};
    st = run_maybe_graph(p, key, s, enqueue);
    p->last_m = m;
    p->last_b = b;
    p->last_engine = 0;
    p->last_persist = 0;
    for (size_t i = 0; i < passes.size(); ++i)
        if (gmem[i] && group[i] >= 2) p->last_persist = 1;
    return st;
}

}  // namespace sg
