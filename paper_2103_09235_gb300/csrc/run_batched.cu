// stencil_run_batched: flattens every grid's time loop into passes and
// (pass, tile) work items, uploads them once per distinct batch, and runs the
// whole batch as one persistent kernel (after one layout-import launch for all
// grids), captured into a CUDA graph that later calls replay.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "plan.h"

namespace sg {
namespace {

constexpr int kBatchTileYMax = 128;  // tallest tile tried; shortened until shared memory fits

struct GridPlan {
    stencil_plan_s *p;
    const float *in;
    float *out;
    int64_t T;
    int m, b;
    int gw;
    int first_pass, npass;
    int ntiles;
};

// Fold depth and temporal-blocking depth for a grid of a batch, chosen from
// the stencil pattern (measured on GB300 with 96-row tiles: the folded star
// prefers m = 3, the box m = 2, both with two fused sweeps) and clamped to
// the grid.
void choose_mb(const stencil_plan_s *p, int req_m, int *m_out, int *b_out)
{
    const int nmin = std::min(p->nx, p->ny);
    int m = req_m > 0 ? req_m : (p->pattern == PAT_STAR ? 3 : 2);
    int b = p->block_b > 0 ? p->block_b : 2;
    if (req_m == 1 && p->block_b == 0) b = 1;
    while (m > 1 && (2 * m * p->r + 1 > nmin || m * p->r > kGhost ||
                     !batched_variant_supported(p->r, m, p->pattern)))
        --m;
    const int max_halo = std::min(kGhost, nmin);
    while (b > 1 && b * m * p->r > max_halo) --b;
    *m_out = m;
    *b_out = b;
}

// The passes of one grid as (m, b) pairs: floor(T/m) folded sweeps in groups
// of b, then the T mod m plain steps in groups of up to the ghost width.
std::vector<std::pair<int, int>> grid_passes(const stencil_plan_s *p, int64_t T, int m, int b)
{
    std::vector<std::pair<int, int>> mb;
    const int64_t q = T / m, rem = T % m;
    const int max_halo = std::min(kGhost, std::min(p->nx, p->ny));
    for (int64_t d = 0; d < q; d += b) mb.push_back({m, (int)std::min<int64_t>(b, q - d)});
    for (int64_t d = 0; d < rem; d += max_halo)
        mb.push_back({1, (int)std::min<int64_t>(max_halo, rem - d)});
    return mb;
}

}  // namespace
}  // namespace sg

using namespace sg;

extern "C" stencil_status_t stencil_run_batched(int n, const stencil_plan_t *plans,
                                                const void *const *in, void *const *out,
                                                const int64_t *T, const int *fold_m,
                                                stencil_stream_t stream)
{
    if (n < 1 || !plans || !in || !out || !T) {
        set_error("stencil_run_batched: bad argument");
        return STENCIL_ERR_INVALID_ARG;
    }
    for (int g = 0; g < n; ++g) {
        const stencil_plan_s *p = plans[g];
        if (!p || !in[g] || !out[g] || T[g] < 0 || (fold_m && (fold_m[g] < 0 || fold_m[g] > 4))) {
            set_error("stencil_run_batched: bad argument for grid %d", g);
            return STENCIL_ERR_INVALID_ARG;
        }
        if (p->ndim != 2 || p->dtype != STENCIL_F32 || p->r != 1 ||
            p->device != plans[0]->device) {
            set_error("stencil_run_batched: grid %d is not a 2D FP32 radius-1 plan on one device", g);
            return STENCIL_ERR_UNSUPPORTED;
        }
    }
    stencil_plan_s *p0 = plans[0];
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> key = {5, n};
    for (int g = 0; g < n; ++g) {
        key.push_back((int64_t)(uintptr_t)plans[g]);
        key.push_back((int64_t)(uintptr_t)in[g]);
        key.push_back((int64_t)(uintptr_t)out[g]);
        key.push_back(T[g]);
        key.push_back(fold_m ? fold_m[g] : 0);
        key.push_back(plans[g]->block_b);
    }
    key.push_back(p0->wait_ms);

    if (p0->graphs.find(key) == p0->graphs.end() || !p0->use_graph) {
        // ---- flatten the batch (host, once per distinct batch)
        ensure_device_facts(p0);
        std::vector<GridPlan> gp(n);
        std::vector<BatchPass> passes;
        std::vector<CUtensorMap> maps;
        std::vector<float> coefs;
        std::map<std::tuple<const void *, int, int>, int> map_index;
        // one tile height for the whole batch: the tallest (up to 128 rows)
        // whose stages and work buffers fit for the widest halo.  Passes that
        // fuse sweeps free their stage after the first one, so one stage
        // suffices; batches of single sweeps keep two.
        int max_h = 1, nwork = 0;
        for (int g = 0; g < n; ++g) {
            if (T[g] == 0) continue;
            int m = 1, b = 1;
            choose_mb(plans[g], fold_m ? fold_m[g] : 0, &m, &b);
            for (auto &x : grid_passes(plans[g], T[g], m, b)) {
                max_h = std::max(max_h, x.first * x.second);
                nwork = std::max(nwork, x.second >= 3 ? 2 : x.second - 1);
            }
        }
        const int nstage = nwork > 0 ? 1 : 2;
        int tile_y = kBatchTileYMax;
        auto smem_for = [&](int ty, int *bf) {
            sweep2d_smem_bytes(ty, max_h, 1, bf);
            return batched_smem_bytes(*bf, nwork, nstage);
        };
        int bf_probe = 0;
        while (tile_y > 16 && (smem_for(tile_y, &bf_probe) > (size_t)p0->max_smem ||
                               tile_y + 2 * max_h > 256))
            tile_y -= 16;
        int buf_floats = 0;
        for (int g = 0; g < n; ++g) {
            stencil_plan_s *p = plans[g];
            GridPlan &G = gp[g];
            G.p = p;
            G.in = (const float *)in[g];
            G.out = (float *)out[g];
            G.T = T[g];
            choose_mb(p, fold_m ? fold_m[g] : 0, &G.m, &G.b);
            G.first_pass = (int)passes.size();
            G.npass = 0;
            G.ntiles = ceil_div(p->nx, kTileX2D) * ceil_div(p->ny, tile_y);
            if (G.T == 0) continue;
            if (!batched_variant_supported(p->r, G.m, p->pattern)) {
                set_error("stencil_run_batched: no batched kernel for m=%d", G.m);
                return STENCIL_ERR_UNSUPPORTED;
            }
            const std::vector<double> *cm = nullptr, *c1 = nullptr;
            stencil_status_t st = plan_folded(p, G.m, &cm);
            if (st == STENCIL_OK) st = plan_folded(p, 1, &c1);
            if (st == STENCIL_OK) st = ensure_padded(p);
            if (st != STENCIL_OK) return st;
            // weight blocks start on 16-byte boundaries and are padded to a
            // multiple of 4 floats: the kernel fetches them with a bulk copy
            auto add_block = [&coefs](const std::vector<double> &c) {
                const int off = (int)coefs.size();
                for (double v : c) coefs.push_back((float)v);
                while (coefs.size() % 4) coefs.push_back(0.f);
                return off;
            };
            const int off_m = add_block(*cm);
            const int off_1 = add_block(*c1);
            // passes: folded sweeps in groups of b, then the plain remainder
            const std::vector<std::pair<int, int>> mb = grid_passes(p, G.T, G.m, G.b);
            G.gw = 0;
            for (auto &x : mb) G.gw = std::max(G.gw, x.first * x.second);
            const bool out_vec4 = (p->nx % 4 == 0) && ((uintptr_t)G.out % 16 == 0);
            for (size_t i = 0; i < mb.size(); ++i) {
                const int mm = mb[i].first, bb = mb[i].second;
                const Padded &src = (i % 2 == 0) ? p->A : p->B;
                const Padded &dstP = (i % 2 == 0) ? p->B : p->A;
                const bool last = i + 1 == mb.size();
                BatchPass ps;
                memset(&ps, 0, sizeof(ps));
                ps.variant = p->pattern * 8 + mm;
                ps.b = bb;
                ps.H = bb * mm;
                ps.HX = round_up(ps.H, 4);
                ps.tiles_x = ceil_div(p->nx, kTileX2D);
                ps.ntiles = G.ntiles;
                const int box0 = kTileX2D + 2 * ps.HX, box1 = tile_y + 2 * ps.H;
                auto mk = std::make_tuple((const void *)src.alloc, box0, box1);
                auto it = map_index.find(mk);
                if (it == map_index.end()) {
                    CUtensorMap tm;
                    const int box[2] = {box0, box1};
                    if (!encode_padded_map(&tm, src, box)) {
                        set_error("stencil_run_batched: tensor map refused");
                        return STENCIL_ERR_CUDA;
                    }
                    it = map_index.emplace(mk, (int)maps.size()).first;
                    maps.push_back(tm);
                }
                ps.map = it->second;
                ps.coef = mm == G.m ? off_m : off_1;
                ps.ncoef = (2 * mm + 1) * (2 * mm + 1);
                ps.dep = i == 0 ? -1 : (int)passes.size() - 1;
                ps.nx = p->nx;
                ps.ny = p->ny;
                ps.map_x0 = src.gx;
                ps.map_y0 = src.gy;
                ps.dst = last ? G.out : dstP.origin;
                ps.dst_py = last ? p->nx : dstP.py;
                ps.dst_gw = last ? 0 : G.gw;
                ps.dst_vec4 = last ? (out_vec4 ? 1 : 0) : 1;
                int bf = 0;
                sweep2d_smem_bytes(tile_y, bb, mm, &bf);
                buf_floats = std::max(buf_floats, bf);
                passes.push_back(ps);
                G.npass += 1;
            }
        }
        // work list, round by round
        std::vector<BatchItem> items;
        int maxp = 0;
        for (auto &G : gp) maxp = std::max(maxp, G.npass);
        for (int r = 0; r < maxp; ++r)
            for (auto &G : gp)
                if (r < G.npass)
                    for (int t = 0; t < G.ntiles; ++t) items.push_back({G.first_pass + r, t});
        // imports of every grid that steps, in one launch
        std::vector<ImportJob> jobs;
        long long import_rows = 0;
        for (const GridPlan &G : gp) {
            if (G.T == 0) continue;
            jobs.push_back(make_import_job(G.p->A, G.in, G.gw, import_rows));
            import_rows += G.p->ny + 2 * G.gw;
        }
        // one device block: maps | passes | items | coefs | import jobs | done | next
        const size_t o_maps = 0;
        const size_t o_pass = round_up((int)(maps.size() * sizeof(CUtensorMap)), 256);
        const size_t o_item = o_pass + round_up((int)(passes.size() * sizeof(BatchPass) + 1), 256);
        const size_t o_coef = o_item + round_up((int)(items.size() * sizeof(BatchItem) + 1), 256);
        const size_t o_jobs = o_coef + round_up((int)(coefs.size() * sizeof(float) + 1), 256);
        const size_t o_done = o_jobs + round_up((int)(jobs.size() * sizeof(ImportJob) + 1), 256);
        const size_t total = o_done + (passes.size() + 1) * sizeof(int) + 256;
        std::vector<unsigned char> host(total, 0);
        if (!maps.empty()) memcpy(host.data() + o_maps, maps.data(), maps.size() * sizeof(CUtensorMap));
        if (!passes.empty()) memcpy(host.data() + o_pass, passes.data(), passes.size() * sizeof(BatchPass));
        if (!items.empty()) memcpy(host.data() + o_item, items.data(), items.size() * sizeof(BatchItem));
        if (!coefs.empty()) memcpy(host.data() + o_coef, coefs.data(), coefs.size() * sizeof(float));
        if (!jobs.empty()) memcpy(host.data() + o_jobs, jobs.data(), jobs.size() * sizeof(ImportJob));
        auto old = p0->batch_mem.find(key);
        if (old != p0->batch_mem.end()) {
            cudaFree(old->second);
            p0->batch_mem.erase(old);
        }
        unsigned char *dev = nullptr;
        cudaError_t e = cudaMalloc(&dev, total);
        if (e == cudaSuccess) e = cudaMemcpy(dev, host.data(), total, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (dev) cudaFree(dev);
            return cuda_fail(e, "stencil_run_batched upload");
        }
        p0->batch_mem[key] = dev;
        BatchArgs a;
        a.maps = reinterpret_cast<const CUtensorMap *>(dev + o_maps);
        a.passes = reinterpret_cast<const BatchPass *>(dev + o_pass);
        a.items = reinterpret_cast<const BatchItem *>(dev + o_item);
        a.nitems = (int)items.size();
        a.coefs = reinterpret_cast<const float *>(dev + o_coef);
        a.done = reinterpret_cast<int *>(dev + o_done);
        a.next = a.done + passes.size();
        a.tile_y = tile_y;
        a.buf_floats = buf_floats;
        a.nwork = nwork;
        a.nstage = nstage;
        a.status = p0->d_status;
        a.wait_ns = (unsigned long long)p0->wait_ms * 1000000ull;
        const size_t smem = batched_smem_bytes(buf_floats, nwork, nstage);
        if (smem > (size_t)p0->max_smem) {
            set_error("stencil_run_batched: shared memory");
            return STENCIL_ERR_UNSUPPORTED;
        }
        const int occ = std::max(1, batched_ctas_per_sm(smem));
        const int grid = std::max(1, std::min(a.nitems, occ * p0->sm_count));
        const size_t counters = (passes.size() + 1) * sizeof(int);

        const ImportJob *d_jobs = reinterpret_cast<const ImportJob *>(dev + o_jobs);
        const int njobs = (int)jobs.size();
        auto enqueue = [=](cudaStream_t st_, int *nl) -> stencil_status_t {
            for (const GridPlan &G : gp) {
                if (G.T != 0) continue;
                const cudaError_t err = cudaMemcpyAsync(
                    G.out, G.in, sizeof(float) * (size_t)G.p->nx * G.p->ny, cudaMemcpyDeviceToDevice, st_);
                if (err != cudaSuccess) return cuda_fail(err, "batched copy");
            }
            if (njobs > 0) {
                const cudaError_t err = launch_import_batch(d_jobs, njobs, import_rows, st_);
                if (err != cudaSuccess) return cuda_fail(err, "batched import");
                *nl += 1;
            }
            if (a.nitems > 0) {
                cudaError_t err = cudaMemsetAsync(a.done, 0, counters, st_);
                if (err == cudaSuccess) err = launch_batched(a, grid, smem, st_);
                if (err != cudaSuccess) return cuda_fail(err, "batched launch");
                *nl += 1;
            }
            return STENCIL_OK;
        };
        stencil_status_t st = run_maybe_graph(p0, key, s, enqueue);
        for (int g = 0; g < n; ++g) {
            plans[g]->last_m = gp[g].m;
            plans[g]->last_b = gp[g].b;
            plans[g]->last_engine = 0;
        }
        return st;
    }
    // replay of a batch seen before
    return run_maybe_graph(p0, key, s, [](cudaStream_t, int *) { return STENCIL_ERR_CUDA; });
}
