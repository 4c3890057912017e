// stencil_run_batched: flattens every grid's time loop into passes and
// (pass, tile) work items, uploads them once per distinct batch, and runs the
// whole batch as one persistent kernel (after one layout-import launch for all
// grids), captured into a CUDA graph that later calls replay.
//
// Grids whose fold request is 0 get their fold depth m and blocking depth b
// from the batch autotuner below; the tile height of the batch is tuned with
// them.  The choices are cached per (base radius, stencil pattern, grid-size
// class, dtype, GPU) in the autotuner's JSON-lines cache file.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <sstream>
#include <string>
#include <tuple>
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

// Largest fold the batched kernel has for a base stencil, at most `want`,
// and no wider than the grid allows.
int clamp_m(const stencil_plan_s *p, int want)
{
    const int nmin = std::min(p->nx, p->ny);
    int m = std::max(1, want);
    while (m > 1 && (2 * m * p->r + 1 > nmin || m * p->r > kGhost ||
                     !batched_variant_supported(p->r, m, p->pattern)))
        --m;
    return m;
}

int clamp_b(const stencil_plan_s *p, int m, int want)
{
    const int max_halo = std::min(kGhost, std::min(p->nx, p->ny));
    int b = std::max(1, want);
    while (b > 1 && b * m * p->r > max_halo) --b;
    return b;
}

// Default fold and blocking depth for a grid with no tuning result (measured
// on GB300 with 96-row tiles: the folded radius-1 star prefers m = 3, the box
// m = 2, both with two fused sweeps).
void default_mb(const stencil_plan_s *p, int req_m, int *m_out, int *b_out)
{
    const int m = clamp_m(p, req_m > 0 ? req_m : (p->pattern == PAT_STAR ? 3 : 2));
    int b = p->block_b > 0 ? p->block_b : 2;
    if (req_m == 1 && p->block_b == 0) b = 1;
    *m_out = m;
    *b_out = clamp_b(p, m, b);
}

// The passes of one grid as (m, b) pairs: floor(T/m) folded sweeps in groups
// of b, then the T mod m plain steps in groups whose halo fits the ghost band.
std::vector<std::pair<int, int>> grid_passes(const stencil_plan_s *p, int64_t T, int m, int b)
{
    std::vector<std::pair<int, int>> mb;
    const int64_t q = T / m, rem = T % m;
    const int max_halo = std::min(kGhost, std::min(p->nx, p->ny));
    const int bplain = std::max(1, max_halo / p->r);
    for (int64_t d = 0; d < q; d += b) mb.push_back({m, (int)std::min<int64_t>(b, q - d)});
    for (int64_t d = 0; d < rem; d += bplain)
        mb.push_back({1, (int)std::min<int64_t>(bplain, rem - d)});
    return mb;
}

// Everything one batched launch needs, uploaded in one device block.
struct BatchBuild {
    std::vector<GridPlan> gp;
    unsigned char *dev = nullptr;
    BatchArgs a;
    int grid = 0;
    size_t smem = 0, counters = 0;
    const ImportJob *d_jobs = nullptr;
    int njobs = 0;
    long long import_rows = 0;
    int tile_y = 0;
    int threads = 0;           // CTA size of the launch
    double *d_sums = nullptr;  // per-job FP64 grid sums (centred storage), null if none
};

// Shared memory a batched CTA may use: all a CTA may opt into, or, for the
// half-size CTA, half an SM's less the 1 KB the runtime reserves per CTA, so
// that two fit on every SM.
size_t batch_smem_budget(const stencil_plan_s *p0, int threads)
{
    const size_t all = (size_t)p0->max_smem;
    if (threads == batched_threads(0) || p0->max_smem_sm <= 0) return all;
    return std::min(all, (size_t)p0->max_smem_sm / 2 - 1024);
}

// The batch's one tile height for per-grid (m, b) choices: the tallest (up to
// ty_max rows, in steps of 16) whose stages and work buffers fit for the
// widest halo.  Passes that fuse sweeps free their stage after the first one,
// so one stage suffices; batches of single sweeps keep two.
int batch_tile_height(int n, stencil_plan_s *const *plans, const int64_t *T, const int *ms,
                      const int *bs, int ty_max, size_t max_smem, int *max_h_out = nullptr,
                      int *nwork_out = nullptr)
{
    int max_h = 1, nwork = 0;
    for (int g = 0; g < n; ++g) {
        if (T[g] == 0) continue;
        for (auto &x : grid_passes(plans[g], T[g], ms[g], bs[g])) {
            max_h = std::max(max_h, x.first * x.second * plans[g]->r);
            nwork = std::max(nwork, x.second >= 3 ? 2 : x.second - 1);
        }
    }
    const int nstage = nwork > 0 ? 1 : 2;
    auto smem_for = [&](int ty) {
        int bf = 0;
        sweep2d_smem_bytes(ty, max_h, 1, &bf);
        return batched_smem_bytes(bf, nwork, nstage);
    };
    int tile_y = ty_max;
    while (tile_y > 16 && (smem_for(tile_y) > max_smem || tile_y + 2 * max_h > 256)) tile_y -= 16;
    if (max_h_out) *max_h_out = max_h;
    if (nwork_out) *nwork_out = nwork;
    return tile_y;
}

// Flattens the batch with per-grid (m, b) choices, a tile height of at most
// ty_max rows and CTAs of the given threads (256 or 512); uploads the work
// description.
stencil_status_t flatten_batch(int n, stencil_plan_s *const *plans, const void *const *in,
                               void *const *out, const int64_t *T, const int *ms, const int *bs,
                               int ty_max, int threads, BatchBuild *bb)
{
    stencil_plan_s *p0 = plans[0];
    ensure_device_facts(p0);
    std::vector<GridPlan> &gp = bb->gp;
    gp.assign(n, GridPlan{});
    std::vector<BatchPass> passes;
    std::vector<CUtensorMap> maps;
    std::vector<float> coefs;
    std::map<std::tuple<const void *, int, int>, int> map_index;
    // one tile height for the whole batch
    int max_h = 1, nwork = 0;
    const int tile_y = batch_tile_height(n, plans, T, ms, bs, ty_max, batch_smem_budget(p0, threads),
                                         &max_h, &nwork);
    const int nstage = nwork > 0 ? 1 : 2;
    auto smem_for = [&](int ty, int *bf) {
        sweep2d_smem_bytes(ty, max_h, 1, bf);
        return batched_smem_bytes(*bf, nwork, nstage);
    };
    int buf_floats = 0;
    for (int g = 0; g < n; ++g) {
        stencil_plan_s *p = plans[g];
        GridPlan &G = gp[g];
        G.p = p;
        G.in = (const float *)in[g];
        G.out = (float *)out[g];
        G.T = T[g];
        G.m = ms[g];
        G.b = bs[g];
        G.first_pass = (int)passes.size();
        G.npass = 0;
        G.ntiles = ceil_div(p->nx, kTileX2D) * ceil_div(p->ny, tile_y);
        if (G.T == 0) continue;
        if (!batched_variant_supported(p->r, G.m, p->pattern) ||
            !batched_variant_supported(p->r, 1, p->pattern)) {
            set_error("stencil_run_batched: no batched kernel for r=%d m=%d", p->r, G.m);
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
            std::vector<float> w(c.size());
            round_f32_mass(c.data(), c.size(), c.size() / 2, w.data());
            for (float v : w) coefs.push_back(v);
            while (coefs.size() % 4) coefs.push_back(0.f);
            return off;
        };
        const int off_m = add_block(*cm);
        const int off_1 = add_block(*c1);
        // passes: folded sweeps in groups of b, then the plain remainder
        const std::vector<std::pair<int, int>> mb = grid_passes(p, G.T, G.m, G.b);
        G.gw = 0;
        for (auto &x : mb) G.gw = std::max(G.gw, x.first * x.second * p->r);
        const bool out_vec4 = grid_vec4(p, G.out);
        for (size_t i = 0; i < mb.size(); ++i) {
            const int mm = mb[i].first, bb_ = mb[i].second;
            const Padded &src = (i % 2 == 0) ? p->A : p->B;
            const Padded &dstP = (i % 2 == 0) ? p->B : p->A;
            const bool last = i + 1 == mb.size();
            BatchPass ps;
            memset(&ps, 0, sizeof(ps));
            ps.variant = batched_variant_id(p->r, mm, p->pattern);
            ps.b = bb_;
            ps.H = bb_ * mm * p->r;
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
            ps.ncoef = (2 * mm * p->r + 1) * (2 * mm * p->r + 1);
            ps.dep = i == 0 ? -1 : (int)passes.size() - 1;
            ps.nx = p->nx;
            ps.ny = p->ny;
            ps.map_x0 = src.gx;
            ps.map_y0 = src.gy;
            ps.dst = last ? G.out : dstP.origin;
            ps.dst_py = last ? p->pitch_y : dstP.py;
            ps.dst_gw = last ? 0 : G.gw;
            ps.dst_vec4 = last ? (out_vec4 ? 1 : 0) : 1;
            int bf = 0;
            sweep2d_smem_bytes(tile_y, bb_, mm * p->r, &bf);
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
    // imports of every grid that steps, in one launch; grids of centred plans
    // are stored minus their mean (an FP64 sum per grid in the sums block)
    // and get mean * (sum c)^T added to their outputs at the end
    std::vector<ImportJob> jobs;
    long long import_rows = 0;
    bool any_centred = false;
    for (const GridPlan &G : gp) {
        if (G.T == 0) continue;
        ImportJob j = make_import_job(G.p->A, G.in, G.gw, import_rows, G.p->pitch_y);
        if (G.p->center) {
            double sc = 0.0;
            for (double v : G.p->coeffs) sc += v;
            j.inv_n = 1.0 / ((double)G.p->nx * G.p->ny);
            j.out = G.out;
            j.out_py = G.p->pitch_y;
            j.factor = pow(sc, (double)G.T);
            any_centred = true;  // mean_sum is set once the device block exists
        }
        jobs.push_back(j);
        import_rows += G.p->ny + 2 * G.gw;
    }
    // one device block: maps | passes | items | coefs | import jobs | sums | done | next
    const size_t o_maps = 0;
    const size_t o_pass = round_up((int)(maps.size() * sizeof(CUtensorMap)), 256);
    const size_t o_item = o_pass + round_up((int)(passes.size() * sizeof(BatchPass) + 1), 256);
    const size_t o_coef = o_item + round_up((int)(items.size() * sizeof(BatchItem) + 1), 256);
    const size_t o_jobs = o_coef + round_up((int)(coefs.size() * sizeof(float) + 1), 256);
    const size_t o_sums = o_jobs + round_up((int)(jobs.size() * sizeof(ImportJob) + 1), 256);
    const size_t o_done = o_sums + round_up((int)(jobs.size() * sizeof(double) + 1), 256);
    const size_t total = o_done + (passes.size() + 1) * sizeof(int) + 256;
    std::vector<unsigned char> host(total, 0);
    if (!maps.empty()) memcpy(host.data() + o_maps, maps.data(), maps.size() * sizeof(CUtensorMap));
    if (!passes.empty()) memcpy(host.data() + o_pass, passes.data(), passes.size() * sizeof(BatchPass));
    if (!items.empty()) memcpy(host.data() + o_item, items.data(), items.size() * sizeof(BatchItem));
    if (!coefs.empty()) memcpy(host.data() + o_coef, coefs.data(), coefs.size() * sizeof(float));
    const size_t smem = batched_smem_bytes(buf_floats, nwork, nstage);
    if (smem > (size_t)p0->max_smem) {
        set_error("stencil_run_batched: shared memory");
        return STENCIL_ERR_UNSUPPORTED;
    }
    unsigned char *dev = nullptr;
    cudaError_t e = cudaMalloc(&dev, total);
    double *d_sums = reinterpret_cast<double *>(dev + o_sums);
    for (size_t k = 0; k < jobs.size(); ++k)
        if (jobs[k].out) jobs[k].mean_sum = d_sums + k;
    if (!jobs.empty()) memcpy(host.data() + o_jobs, jobs.data(), jobs.size() * sizeof(ImportJob));
    if (e == cudaSuccess) e = cudaMemcpy(dev, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (dev) cudaFree(dev);
        return cuda_fail(e, "stencil_run_batched upload");
    }
    bb->dev = dev;
    BatchArgs &a = bb->a;
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
    a.fault_withhold_dep = p0->fault_withhold_dep;
    bb->smem = smem;
    bb->threads = threads;
    const int occ = std::max(1, batched_ctas_per_sm(smem, bb->threads));
    bb->grid = std::max(1, std::min(a.nitems, occ * p0->sm_count));
    bb->counters = (passes.size() + 1) * sizeof(int);
    bb->d_jobs = reinterpret_cast<const ImportJob *>(dev + o_jobs);
    bb->njobs = (int)jobs.size();
    bb->d_sums = any_centred ? d_sums : nullptr;
    bb->import_rows = import_rows;
    bb->tile_y = tile_y;
    return STENCIL_OK;
}

// The batch's work in stream order: copies of the grids with T = 0, the one
// import launch, the counter reset and the persistent launch.
stencil_status_t enqueue_batch(const BatchBuild &bb, cudaStream_t st_, int *nl)
{
    for (const GridPlan &G : bb.gp) {
        if (G.T != 0) continue;
        const cudaError_t err = copy_grid(G.p, G.out, G.in, cudaMemcpyDeviceToDevice, st_);
        if (err != cudaSuccess) return cuda_fail(err, "batched copy");
    }
    if (bb.njobs > 0 && bb.d_sums) {
        cudaError_t err = cudaMemsetAsync(bb.d_sums, 0, sizeof(double) * bb.njobs, st_);
        if (err == cudaSuccess) err = launch_grid_sum_batch(bb.d_jobs, bb.njobs, bb.import_rows, st_);
        if (err != cudaSuccess) return cuda_fail(err, "batched grid sums");
        *nl += 1;
    }
    if (bb.njobs > 0) {
        const cudaError_t err = launch_import_batch(bb.d_jobs, bb.njobs, bb.import_rows, st_);
        if (err != cudaSuccess) return cuda_fail(err, "batched import");
        *nl += 1;
    }
    if (bb.a.nitems > 0) {
        cudaError_t err = cudaMemsetAsync(bb.a.done, 0, bb.counters, st_);
        if (err == cudaSuccess) err = launch_batched(bb.a, bb.grid, bb.smem, bb.threads, st_);
        if (err != cudaSuccess) return cuda_fail(err, "batched launch");
        *nl += 1;
    }
    if (bb.njobs > 0 && bb.d_sums) {
        const cudaError_t err = launch_add_bias_batch(bb.d_jobs, bb.njobs, bb.import_rows, st_);
        if (err != cudaSuccess) return cuda_fail(err, "batched bias");
        *nl += 1;
    }
    return STENCIL_OK;
}

// ---- batch autotuner ----------------------------------------------------------

// A class of automatic grids that share one (m, b) choice: same base radius
// and pattern, and a grid size within a factor of two (log2 of the area).
struct ClassKey {
    int r, pattern, size_class;
    bool operator<(const ClassKey &o) const
    {
        return std::tie(r, pattern, size_class) < std::tie(o.r, o.pattern, o.size_class);
    }
};

ClassKey class_of(const stencil_plan_s *p)
{
    return {p->r, p->pattern, (int)floor(log2((double)p->nx * p->ny))};
}

std::string class_cache_key(const ClassKey &k, const char *gpu)
{
    char buf[256];
    snprintf(buf, sizeof(buf), "batched|2d|r%d|pat%d|area2^%d|f32|%s", k.r, k.pattern,
             k.size_class, gpu);
    return buf;
}

// Event-timed duration of one launch of the batch with the given choices
// (after one untimed launch), or a negative value if it cannot run.
double time_batch(int n, stencil_plan_s *const *plans, const void *const *in, void *const *out,
                  const int64_t *T, const std::vector<int> &ms, const std::vector<int> &bs,
                  int ty, int threads, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1)
{
    BatchBuild bb;
    if (flatten_batch(n, plans, in, out, T, ms.data(), bs.data(), ty, threads, &bb) != STENCIL_OK) {
        if (bb.dev) cudaFree(bb.dev);
        return -1.0;
    }
    int nl = 0;
    stencil_status_t st = enqueue_batch(bb, s, &nl);
    if (st == STENCIL_OK) cudaEventRecord(e0, s);
    if (st == STENCIL_OK) st = enqueue_batch(bb, s, &nl);
    if (st == STENCIL_OK) cudaEventRecord(e1, s);
    float ms_el = -1.f;
    if (st == STENCIL_OK && cudaEventSynchronize(e1) == cudaSuccess)
        cudaEventElapsedTime(&ms_el, e0, e1);
    cudaStreamSynchronize(s);
    cudaFree(bb.dev);
    cudaGetLastError();
    return st == STENCIL_OK ? (double)ms_el : -1.0;
}

// Chooses (m, b) for every automatic grid (auto_g[g]), the batch's tile
// height and its CTA shape: cached choices where the cache has them, else,
// for each tile height and shape (128, 96 and 64 rows with 512-thread CTAs;
// 80 and 64 rows with two 256-thread CTAs per SM, whose tiles must fit half
// an SM's shared memory), one class at a time among the choices that keep
// that height; then the starting set, the tuned sets and each tuned set on
// the other CTA shape are timed as whole batches in turns, and a tuned set
// replaces the starting one only if it is 2 % faster (two timings of one set
// agree to about 0.1 %).  A first plan with cta_threads 256 limits the search to the
// half-size CTA.  Every candidate is timed as a batched launch that writes
// scratch outputs, never the caller's grids.
stencil_status_t tune_batch(int n, stencil_plan_s *const *plans, const void *const *in,
                            const int64_t *T, const std::vector<bool> &auto_g,
                            std::vector<int> &ms, std::vector<int> &bs, int *ty_out,
                            int *thr_out, cudaStream_t s)
{
    stencil_plan_s *p0 = plans[0];
    const int thr_wide = batched_threads(0), thr_half = batched_threads(256);
    const bool half_only = p0->cta_threads == 256;
    const int thr_start = half_only ? thr_half : thr_wide;
    *ty_out = kBatchTileYMax;
    *thr_out = thr_start;
    cudaDeviceProp prop;
    memset(&prop, 0, sizeof(prop));
    cudaGetDeviceProperties(&prop, p0->device);
    std::map<ClassKey, std::vector<int>> classes;
    for (int g = 0; g < n; ++g)
        if (auto_g[g] && T[g] > 0) classes[class_of(plans[g])].push_back(g);
    if (classes.empty()) return STENCIL_OK;
    auto apply = [&](const ClassKey &k, int m, int b) {
        for (int g : classes[k]) {
            ms[g] = clamp_m(plans[g], m);
            bs[g] = clamp_b(plans[g], ms[g], b);
        }
    };
    // The cache holds one entry per batch composition (its set of classes):
    // "tile_y threads" and then every class's "m b" in class order.  Class
    // entries (one per class, "m b") are written too and read only for a
    // composition entry without the per-class choices.  Another batch's
    // choice for a class (e.g. b = 3, fine for a few small grids) can shorten
    // every tile of a batch it does not suit, so a new composition is tuned
    // from the default choices.
    std::string tile_key = "batched-tile|";
    for (auto &kv : classes) {
        char cls[64];
        snprintf(cls, sizeof(cls), "r%d.p%d.a%d;", kv.first.r, kv.first.pattern,
                 kv.first.size_class);
        tile_key += cls;
    }
    if (half_only) tile_key += "t256;";
    tile_key += std::string("|") + prop.name;
    int ty = kBatchTileYMax, thr = thr_start;
    bool all_cached = false;
    {
        std::string v;
        int t = 0, h = 0;
        if (tune_cache_get(tile_key, &v) && sscanf(v.c_str(), "%d %d", &t, &h) == 2 && t >= 16 &&
            t <= kBatchTileYMax && (h == thr_wide || h == thr_half) && !(half_only && h != thr_half)) {
            all_cached = true;
            // the composition's own per-class choices, if it carries them
            std::vector<int> own;
            {
                std::istringstream is(v);
                int x = 0;
                while (is >> x) own.push_back(x);
            }
            const bool has_own = own.size() == 2 + 2 * classes.size();
            std::vector<std::pair<ClassKey, std::pair<int, int>>> got;
            size_t ci = 0;
            for (auto &kv : classes) {
                std::string cv;
                int m = 0, b = 0;
                if (has_own) {
                    m = own[2 + 2 * ci];
                    b = own[3 + 2 * ci];
                } else if (!(tune_cache_get(class_cache_key(kv.first, prop.name), &cv) &&
                             sscanf(cv.c_str(), "%d %d", &m, &b) == 2)) {
                    m = b = 0;
                }
                ++ci;
                if (m >= 1 && b >= 1)
                    got.push_back({kv.first, {m, b}});
                else
                    all_cached = false;
            }
            if (all_cached) {
                for (auto &g : got) apply(g.first, g.second.first, g.second.second);
                ty = t;
                thr = h;
            }
        }
    }
    if (all_cached || !p0->autotune) {
        *ty_out = ty;
        *thr_out = thr;
        return STENCIL_OK;
    }
    // scratch outputs in each grid's own layout
    std::vector<size_t> off(n, 0);
    size_t total = 0;
    for (int g = 0; g < n; ++g) {
        off[g] = total;
        total += (grid_extent(plans[g]) * 4 + 255) / 256 * 256;
    }
    unsigned char *scratch = nullptr;
    cudaError_t e = cudaMalloc(&scratch, std::max<size_t>(total, 256));
    if (e != cudaSuccess) return cuda_fail(e, "batch autotune scratch");
    std::vector<void *> sout(n);
    for (int g = 0; g < n; ++g) sout[g] = scratch + off[g];
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // each timing is the best of two launches
    auto best_of_two = [&](int nn, stencil_plan_s *const *pl, const void *const *ii,
                           void *const *oo, const int64_t *tt, const std::vector<int> &mm,
                           const std::vector<int> &bb_, int ty_, int thr_) {
        const double t0 = time_batch(nn, pl, ii, oo, tt, mm, bb_, ty_, thr_, s, e0, e1);
        const double t1 = time_batch(nn, pl, ii, oo, tt, mm, bb_, ty_, thr_, s, e0, e1);
        return (t0 > 0 && t1 > 0) ? std::min(t0, t1) : -1.0;
    };
    ensure_device_facts(p0);
    // The batch shares one tile height, and a class whose halo or work
    // buffers need more shared memory shortens every grid's tiles.  So each
    // candidate height is tried in turn: the classes are tuned one at a time
    // on their own grids (every supported m, b in 1..3) among the choices
    // that keep that height, and the whole batch is then timed with them.
    // The starting choices (defaults, or a class's cached choice) at the
    // tallest tile that fits them are the baseline a tuned set must beat.
    // Per class, the (m, b) to cache: the largest over its grids, which the
    // clamp to a small grid's size may have lowered.
    std::map<ClassKey, std::pair<int, int>> best_choice;
    for (auto &kv : classes) {
        int m = 1, b = 1;
        for (int g : kv.second) {
            m = std::max(m, ms[g]);
            b = std::max(b, bs[g]);
        }
        best_choice[kv.first] = {m, b};
    }
    std::vector<int> best_ms = ms, best_bs = bs;
    int best_ty = batch_tile_height(n, plans, T, ms.data(), bs.data(), kBatchTileYMax,
                                    batch_smem_budget(p0, thr_start));
    // The starting set and the tuned sets (one per tile height) are timed as
    // whole batches in turns, five rounds of one launch each, so that drift
    // over the tuning run affects them alike; each keeps its best launch, and
    // a tuned set must beat the starting one by 2 %.
    struct SetChoice {
        std::vector<int> ms, bs;
        int ty, thr;
        std::map<ClassKey, std::pair<int, int>> choice;
        double t;
    };
    std::vector<SetChoice> sets;
    sets.push_back({ms, bs, best_ty, thr_start, best_choice, -1.0});
    const std::pair<int, int> shapes[] = {{128, thr_wide}, {96, thr_wide}, {64, thr_wide},
                                          {80, thr_half}, {64, thr_half}};
    for (const auto &shape : shapes) {
        const int ty_c = shape.first, thr_c = shape.second;
        if (half_only && thr_c != thr_half) continue;
        const size_t max_smem = batch_smem_budget(p0, thr_c);
        std::vector<int> tm = ms, tb = bs;
        std::map<ClassKey, std::pair<int, int>> choice = best_choice;
        for (auto &kv : classes) {
            const ClassKey &k = kv.first;
            const std::vector<int> &gs = kv.second;
            std::vector<stencil_plan_s *> cp;
            std::vector<const void *> ci;
            std::vector<void *> co;
            std::vector<int64_t> ct;
            for (int g : gs) {
                cp.push_back(plans[g]);
                ci.push_back(in[g]);
                co.push_back(sout[g]);
                ct.push_back(T[g]);
            }
            std::vector<int> cm(gs.size()), cb(gs.size());
            int bm = 0, bbst = 0;
            double best = -1.0;
            for (int m = 1; m <= 4; ++m) {
                if (!batched_variant_supported(k.r, m, k.pattern) ||
                    clamp_m(plans[gs[0]], m) != m)
                    continue;
                for (int b = 1; b <= 3; ++b) {
                    for (size_t i = 0; i < gs.size(); ++i) {
                        cm[i] = clamp_m(cp[i], m);
                        cb[i] = clamp_b(cp[i], cm[i], b);
                    }
                    if (batch_tile_height((int)gs.size(), cp.data(), ct.data(), cm.data(),
                                          cb.data(), ty_c, max_smem) != ty_c)
                        continue;
                    const double t = best_of_two((int)gs.size(), cp.data(), ci.data(),
                                                 co.data(), ct.data(), cm, cb, ty_c, thr_c);
                    if (t > 0 && (best < 0 || t < best)) {
                        best = t;
                        bm = m;
                        bbst = b;
                    }
                }
            }
            if (bm == 0) continue;  // no choice keeps this height: the class keeps its start
            choice[k] = {bm, bbst};
            for (int g : gs) {
                tm[g] = clamp_m(plans[g], bm);
                tb[g] = clamp_b(plans[g], tm[g], bbst);
            }
        }
        const int ty_real = batch_tile_height(n, plans, T, tm.data(), tb.data(), ty_c, max_smem);
        sets.push_back({tm, tb, ty_real, thr_c, choice, -1.0});
    }
    // every tuned set also on the other CTA shape, at the tallest tile that
    // shape fits, unless an identical set is already listed
    if (!half_only) {
        const size_t ntuned = sets.size();
        for (size_t i = 1; i < ntuned; ++i) {
            SetChoice c = sets[i];
            c.thr = c.thr == thr_wide ? thr_half : thr_wide;
            c.ty = batch_tile_height(n, plans, T, c.ms.data(), c.bs.data(), kBatchTileYMax,
                                     batch_smem_budget(p0, c.thr));
            bool dup = false;
            for (const SetChoice &o : sets)
                dup = dup || (o.thr == c.thr && o.ty == c.ty && o.ms == c.ms && o.bs == c.bs);
            if (!dup) sets.push_back(c);
        }
    }
    for (int round = 0; round < 5; ++round)
        for (SetChoice &c : sets) {
            const double t =
                time_batch(n, plans, in, sout.data(), T, c.ms, c.bs, c.ty, c.thr, s, e0, e1);
            if (t > 0 && (c.t < 0 || t < c.t)) c.t = t;
        }
    size_t pick = 0;
    for (size_t i = 1; i < sets.size(); ++i)
        if (sets[i].t > 0 && sets[0].t > 0 && sets[i].t < 0.98 * sets[0].t &&
            (pick == 0 || sets[i].t < sets[pick].t))
            pick = i;
    std::vector<int> best_ms2 = sets[pick].ms, best_bs2 = sets[pick].bs;
    best_ty = sets[pick].ty;
    thr = sets[pick].thr;
    best_choice = sets[pick].choice;
    best_ms = best_ms2;
    best_bs = best_bs2;
    ms = best_ms;
    bs = best_bs;
    ty = best_ty;
    for (auto &kv : best_choice) {
        char v[32];
        snprintf(v, sizeof(v), "%d %d", kv.second.first, kv.second.second);
        tune_cache_put(class_cache_key(kv.first, prop.name), v);
    }
    std::string tv = std::to_string(ty) + " " + std::to_string(thr);
    for (auto &kv : classes) {
        const std::pair<int, int> &mb = best_choice[kv.first];
        tv += " " + std::to_string(mb.first) + " " + std::to_string(mb.second);
    }
    tune_cache_put(tile_key, tv);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scratch);
    *ty_out = ty;
    *thr_out = thr;
    return STENCIL_OK;
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
        if (!p || !in[g] || !out[g] || T[g] < 0 || (fold_m && (fold_m[g] < 0 || fold_m[g] > 16))) {
            set_error("stencil_run_batched: bad argument for grid %d", g);
            return STENCIL_ERR_INVALID_ARG;
        }
        if (p->ndim != 2 || p->dtype != STENCIL_F32 || !batched_variant_supported(p->r, 1, p->pattern) ||
            p->device != plans[0]->device) {
            set_error("stencil_run_batched: grid %d is not a 2D FP32 plan of radius 1 or 2 on "
                      "one device", g);
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
        key.push_back(plans[g]->center);
    }
    key.push_back(p0->wait_ms);
    key.push_back(p0->fault_withhold_dep);
    key.push_back(p0->autotune);
    key.push_back(p0->tile_y);
    key.push_back(p0->cta_threads);

    if (p0->use_graph && p0->graphs.find(key) != p0->graphs.end())  // a batch seen before
        return run_maybe_graph(p0, key, s, [](cudaStream_t, int *) { return STENCIL_ERR_CUDA; });

    // ---- per-grid fold and blocking depth: requested (a fold the batched
    // kernel lacks is lowered to the largest it has; the result is the same
    // T steps), or tuned
    std::vector<int> ms(n, 1), bs(n, 1);
    std::vector<bool> auto_g(n, false);
    for (int g = 0; g < n; ++g) {
        const int req = fold_m ? fold_m[g] : 0;
        default_mb(plans[g], req, &ms[g], &bs[g]);
        // a grid is tuned when its fold is automatic and its plan pins no depth
        auto_g[g] = req == 0 && plans[g]->block_b == 0;
    }
    int ty = kBatchTileYMax, thr = batched_threads(0);
    stencil_status_t st = tune_batch(n, plans, in, T, auto_g, ms, bs, &ty, &thr, s);
    if (st != STENCIL_OK) return st;
    // the first plan's tile_y option pins the batch's tile height, and its
    // cta_threads option (256) the half-size CTA
    if (p0->tile_y > 0) ty = std::min(p0->tile_y, kBatchTileYMax);
    if (p0->cta_threads == 256) thr = batched_threads(256);

    // ---- flatten the batch (host, once per distinct batch)
    BatchBuild bb;
    st = flatten_batch(n, plans, in, out, T, ms.data(), bs.data(), ty, thr, &bb);
    if (st != STENCIL_OK) {
        if (bb.dev) cudaFree(bb.dev);
        return st;
    }
    auto old = p0->batch_mem.find(key);
    if (old != p0->batch_mem.end()) {
        cudaFree(old->second);
        p0->batch_mem.erase(old);
    }
    p0->batch_mem[key] = bb.dev;
    st = run_maybe_graph(p0, key, s,
                         [bb](cudaStream_t st_, int *nl) { return enqueue_batch(bb, st_, nl); });
    for (int g = 0; g < n; ++g) {
        plans[g]->last_m = ms[g];
        plans[g]->last_b = bs[g];
        plans[g]->last_ty = bb.tile_y;
        plans[g]->last_threads = bb.threads;
        plans[g]->last_engine = 0;
    }
    return st;
}
