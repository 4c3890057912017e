// Autotuner for stencil_run with fold_m = 0: times candidate (engine, m, b,
// tile_y) configurations on the plan's own grid and keeps the fastest.
//
// The paper leaves the choice of blocking sizes and unrolling factor to hand
// tuning and names automatic tuning as future work (Section 4.1).  Candidates
// are pruned with the paper's scalar profitability index (Section 3.2,
// Eq. pi): a fold depth m is tried only if P = |C(E)| / |C(E_lambda)| >= 1.
// The choice is cached in the plan and in a line-per-entry JSON file keyed by
// (ndim, shape, radius, pattern, coefficient hash, dtype, GPU name, library
// version): $STENCIL_TUNE_CACHE, else $HOME/.cache/stencil_gb300/tune.jsonl.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "plan.h"

extern "C" stencil_status_t stencil_fold_cost(int ndim, int radius, const double *coeffs, int m,
                                              int64_t *out);

namespace sg {

namespace {

constexpr const char *kLibVersion = "10";
// Steps of a timed candidate run: 48 for 2D/3D; for 1D the run's own step
// count within 16..512 (96 if unknown), so that each fold's plain remainder
// pass is timed as the run will make it (a 1D run is short, and one extra
// pass is a large share of it: at T = 100, m = 6 leaves 4 plain steps where
// m = 4 leaves none).
int64_t tune_steps(const stencil_plan_s *p, int64_t T_run)
{
    if (p->ndim != 1) return 48;
    return T_run > 0 ? std::min<int64_t>(512, std::max<int64_t>(16, T_run)) : 96;
}

struct Cand {
    int engine;  // 0 CUDA core, 1 tensor core
    int m, b, ty;  // ty: 2D tile rows; 1D points per CTA tile (0 = the default)
    int tess;    // 1D: exact tessellate tiling instead of overlapped tiles
    int thr = 0;  // 2D: threads per CTA (0 = the kernel's own, 256 = two half-size CTAs)
    int ns = 0;   // 2D: TMA stages per CTA (0 = automatic)
};

uint64_t fnv1a(const void *data, size_t n, uint64_t h = 1469598103934665603ull)
{
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

std::string cache_key(const stencil_plan_s *p)
{
    cudaDeviceProp prop;
    memset(&prop, 0, sizeof(prop));
    cudaGetDeviceProperties(&prop, p->device);
    char buf[512];
    const uint64_t h = fnv1a(p->coeffs.data(), p->coeffs.size() * sizeof(double));
    // every option that changes which kernels a candidate can run is part of the key
    snprintf(buf, sizeof(buf), "%d|%lld,%lld,%lld|%d|%d|%016llx|%d|%d|cp%d|%s|%s", p->ndim,
             (long long)p->shape[0], (long long)p->shape[1], (long long)p->shape[2], p->r,
             p->pattern, (unsigned long long)h, (int)p->dtype, p->precision, p->counterparts,
             prop.name, kLibVersion);
    return buf;
}

std::string cache_path()
{
    const char *e = getenv("STENCIL_TUNE_CACHE");
    if (e && *e) return e;
    const char *home = getenv("HOME");
    if (!home || !*home) return "";
    std::string d = std::string(home) + "/.cache";
    mkdir(d.c_str(), 0755);
    d += "/stencil_gb300";
    mkdir(d.c_str(), 0755);
    return d + "/tune.jsonl";
}

bool cache_lookup(const std::string &key, Cand *c)
{
    const std::string path = cache_path();
    if (path.empty()) return false;
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    const std::string needle = "\"key\": \"" + key + "\"";
    while (fgets(line, sizeof(line), f)) {
        if (!strstr(line, needle.c_str())) continue;
        Cand t{0, 1, 1, 0, 0};
        const char *q = strstr(line, "\"engine\": ");
        if (q && sscanf(q, "\"engine\": %d, \"m\": %d, \"b\": %d, \"tile_y\": %d", &t.engine, &t.m,
                        &t.b, &t.ty) == 4) {
            const char *ts = strstr(line, "\"tess\": ");
            if (ts) sscanf(ts, "\"tess\": %d", &t.tess);
            const char *th = strstr(line, "\"threads\": ");
            if (th) sscanf(th, "\"threads\": %d, \"stages\": %d", &t.thr, &t.ns);
            *c = t;  // the last entry for a key wins
            found = true;
        }
    }
    fclose(f);
    return found;
}

void cache_store(const std::string &key, const Cand &c, double gstencil)
{
    const std::string path = cache_path();
    if (path.empty()) return;
    FILE *f = fopen(path.c_str(), "a");
    if (!f) return;
    fprintf(f,
            "{\"key\": \"%s\", \"engine\": %d, \"m\": %d, \"b\": %d, \"tile_y\": %d, \"tess\": %d, "
            "\"threads\": %d, \"stages\": %d, \"gstencil_s\": %.1f}\n",
            key.c_str(), c.engine, c.m, c.b, c.ty, c.tess, c.thr, c.ns, gstencil);
    fclose(f);
}

std::mutex g_cache_mu;
// entries read or written by this process, keyed by cache file and key
std::map<std::string, std::string> g_cache_mem;

}  // namespace

bool tune_cache_get(const std::string &key, std::string *value)
{
    std::lock_guard<std::mutex> lock(g_cache_mu);
    const std::string path = cache_path();
    auto it = g_cache_mem.find(path + "\n" + key);
    if (it != g_cache_mem.end()) {
        *value = it->second;
        return true;
    }
    if (path.empty()) return false;
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    const std::string needle = "{\"key\": \"" + key + "\", \"value\": \"";
    while (fgets(line, sizeof(line), f)) {
        if (strncmp(line, needle.c_str(), needle.size()) != 0) continue;
        const char *v = line + needle.size();
        const char *q = strchr(v, '"');
        if (!q) continue;
        *value = std::string(v, q - v);  // the last entry for a key wins
        found = true;
    }
    fclose(f);
    if (found) g_cache_mem[path + "\n" + key] = *value;
    return found;
}

void tune_cache_put(const std::string &key, const std::string &value)
{
    std::lock_guard<std::mutex> lock(g_cache_mu);
    const std::string path = cache_path();
    g_cache_mem[path + "\n" + key] = value;
    if (path.empty()) return;
    FILE *f = fopen(path.c_str(), "a");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\", \"value\": \"%s\"}\n", key.c_str(), value.c_str());
    fclose(f);
}

stencil_status_t autotune2d(stencil_plan_s *p, cudaStream_t s, int64_t T_run)
{
    const int64_t T_tune = tune_steps(p, T_run);
    // 1D choices depend on the steps they were timed over
    const std::string key = cache_key(p) + (p->ndim == 1 ? "|T" + std::to_string(T_tune) : "");
    Cand best{0, 1, 1, 0, 0};
    if (cache_lookup(key, &best)) {
        p->tuned_engine = best.engine;
        p->tuned_m = best.m;
        p->tuned_b = best.b;
        p->tuned_ty = best.ty;
        p->tuned_tess = best.tess;
        p->tuned_thr = best.thr;
        p->tuned_ns = best.ns;
        return STENCIL_OK;
    }
    // candidate list
    const int nmin = p->ndim == 1 ? p->nx : std::min(p->nx, p->ndim == 3 ? std::min(p->ny, p->nz) : p->ny);
    std::vector<Cand> cands;
    for (int m = 1; m <= (p->ndim == 1 ? 16 : 8); ++m) {
        const int R = m * p->r;
        if (2 * R + 1 > nmin || R > kGhost) break;
        if (m > 1) {
            int64_t cost[2];
            if (stencil_fold_cost(p->ndim, p->r, p->coeffs.data(), m, cost) != STENCIL_OK ||
                cost[0] < cost[1])
                continue;  // P = |C(E)| / |C(E_lambda)| < 1: folding is not profitable
        }
        if (p->dtype == STENCIL_F64 && p->ndim >= 2) {
            // FP64 2D/3D: one sweep per launch, folds up to the kernel's radius
            if (R <= (p->ndim == 3 ? kMaxRF64_3D : kMaxRF64_2D)) cands.push_back({0, m, 1, 0, 0});
        } else if (p->ndim == 1) {
            // every fold the 1D kernel has (radius up to 16): a fold costs
            // (2m+1)/m multiply-adds per step but saves m-1 shared-memory
            // round trips, and FP64 in particular is bound by the former
            // and tile sizes: short tiles give more CTAs per SM for the
            // latency-bound sweeps (measured on GB300, 2^20 points, T = 100:
            // FP32 m = 4, b = 32 overlapped 3293 GS/s with 1024-point tiles
            // against 2624 with 4096; FP64 m = 16 tessellated 238 with 256
            // against 203 with 2048), long ones waste less rim at larger R
            if (sweep1d_supported(R, p->dtype == STENCIL_F64))
                for (int b : {16, 32, 64})
                    for (int w : (p->dtype == STENCIL_F64 ? std::vector<int>{256, 512, 1024, 2048}
                                                          : std::vector<int>{512, 1024, 2048, 4096})) {
                        cands.push_back({0, m, b, w, 0});
                        // exact tessellate tiling (Section 3.4) of the same passes
                        if (tess1d_fits(p->nx, w, std::min<int64_t>(b, T_tune / m + 1), R))
                            cands.push_back({0, m, b, w, 1});
                    }
        } else if (p->ndim == 3) {
            if (sweep3d_supported(p->r, m, p->pattern)) cands.push_back({0, m, 1, 0, 0});
            if (sweep3d_tb_supported(p->r, m, p->pattern) && 2 * R <= std::min(kGhost, nmin))
                cands.push_back({0, m, 2, 0, 0});
        } else {
            // a direct kernel, or the counterpart form of c^(m) (which also
            // reaches the folds with no direct kernel, m = 6 and 8)
            const sg::CpFactor *cp = nullptr;
            const bool cp_ok = R <= kMaxR2D && plan_counterparts(p, m, &cp) == STENCIL_OK && cp->k > 0;
            if (sweep2d_supported(p->r, m, p->pattern) || cp_ok)
                for (int b : {1, 2, 3, 4, 6, 8})
                    if (b * R <= std::min(kGhost, nmin) && (m > 1 || b <= 8))
                        for (int ty : {32, 64, 96, 128, 160})
                            if (ty + 2 * b * R <= 256) {
                                cands.push_back({0, m, b, ty, 0});
                                // blocked passes also as two half-size CTAs per SM
                                // with one stage (measured on GB300: the 8192^2 box,
                                // m = 2, b = 2, 96-row tiles, 1737 against 1680 GS/s
                                // for the best one-CTA shape)
                                if (b >= 2 && ty >= 96) cands.push_back({0, m, b, ty, 0, 256, 1});
                            }
            if (m > 1 && p->precision != STENCIL_PREC_FP32 && tc2d_supported(R))
                cands.push_back({1, m, 1, 0, 0});
        }
    }
    if (cands.empty()) cands.push_back({0, 1, 1, 0, 0});
    // timing on scratch copies of a seeded-free grid (all ones keeps values finite)
    const size_t esz = p->dtype == STENCIL_F64 ? 8 : 4;
    const size_t npts = (size_t)p->nx * p->ny * p->nz;
    const size_t span = grid_extent(p);  // the caller's layout, gaps included
    void *din = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&din, span * esz);
    if (e == cudaSuccess) e = cudaMalloc(&dout, span * esz);
    if (e == cudaSuccess) e = cudaMemsetAsync(din, 0, span * esz, s);
    if (e != cudaSuccess) {
        if (din) cudaFree(din);
        return cuda_fail(e, "autotune scratch");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int saved_prec = p->precision, saved_b = p->block_b, saved_ty = p->tile_y;
    const int saved_thr = p->cta_threads, saved_ns = p->stages;
    const int saved_tess = p->tessellate, saved_t1 = p->tile_1d;
    const int saved_graph = p->use_graph;
    // 2D/3D tuning runs are not worth capturing; 1D runs are launch-bound, so
    // their candidates are timed as the captured graphs a real run replays
    // (the tessellated form's second launch per pass would otherwise look
    // dearer than it is), and those graphs are dropped afterwards
    if (p->ndim != 1) p->use_graph = 0;
    // steps per timed run: 1D runs are short and launch-bound, so their
    // candidates are timed over more steps, closer to a whole run
    const int64_t T = T_tune;
    double best_rate = -1.0;
    for (const Cand &c : cands) {
        p->precision = c.engine == 1 ? (saved_prec ? saved_prec : STENCIL_PREC_BF16X3) : STENCIL_PREC_FP32;
        p->block_b = c.b;
        if (p->ndim == 1)
            p->tile_1d = c.ty;
        else
            p->tile_y = c.ty;
        p->tessellate = c.tess;
        if (p->ndim == 2 && c.engine == 0) {
            p->cta_threads = c.thr ? c.thr : saved_thr;
            p->stages = c.ns ? c.ns : saved_ns;
        }
        stencil_status_t st = STENCIL_OK;
        auto once = [&]() {
            if (p->ndim == 1) return run1d(p, din, dout, T, c.m, s);
            if (p->dtype == STENCIL_F64)
                return run_f64nd(p, (const double *)din, (double *)dout, T, c.m, s);
            if (p->ndim == 3) return run3d(p, (const float *)din, (float *)dout, T, c.m, s);
            return run2d(p, (const float *)din, (float *)dout, T, c.m, s);
        };
        st = once();  // warm-up (also builds panels, maps and configs)
        if (st != STENCIL_OK) continue;
        cudaEventRecord(e0, s);
        for (int k = 0; k < 2 && st == STENCIL_OK; ++k) st = once();
        cudaEventRecord(e1, s);
        if (st != STENCIL_OK || cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double rate = ms > 0 ? 2.0 * (double)npts * T / (ms * 1e-3) / 1e9 : 0.0;
        if (rate > best_rate) {
            best_rate = rate;
            best = c;
        }
    }
    p->precision = saved_prec;
    p->block_b = saved_b;
    p->tile_y = saved_ty;
    p->cta_threads = saved_thr;
    p->stages = saved_ns;
    p->tessellate = saved_tess;
    p->tile_1d = saved_t1;
    p->use_graph = saved_graph;
    if (p->ndim == 1) {
        cudaStreamSynchronize(s);
        clear_graphs(p);  // they name the tuning's scratch grids
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(din);
    cudaFree(dout);
    cudaGetLastError();
    p->tuned_engine = best.engine;
    p->tuned_m = best.m;
    p->tuned_b = best.b;
    p->tuned_ty = best.ty;
    p->tuned_tess = best.tess;
    p->tuned_thr = best.thr;
    p->tuned_ns = best.ns;
    cache_store(key, best, best_rate);
    return STENCIL_OK;
}

}  // namespace sg
