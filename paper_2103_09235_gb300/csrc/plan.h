// The plan object behind the opaque stencil_plan_t, shared by the host
// translation units of the library.
#pragma once

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/stencil.h"
#include "internal.h"

namespace sg {
// Counterpart form of c^(m): k separable terms sum_k u_k (x) v_k (u over row
// offsets, v over column offsets, 2R+1 each); k = 0: the direct form.
struct CpFactor {
    int k = 0;
    std::vector<double> u, v;
};
}  // namespace sg

struct stencil_plan_s {
    int device = 0;
    int ndim = 0;
    int64_t shape[3] = {1, 1, 1};  // C order, as given
    int nx = 1, ny = 1, nz = 1;    // x fastest
    // strides of the caller's grids (elements): rows pitch_y, planes pitch_z
    // apart; nx and nx*ny unless stencil_plan_ex gave others
    int64_t pitch_y = 1, pitch_z = 1;
    int r = 1;
    stencil_dtype_t dtype = STENCIL_F32;
    std::vector<double> coeffs;  // (2r+1)^ndim, axis order (z, y, x)
    int pattern = sg::PAT_BOX;

    // options
    int precision = STENCIL_PREC_FP32;
    int block_b = 0;
    int tile_y = 0;
    int stages = 0;  // TMA stages per CTA of the 2D sweep (0 = automatic)
    int cta_threads = 0;  // threads per CTA of the 2D sweep (0 = automatic, or 256)
    int z_chunk = 0;  // output planes per CTA of the 3D sweeps (0 = automatic)
    int tile_1d = 0;  // points per CTA of the 1D sweeps (0 = automatic)
    int persistent = -1;  // 3D single sweeps in one persistent launch: 1 always, 0 never, -1 automatic
    int tc_center = 1;
    int tc_tma_store = 1;
    int tc_form = 0;  // tensor cores: 0 by folded radius, 1 one MMA per row offset, 2 grouped
    int counterparts = 0;  // 2D counterpart form: 0 when cheaper, 1 always (rank <= 2), 2 never
    int autotune = 1;
    long long wait_ms = 2000;
    int fault_withhold_copy = 0;  // test hook, see stencil_plan_set_option
    int fault_withhold_dep = 0;   // test hook: batched dependency counters never complete
    int fault_withhold_mma = 0;   // test hook: tensor-core MMA completions never signalled

    // FP64 folded weights computed on the GPU, by m
    std::map<int, std::vector<double>> folded;
    // their counterpart form (2D), by m
    std::map<int, sg::CpFactor> cp;

    // device state
    int *d_status = nullptr;
    sg::Padded A, B;                          // 2D / 3D working grids
    void *d1a = nullptr, *d1b = nullptr;      // 1D working grids
    void *d1p0 = nullptr, *d1p1 = nullptr;    // 1D tessellation: edge values between stages
    int tessellate = 0;                       // 1D passes by exact tessellate tiling
    int center = 1;                           // 2D/3D CUDA-core runs store the grid minus its mean
    void *stage_in = nullptr, *stage_out = nullptr;  // host-pointer staging
    double *d_acc = nullptr;                  // small FP64 reduction buffer
    std::map<int, uint16_t *> panels;         // tensor-core Toeplitz panels by m
    std::map<int, double> panel_sum;          // FP64 sum of the folded weights by m
    std::map<std::tuple<const void *, int, int, int>, CUtensorMap> maps;
    size_t scratch_bytes = 0;

    // cached launch facts
    int sm_count = 0, max_smem = 0, max_smem_sm = 0;  // SMs, shared bytes per CTA (opt-in) and per SM
    struct PassCfg {
        int ty, bf, grid, nstages, threads;
        size_t smem;
    };
    // (m, b, tile/stage/thread options and counterpart terms)
    std::map<std::tuple<int, int, int>, PassCfg> pass_cfg;

    // executable graphs of whole runs, keyed by everything a run enqueues
    struct GraphEnt {
        cudaGraphExec_t exec;
        int launches;
    };
    std::map<std::vector<int64_t>, GraphEnt> graphs;
    cudaStream_t cap_stream = nullptr;
    int use_graph = 1;
    // device work lists of batched runs led by this plan, by batch key
    std::map<std::vector<int64_t>, unsigned char *> batch_mem;
    // multi-pass 3D sweeps: per (R, z chunk, halo columns) the pieces' pass
    // counters and neighbour lists
    std::map<std::tuple<int, int, int>, int *> q3_mem;

    // bookkeeping
    long long launches = 0;
    int last_m = 0, last_b = 0, last_engine = 0;
    int last_tc_form = 0;  // tensor-core kernel of the last tensor-core run (1 or 2)
    int last_ty = 0;  // tile height of the last 2D CUDA-core run's first pass
    int last_threads = 0;  // threads per CTA: the last batched launch, or the last 2D run's first pass
    int last_stages = 0;   // TMA stages per CTA of the last 2D CUDA-core run's first pass
    int last_persist = 0;  // 1 if the last 3D run used the multi-pass persistent launch
    int last_cp = 0;  // counterpart terms of the last 2D CUDA-core run's folded passes (0 = direct)
    int last_tess = 0;  // 1 if the last 1D run's folded passes used exact tessellate tiling
    // autotuner choice for fold_m = 0: m, b, tile_y, engine (m = 0: not tuned yet)
    int tuned_m = 0, tuned_b = 0, tuned_ty = 0, tuned_engine = 0, tuned_tess = 0;
    int tuned_thr = 0, tuned_ns = 0;  // 2D: CTA size and stages of the tuned choice
};

namespace sg {

// Elements a caller's grid spans: the last point's index plus one.
inline size_t grid_extent(const stencil_plan_s *p)
{
    return (size_t)(p->nz - 1) * p->pitch_z + (size_t)(p->ny - 1) * p->pitch_y + p->nx;
}

// Whether a caller's grid is dense (no gaps between rows or planes).
inline bool grid_dense(const stencil_plan_s *p)
{
    return p->pitch_y == p->nx && (p->ndim < 3 || p->pitch_z == (int64_t)p->nx * p->ny);
}

// Whether 16-byte stores of whole rows reach every row of a caller's grid.
inline bool grid_vec4(const stencil_plan_s *p, const void *base)
{
    return p->nx % 4 == 0 && p->pitch_y % 4 == 0 && (p->ndim < 3 || p->pitch_z % 4 == 0) &&
           (uintptr_t)base % 16 == 0;
}

// One axis of the multi-pass sweep's neighbour lists.  Tile t (of ntile
// tiles of S cells over n cells) reads the cells [lo(t), hi(t)) of the
// previous pass's grid, ghost cells standing for their periodic images.  Its
// list holds the tiles owning such a cell (whose output it reads) and the
// tiles whose window holds one of its cells (whose reads of the grid it will
// overwrite two passes on), -1 padded to kDep3 entries.  False if a list
// would be longer.
template <class Window>
inline bool axis_deps(int n, int S, int ntile, Window window, int *out)
{
    std::vector<std::vector<char>> rel(ntile, std::vector<char>(ntile, 0));
    for (int t = 0; t < ntile; ++t) {
        const std::pair<int, int> w = window(t);
        for (int c = w.first; c < w.second; ++c) {
            const int o = (((c % n) + n) % n) / S;
            rel[t][o] = 1;  // t reads o's cells
            rel[o][t] = 1;  // o's writes replace what t read
        }
    }
    for (int t = 0; t < ntile; ++t) {
        int k = 0;
        for (int o = 0; o < ntile; ++o) {
            if (!rel[t][o]) continue;
            if (k == kDep3) return false;
            out[t * kDep3 + k++] = o;
        }
        for (; k < kDep3; ++k) out[t * kDep3 + k] = -1;
    }
    return true;
}

// Copies the nx x ny x nz points of a caller-layout grid (both sides use the
// plan's pitches), skipping the gaps between rows and planes.
cudaError_t copy_grid(const stencil_plan_s *p, void *dst, const void *src, cudaMemcpyKind kind,
                      cudaStream_t s);

// Thread-local error detail.
void set_error(const char *fmt, ...);
stencil_status_t cuda_fail(cudaError_t e, const char *what);

// FP64 folded weights c^(m) of the plan, computed on the GPU once per m.
stencil_status_t plan_folded(stencil_plan_s *p, int m, const std::vector<double> **out);
stencil_status_t ensure_padded(stencil_plan_s *p);
const CUtensorMap *plan_map(stencil_plan_s *p, const Padded &P, const int *box);

// Per-dimension drivers of stencil_run on device pointers.
stencil_status_t run1d(stencil_plan_s *p, const void *in, void *out, int64_t T, int m,
                       cudaStream_t s);
stencil_status_t run2d(stencil_plan_s *p, const float *in, float *out, int64_t T, int m,
                       cudaStream_t s);
stencil_status_t run3d(stencil_plan_s *p, const float *in, float *out, int64_t T, int m,
                       cudaStream_t s);
// Folded 3D sweeps on the tensor cores (explicit m > 1 with a BF16 or TF32
// precision): per sweep, one per-offset tensor-core launch per plane offset.
stencil_status_t run3d_tc(stencil_plan_s *p, const float *in, float *out, int64_t T, int m,
                          cudaStream_t s);
// One 3D CUDA-core pass of b (1 or 2) fused sweeps of c = c^(m) from padded
// grid src to dst (padded origin or the caller's grid).
stencil_status_t launch_pass3d(stencil_plan_s *p, const Padded &src, int m, int b,
                               const std::vector<double> &c, float *dst, int64_t dst_py,
                               int64_t dst_pz, int dst_gw, bool dst_vec4, cudaStream_t s);
// FP64 2D and 3D grids (k_sweep_f64.cu), plain or folded.
stencil_status_t run_f64nd(stencil_plan_s *p, const double *in, double *out, int64_t T, int m,
                           cudaStream_t s);
// T_run: the steps of the run that asked (1D candidates are timed over them, capped).
stencil_status_t autotune2d(stencil_plan_s *p, cudaStream_t s, int64_t T_run = 0);

void clear_graphs(stencil_plan_s *p);
// cpk: counterpart terms of the pass (0 = direct form); cp: their factors.
stencil_status_t pass2d_config(stencil_plan_s *p, int m, int b, stencil_plan_s::PassCfg *cfg,
                               int cpk = 0);
stencil_status_t launch_pass2d(stencil_plan_s *p, const Padded &src, int m, int b,
                               const std::vector<double> &c, float *dst, int64_t dst_py,
                               int dst_gw, bool dst_vec4, cudaStream_t s,
                               const CpFactor *cp = nullptr);
// Counterpart factorisation of W x W folded weights (complete pivoting):
// returns the rank K (max_k + 1 when above max_k) and fills K rows of u, v.
int cp_factor(const double *c, int W, int max_k, double *u, double *v);
stencil_status_t plan_counterparts(stencil_plan_s *p, int m, const CpFactor **out);
// The autotuner's persistent cache (JSON lines, one {"key", "value"} per
// line; the last line for a key wins), also held in memory per process.
bool tune_cache_get(const std::string &key, std::string *value);
void tune_cache_put(const std::string &key, const std::string &value);
void ensure_device_facts(stencil_plan_s *p);
// Centred storage of a CUDA-core 2D/3D run (k_center.cu): the device FP64
// slot the input's sum goes to, 1 / points, and (sum c)^T, the factor of the
// mean over the run.
struct CentredRun {
    bool on;
    double *sum;
    double inv_n, factor;
};
CentredRun centred_run(stencil_plan_s *p, int64_t T);

// Runs enqueue(stream, &kernels) on stream s.  With graphs enabled and s not
// itself being captured, the work is captured once per key on a private
// stream into an executable graph, which is then replayed on s: a run of many
// short passes costs one graph launch on the host.
template <class F>
stencil_status_t run_maybe_graph(stencil_plan_s *p, const std::vector<int64_t> &key,
                                 cudaStream_t s, F enqueue)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;
    }
    if (!p->use_graph || cs != cudaStreamCaptureStatusNone) {
        int n = 0;
        stencil_status_t st = enqueue(s, &n);
        p->launches += n;
        return st;
    }
    auto it = p->graphs.find(key);
    if (it == p->graphs.end()) {
        cudaError_t e = cudaSuccess;
        if (!p->cap_stream) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "graph capture begin");
        int n = 0;
        stencil_status_t st = enqueue(p->cap_stream, &n);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(p->cap_stream, &g);
        if (st != STENCIL_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "graph capture end");
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
        it = p->graphs.emplace(key, stencil_plan_s::GraphEnt{ex, n}).first;
    }
    cudaError_t e = cudaGraphLaunch(it->second.exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    p->launches += it->second.launches;
    return STENCIL_OK;
}

}  // namespace sg
