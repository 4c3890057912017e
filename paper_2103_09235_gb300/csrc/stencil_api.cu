// C-ABI entry points: plan life cycle, options, folded weights, error
// reduction, the host-only profitability counts, and the dispatch of
// stencil_run to the per-dimension drivers.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "plan.h"

namespace sg {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

stencil_status_t cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? STENCIL_ERR_OOM : STENCIL_ERR_CUDA;
}

void round_f32_mass(const double *c, size_t n, size_t centre, float *out)
{
    double want = 0.0, got = 0.0;
    for (size_t i = 0; i < n; ++i) {
        out[i] = (float)c[i];
        want += c[i];
        got += (double)out[i];
    }
    if (n > 0) out[centre] = (float)((double)out[centre] + (want - got));
}

cudaError_t smem_optin(const void *kernel)
{
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({kernel, dev})) return cudaSuccess;
    int maxs = 0;
    e = cudaDeviceGetAttribute(&maxs, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
    if (e == cudaSuccess) done.insert({kernel, dev});
    return e;
}

static int taps_count(int ndim, int r)
{
    int n = 1;
    for (int d = 0; d < ndim; ++d) n *= 2 * r + 1;
    return n;
}

stencil_status_t plan_folded(stencil_plan_s *p, int m, const std::vector<double> **out)
{
    auto it = p->folded.find(m);
    if (it != p->folded.end()) {
        *out = &it->second;
        return STENCIL_OK;
    }
    if (m == 1) {
        p->folded[1] = p->coeffs;
        *out = &p->folded[1];
        return STENCIL_OK;
    }
    const int nin = taps_count(p->ndim, p->r);
    const int nout = taps_count(p->ndim, m * p->r);
    double *d_c = nullptr, *d_out = nullptr, *d_work = nullptr;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&d_c, sizeof(double) * nin);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(double) * nout);
    if (e == cudaSuccess) e = cudaMalloc(&d_work, sizeof(double) * 2 * nout);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_c, p->coeffs.data(), sizeof(double) * nin, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_fold_power(p->ndim, p->r, m, d_c, d_out, d_work, s);
    std::vector<double> host(nout);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host.data(), d_out, sizeof(double) * nout, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (d_c) cudaFree(d_c);
    if (d_out) cudaFree(d_out);
    if (d_work) cudaFree(d_work);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) return cuda_fail(e, "folded weights");
    p->launches += 1;
    p->folded[m] = std::move(host);
    *out = &p->folded[m];
    return STENCIL_OK;
}

static stencil_status_t alloc_padded(stencil_plan_s *p, Padded &P)
{
    P.ndim = p->ndim;
    P.nx = p->nx;
    P.ny = p->ny;
    P.nz = p->nz;
    P.gx = kGhost;
    P.gy = p->ndim >= 2 ? kGhost : 0;
    P.gz = p->ndim >= 3 ? kGhost : 0;
    P.py = round_up(p->nx + 2 * kGhost, 32);
    P.pz = P.py * (p->ny + 2 * P.gy);
    P.elems = (size_t)P.pz * (p->nz + 2 * P.gz);
    cudaError_t e = cudaMalloc(&P.alloc, P.elems * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, "allocating a padded grid");
    e = cudaMemset(P.alloc, 0, P.elems * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, "clearing a padded grid");
    P.origin = P.alloc + (size_t)P.gz * P.pz + (size_t)P.gy * P.py + P.gx;
    p->scratch_bytes += P.elems * sizeof(float);
    return STENCIL_OK;
}

stencil_status_t ensure_padded(stencil_plan_s *p)
{
    if (p->A.alloc) return STENCIL_OK;
    stencil_status_t st = alloc_padded(p, p->A);
    if (st == STENCIL_OK) st = alloc_padded(p, p->B);
    return st;
}

const CUtensorMap *plan_map(stencil_plan_s *p, const Padded &P, const int *box)
{
    auto key = std::make_tuple((const void *)P.alloc, box[0], P.ndim >= 2 ? box[1] : 0,
                               P.ndim >= 3 ? box[2] : 0);
    auto it = p->maps.find(key);
    if (it != p->maps.end()) return &it->second;
    CUtensorMap m;
    if (!encode_padded_map(&m, P, box)) {
        set_error("cuTensorMapEncodeTiled refused box %d x %d", box[0], P.ndim >= 2 ? box[1] : 0);
        return nullptr;
    }
    return &(p->maps[key] = m);
}

cudaError_t copy_grid(const stencil_plan_s *p, void *dst, const void *src, cudaMemcpyKind kind,
                      cudaStream_t s)
{
    const size_t esz = p->dtype == STENCIL_F64 ? 8 : 4;
    if (grid_dense(p)) return cudaMemcpyAsync(dst, src, esz * grid_extent(p), kind, s);
    // rows of nx points, pitch_y apart; planes pitch_z apart
    if (p->ndim < 3 || p->pitch_z == p->pitch_y * p->ny)
        return cudaMemcpy2DAsync(dst, esz * p->pitch_y, src, esz * p->pitch_y, esz * p->nx,
                                 (size_t)p->ny * p->nz, kind, s);
    for (int z = 0; z < p->nz; ++z) {
        const size_t off = esz * (size_t)z * p->pitch_z;
        cudaError_t e = cudaMemcpy2DAsync((char *)dst + off, esz * p->pitch_y,
                                          (const char *)src + off, esz * p->pitch_y, esz * p->nx,
                                          (size_t)p->ny, kind, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sg

using namespace sg;

extern "C" {

const char *stencil_status_string(stencil_status_t s)
{
    switch (s) {
    case STENCIL_OK: return "STENCIL_OK";
    case STENCIL_ERR_INVALID_ARG: return "STENCIL_ERR_INVALID_ARG";
    case STENCIL_ERR_UNSUPPORTED: return "STENCIL_ERR_UNSUPPORTED";
    case STENCIL_ERR_OOM: return "STENCIL_ERR_OOM";
    case STENCIL_ERR_CUDA: return "STENCIL_ERR_CUDA";
    case STENCIL_ERR_TIMEOUT: return "STENCIL_ERR_TIMEOUT";
    case STENCIL_ERR_DEVICE_CHECK: return "STENCIL_ERR_DEVICE_CHECK";
    }
    return "STENCIL_ERR_UNKNOWN";
}

const char *stencil_last_error(void) { return g_err; }

stencil_status_t stencil_fold_cost(int ndim, int radius, const double *coeffs, int m,
                                   int64_t *out)
{
    if (ndim < 1 || ndim > 3 || radius < 1 || radius > 8 || !coeffs || m < 1 || m > 16 || !out) {
        set_error("stencil_fold_cost: bad argument");
        return STENCIL_ERR_INVALID_ARG;
    }
    // Support of c^(s) as a set of offsets, built by Minkowski sums of the
    // base support (exact, no floating point).
    typedef std::vector<int> Off;
    std::set<Off> base;
    const int w = 2 * radius + 1;
    const int n = taps_count(ndim, radius);
    for (int i = 0; i < n; ++i) {
        if (coeffs[i] == 0.0) continue;
        Off o(ndim);
        int t = i;
        for (int d = ndim - 1; d >= 0; --d) {
            o[d] = t % w - radius;
            t /= w;
        }
        base.insert(o);
    }
    std::set<Off> cur;
    cur.insert(Off(ndim, 0));
    int64_t naive = 0;
    for (int s = 0; s < m; ++s) {
        naive += (int64_t)cur.size();
        std::set<Off> nxt;
        for (const Off &a : cur)
            for (const Off &b : base) {
                Off c(ndim);
                for (int d = 0; d < ndim; ++d) c[d] = a[d] + b[d];
                nxt.insert(c);
            }
        cur.swap(nxt);
    }
    out[0] = naive * (int64_t)base.size();
    out[1] = (int64_t)cur.size();
    return STENCIL_OK;
}

stencil_status_t stencil_plan(stencil_plan_t *out_plan, int ndim, const int64_t *shape,
                              int radius, const double *coeffs, stencil_dtype_t dtype)
{
    if (!out_plan || !shape || !coeffs || ndim < 1 || ndim > 3 || radius < 1 || radius > 4) {
        set_error("stencil_plan: bad ndim/radius/pointer");
        return STENCIL_ERR_INVALID_ARG;
    }
    *out_plan = nullptr;
    if (dtype != STENCIL_F32 && dtype != STENCIL_F64) {
        set_error("stencil_plan: unknown dtype");
        return STENCIL_ERR_INVALID_ARG;
    }
    for (int d = 0; d < ndim; ++d) {
        if (shape[d] < 2 * radius + 1 || shape[d] > (int64_t)1 << 30) {
            set_error("stencil_plan: extent %lld outside [2r+1, 2^30]", (long long)shape[d]);
            return STENCIL_ERR_INVALID_ARG;
        }
    }
    int64_t total = 1;
    for (int d = 0; d < ndim; ++d) total *= shape[d];
    if (total > ((int64_t)1 << 34)) {
        set_error("stencil_plan: grid too large");
        return STENCIL_ERR_INVALID_ARG;
    }
    stencil_plan_s *p = new stencil_plan_s();
    cudaGetDevice(&p->device);
    p->ndim = ndim;
    for (int d = 0; d < ndim; ++d) p->shape[d] = shape[d];
    p->nx = (int)shape[ndim - 1];
    p->ny = ndim >= 2 ? (int)shape[ndim - 2] : 1;
    p->nz = ndim >= 3 ? (int)shape[0] : 1;
    p->pitch_y = p->nx;
    p->pitch_z = (int64_t)p->nx * p->ny;
    p->r = radius;
    p->dtype = dtype;
    const int n = taps_count(ndim, radius);
    p->coeffs.assign(coeffs, coeffs + n);
    // star if every tap off the axes is zero
    bool star = ndim >= 2;
    const int w = 2 * radius + 1;
    for (int i = 0; i < n && star; ++i) {
        int t = i, nzax = 0;
        for (int d = 0; d < ndim; ++d) {
            if (t % w != radius) ++nzax;
            t /= w;
        }
        if (nzax > 1 && coeffs[i] != 0.0) star = false;
    }
    p->pattern = star ? PAT_STAR : PAT_BOX;
    cudaError_t e = cudaMalloc(&p->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_acc, 8 * sizeof(double));
    if (e != cudaSuccess) {
        stencil_status_t st = cuda_fail(e, "stencil_plan");
        if (p->d_status) cudaFree(p->d_status);
        delete p;
        return st;
    }
    *out_plan = p;
    return STENCIL_OK;
}

stencil_status_t stencil_plan_ex(stencil_plan_t *out_plan, int ndim, const int64_t *shape,
                                 int radius, const double *coeffs, stencil_dtype_t dtype,
                                 const int64_t *pitch_elems, unsigned flags)
{
    if (!out_plan) {
        set_error("stencil_plan_ex: null out_plan");
        return STENCIL_ERR_INVALID_ARG;
    }
    *out_plan = nullptr;
    if (flags & ~(unsigned)STENCIL_FLAG_NONPERIODIC) {
        set_error("stencil_plan_ex: unknown flag bits 0x%x", flags);
        return STENCIL_ERR_INVALID_ARG;
    }
    if (flags & STENCIL_FLAG_NONPERIODIC) {
        set_error("stencil_plan_ex: only periodic boundaries are supported (folding is exact "
                  "only on periodic grids)");
        return STENCIL_ERR_UNSUPPORTED;
    }
    // pitch_elems[d] is the stride of axis d (C order), d = 0 .. ndim-2;
    // checked before any device work
    int64_t py = 0, pz = 0;
    if (pitch_elems && shape && ndim >= 2 && ndim <= 3) {
        const int64_t nx = shape[ndim - 1], ny = shape[ndim - 2];
        py = pitch_elems[ndim - 2];
        pz = ndim == 3 ? pitch_elems[0] : py * ny;
        if (py < nx || (ndim == 3 && pz < py * ny) || py > ((int64_t)1 << 31) ||
            pz > ((int64_t)1 << 40)) {
            set_error("stencil_plan_ex: pitches must satisfy row >= nx and plane >= row * ny");
            return STENCIL_ERR_INVALID_ARG;
        }
    }
    stencil_plan_t p = nullptr;
    stencil_status_t st = stencil_plan(&p, ndim, shape, radius, coeffs, dtype);
    if (st != STENCIL_OK) return st;
    if (py > 0) {
        p->pitch_y = py;
        p->pitch_z = pz;
    }
    *out_plan = p;
    return STENCIL_OK;
}

stencil_status_t stencil_plan_set_option(stencil_plan_t p, const char *key, int64_t v)
{
    if (!p || !key) {
        set_error("stencil_plan_set_option: null argument");
        return STENCIL_ERR_INVALID_ARG;
    }
    if (!strcmp(key, "precision")) {
        if (v < 0 || v > 3) goto bad;
        p->precision = (int)v;
    } else if (!strcmp(key, "block_b")) {
        if (v < 0 || v > 64) goto bad;
        p->block_b = (int)v;
    } else if (!strcmp(key, "tile_y")) {
        if (v != 0 && (v < 8 || v > 192)) goto bad;
        p->tile_y = (int)v;
    } else if (!strcmp(key, "cta_threads")) {
        if (v != 0 && v != 256) goto bad;
        p->cta_threads = (int)v;
    } else if (!strcmp(key, "tile_1d")) {
        if (v != 0 && (v < 256 || v > 16384 || v % 256)) goto bad;
        p->tile_1d = (int)v;
    } else if (!strcmp(key, "persistent")) {
        if (v < -1 || v > 1) goto bad;
        p->persistent = (int)v;
    } else if (!strcmp(key, "z_chunk")) {
        if (v != 0 && (v < 2 || v > 1024)) goto bad;
        p->z_chunk = (int)v;
    } else if (!strcmp(key, "stages")) {
        if (v < 0 || v > 6) goto bad;
        p->stages = (int)v;
    } else if (!strcmp(key, "tc_center")) {
        if (v != 0 && v != 1) goto bad;
        p->tc_center = (int)v;
    } else if (!strcmp(key, "wait_limit_ms")) {
        if (v < 1 || v > 600000) goto bad;
        p->wait_ms = v;
    } else if (!strcmp(key, "fault_withhold_copy")) {
        if (v != 0 && v != 1) goto bad;
        p->fault_withhold_copy = (int)v;
    } else if (!strcmp(key, "fault_withhold_dep")) {
        if (v != 0 && v != 1) goto bad;
        p->fault_withhold_dep = (int)v;
    } else if (!strcmp(key, "fault_withhold_mma")) {
        if (v != 0 && v != 1) goto bad;
        p->fault_withhold_mma = (int)v;
    } else if (!strcmp(key, "counterparts")) {
        if (v < 0 || v > 2) goto bad;
        p->counterparts = (int)v;
        p->cp.clear();  // the choice per m follows the option
        p->tuned_m = 0;
    } else if (!strcmp(key, "tc_form")) {
        if (v < 0 || v > 2) goto bad;
        p->tc_form = (int)v;
    } else if (!strcmp(key, "tc_tma_store")) {
        if (v != 0 && v != 1) goto bad;
        p->tc_tma_store = (int)v;
    } else if (!strcmp(key, "center")) {
        if (v != 0 && v != 1) goto bad;
        p->center = (int)v;
    } else if (!strcmp(key, "tessellate")) {
        if (v != 0 && v != 1) goto bad;
        p->tessellate = (int)v;
    } else if (!strcmp(key, "graph")) {
        if (v != 0 && v != 1) goto bad;
        p->use_graph = (int)v;
    } else if (!strcmp(key, "autotune")) {
        if (v != 0 && v != 1) goto bad;
        p->autotune = (int)v;
    } else {
        set_error("stencil_plan_set_option: unknown key '%s'", key);
        return STENCIL_ERR_INVALID_ARG;
    }
    clear_graphs(p);  // captured runs bake the options in
    return STENCIL_OK;
bad:
    set_error("stencil_plan_set_option: value %lld out of range for '%s'", (long long)v, key);
    return STENCIL_ERR_INVALID_ARG;
}

stencil_status_t stencil_plan_get(stencil_plan_t p, const char *key, int64_t *value)
{
    if (!p || !key || !value) {
        set_error("stencil_plan_get: null argument");
        return STENCIL_ERR_INVALID_ARG;
    }
    if (!strcmp(key, "last_m")) *value = p->last_m;
    else if (!strcmp(key, "last_b")) *value = p->last_b;
    else if (!strcmp(key, "last_tile_y")) *value = p->last_ty;
    else if (!strcmp(key, "last_engine")) *value = p->last_engine;
    else if (!strcmp(key, "last_threads")) *value = p->last_threads;
    else if (!strcmp(key, "last_stages")) *value = p->last_stages;
    else if (!strcmp(key, "last_persistent")) *value = p->last_persist;
    else if (!strcmp(key, "last_tc_form")) *value = p->last_tc_form;
    else if (!strcmp(key, "last_cp")) *value = p->last_cp;
    else if (!strcmp(key, "last_tess")) *value = p->last_tess;
    else if (!strcmp(key, "launches")) *value = p->launches;
    else if (!strcmp(key, "scratch_bytes")) *value = (int64_t)p->scratch_bytes;
    else {
        set_error("stencil_plan_get: unknown key '%s'", key);
        return STENCIL_ERR_INVALID_ARG;
    }
    return STENCIL_OK;
}

stencil_status_t stencil_folded_coeffs(stencil_plan_t p, int m, double *host_out, size_t n)
{
    if (!p || !host_out || m < 1 || m * p->r > 16) {
        set_error("stencil_folded_coeffs: bad argument");
        return STENCIL_ERR_INVALID_ARG;
    }
    const size_t need = (size_t)taps_count(p->ndim, m * p->r);
    if (n < need) {
        set_error("stencil_folded_coeffs: need %zu doubles", need);
        return STENCIL_ERR_INVALID_ARG;
    }
    const std::vector<double> *f = nullptr;
    stencil_status_t st = plan_folded(p, m, &f);
    if (st != STENCIL_OK) return st;
    memcpy(host_out, f->data(), need * sizeof(double));
    return STENCIL_OK;
}

stencil_status_t stencil_rel_l2(const void *y, stencil_dtype_t ydtype, const double *ref,
                                int64_t n, double *host_out, stencil_stream_t stream)
{
    if (!y || !ref || !host_out || n < 1 || (ydtype != STENCIL_F32 && ydtype != STENCIL_F64)) {
        set_error("stencil_rel_l2: bad argument");
        return STENCIL_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *acc = nullptr;
    cudaError_t e = cudaMallocAsync(&acc, 4 * sizeof(double), s);
    if (e != cudaSuccess) return cuda_fail(e, "stencil_rel_l2 scratch");
    double h[4] = {0, 0, 0, 0};
    e = cudaMemsetAsync(acc, 0, 4 * sizeof(double), s);
    if (e == cudaSuccess) e = launch_rel_l2(y, ydtype == STENCIL_F64, ref, n, acc, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(acc, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "stencil_rel_l2");
    // h = {sum (y-r)^2, sum r^2, sum y, sum r}
    const double dn = (double)n;
    host_out[0] = h[1] > 0 ? sqrt(h[0] / h[1]) : (h[0] > 0 ? INFINITY : 0.0);
    const double dm = (h[2] - h[3]) / dn;
    const double e0 = h[0] - dn * dm * dm;
    const double r0 = h[1] - h[3] * h[3] / dn;
    host_out[1] = r0 > 0 ? sqrt(fmax(e0, 0.0) / r0) : 0.0;
    return STENCIL_OK;
}

stencil_status_t stencil_sync(stencil_plan_t p, stencil_stream_t stream)
{
    if (!p) {
        set_error("stencil_sync: null plan");
        return STENCIL_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "stencil_sync");
    int h = 0;
    e = cudaMemcpy(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "stencil_sync status read");
    if (h != 0) {
        cudaMemset(p->d_status, 0, sizeof(int));
        set_error("device status %d recorded by a kernel", h);
        return (stencil_status_t)h;
    }
    return STENCIL_OK;
}

static bool is_device_ptr(const void *ptr)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

stencil_status_t stencil_run(stencil_plan_t p, const void *in, void *out, int64_t T, int fold_m,
                             stencil_stream_t stream)
{
    if (!p || !in || !out || T < 0 || fold_m < 0 || fold_m > 16) {
        set_error("stencil_run: bad argument");
        return STENCIL_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool din = is_device_ptr(in), dout = is_device_ptr(out);
    if (din != dout) {
        set_error("stencil_run: in and out must both be device or both be host pointers");
        return STENCIL_ERR_INVALID_ARG;
    }
    const size_t esz = p->dtype == STENCIL_F64 ? 8 : 4;
    // the span of the caller's layout: with pitches, gaps between rows and
    // planes are inside it but never read or written
    const size_t bytes = esz * grid_extent(p);
    const void *din_p = in;
    void *dout_p = out;
    cudaError_t e;
    if (!din) {
        if (!p->stage_in) {
            e = cudaMalloc(&p->stage_in, bytes);
            if (e == cudaSuccess) e = cudaMalloc(&p->stage_out, bytes);
            if (e != cudaSuccess) return cuda_fail(e, "host staging buffers");
            p->scratch_bytes += 2 * bytes;
        }
        e = copy_grid(p, p->stage_in, in, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
        din_p = p->stage_in;
        dout_p = p->stage_out;
    }
    stencil_status_t st;
    if (T == 0) {
        e = copy_grid(p, dout_p, din_p, cudaMemcpyDeviceToDevice, s);
        st = e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "copy for T = 0");
    } else if (p->ndim == 1) {
        st = run1d(p, din_p, dout_p, T, fold_m, s);
    } else if (p->dtype == STENCIL_F64) {
        st = run_f64nd(p, (const double *)din_p, (double *)dout_p, T, fold_m, s);
    } else if (p->ndim == 2) {
        st = run2d(p, (const float *)din_p, (float *)dout_p, T, fold_m, s);
    } else {
        st = run3d(p, (const float *)din_p, (float *)dout_p, T, fold_m, s);
    }
    if (st != STENCIL_OK) return st;
    if (!din) {
        e = copy_grid(p, out, dout_p, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    }
    return STENCIL_OK;
}

void stencil_plan_destroy(stencil_plan_t p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    clear_graphs(p);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->d_status) cudaFree(p->d_status);
    if (p->d_acc) cudaFree(p->d_acc);
    if (p->A.alloc) cudaFree(p->A.alloc);
    if (p->B.alloc) cudaFree(p->B.alloc);
    if (p->d1a) cudaFree(p->d1a);
    if (p->d1b) cudaFree(p->d1b);
    if (p->d1p0) cudaFree(p->d1p0);
    if (p->d1p1) cudaFree(p->d1p1);
    if (p->stage_in) cudaFree(p->stage_in);
    if (p->stage_out) cudaFree(p->stage_out);
    for (auto &kv : p->panels) cudaFree(kv.second);
    for (auto &kv : p->batch_mem) cudaFree(kv.second);
    for (auto &kv : p->q3_mem) cudaFree(kv.second);
    delete p;
}

}  // extern "C"
