// Batched persistent sweep: many independent 2D grids of uneven size,
// stencil (star / box) and step count advance in ONE launch.
//
// The host flattens every grid's time loop (its folded passes of b fused
// sweeps, then its plain remainder passes, Section 3.4) into passes, and the
// passes into a work list of (pass, tile) items ordered round by round: all
// grids' first passes, then all grids' second passes, and so on.  Persistent
// CTAs pop items from a device queue (one atomic counter).  Before loading
// its tile a CTA waits, with a bounded spin, until every tile of the grid's
// previous pass has been counted done; items only ever wait for items earlier
// in the list, and every CTA is resident, so the queue cannot deadlock.  A
// tile is the same TMA-staged, register-window, temporally blocked body as the
// single-grid 2D sweep, with the grid's folded weights read from shared
// memory.  Completion is published with a release fence and an atomic add;
// the waiter acquires it and issues a proxy fence before its TMA load, so the
// copy engine sees the other CTAs' stores.
#include "sweep2d_tile.cuh"

namespace sg {
namespace {

using namespace tile2d;

constexpr int kThreadsBatched = 512;

struct SmemCoef {
    const float *c;
    __device__ __forceinline__ float operator()(int k) const { return c[k]; }
};

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Runs the tile body of the variant (pattern, m); radius-1 base stencils.
__device__ __forceinline__ void run_variant(int variant, const float *stage, float *w0, float *w1,
                                            int TY, int H, int HX, int b, const SmemCoef &cf,
                                            const TileOut &o, int gx0, int gy0)
{
    switch (variant) {
    case PAT_STAR * 8 + 1: process_tile<1, 1, PAT_STAR>(stage, w0, w1, TY, H, HX, b, cf, o, gx0, gy0); break;
    case PAT_STAR * 8 + 2: process_tile<1, 2, PAT_STAR>(stage, w0, w1, TY, H, HX, b, cf, o, gx0, gy0); break;
    case PAT_STAR * 8 + 3: process_tile<1, 3, PAT_STAR>(stage, w0, w1, TY, H, HX, b, cf, o, gx0, gy0); break;
    case PAT_STAR * 8 + 4: process_tile<1, 4, PAT_STAR>(stage, w0, w1, TY, H, HX, b, cf, o, gx0, gy0); break;
    case PAT_BOX * 8 + 1: process_tile<1, 1, PAT_BOX>(stage, w0, w1, TY, H, HX, b, cf, o, gx0, gy0); break;
    case PAT_BOX * 8 + 2: process_tile<1, 2, PAT_BOX>(stage, w0, w1, TY, H, HX, b, cf, o, gx0, gy0); break;
    default: break;
    }
}

__device__ __forceinline__ bool dep_met(const BatchArgs &a, const BatchPass &ps)
{
    return ps.dep < 0 || ld_acquire(&a.done[ps.dep]) >= a.passes[ps.dep].ntiles;
}

// Bounded wait for an item's dependency; false when the limit ran out.
__device__ __forceinline__ bool dep_wait(const BatchArgs &a, const BatchPass &ps)
{
    if (dep_met(a, ps)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!dep_met(a, ps))
        if (globaltimer_ns() - t0 > a.wait_ns) return false;
    return true;
}

__device__ __forceinline__ void issue_item(const BatchArgs &a, int idx, float *stage,
                                           uint64_t *bar)
{
    const BatchItem item = a.items[idx];
    const BatchPass &ps = a.passes[item.pass];
    const int tx = item.tile % ps.tiles_x, ty = item.tile / ps.tiles_x;
    fence_proxy_async_global();  // other CTAs' stores, acquired above, before the copy reads them
    const uint32_t bytes = (uint32_t)((kTileX2D + 2 * ps.HX) * (a.tile_y + 2 * ps.H) * 4);
    mbar_arrive_expect_tx(bar, bytes);
    tma_load_2d(stage, &a.maps[ps.map], bar, ps.map_x0 + tx * kTileX2D - ps.HX,
                ps.map_y0 + ty * a.tile_y - ps.H);
}

// Each CTA keeps two items in flight: while it computes the current one, the
// next item's tile is already being copied into the other stage if that
// item's dependency is met; otherwise it is requested once the current item
// is done (the current item may be one of its dependencies).
__global__ void __launch_bounds__(kThreadsBatched, 1) k_batched(const __grid_constant__ BatchArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);  // bar[0], bar[1]: one per stage
    int *ctl = reinterpret_cast<int *>(smem + 64);       // cur, next, issued, ok
    float *cs = reinterpret_cast<float *>(smem + 128);   // up to kMaxTaps2D weights
    float *base = reinterpret_cast<float *>(smem + 128 + round_up(kMaxTaps2D * 4, 128)) + BUF_PAD;
    auto stage = [&](int i) { return base + i * a.buf_floats; };  // two TMA stages
    float *w0 = base + 2 * a.buf_floats, *w1 = base + 3 * a.buf_floats;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        int ok = 1;
        const int cur = atomicAdd(a.next, 1);
        if (cur < a.nitems) {
            ok = dep_wait(a, a.passes[a.items[cur].pass]) ? 1 : 0;
            if (ok) issue_item(a, cur, stage(0), &bar[0]);
        }
        ctl[0] = cur;
        ctl[3] = ok;
    }
    __syncthreads();

    for (uint32_t k = 0;; ++k) {
        const int cur = ctl[0];
        if (cur >= a.nitems) break;
        if (!ctl[3]) {
            if (tid == 0) record_status(a.status, DEV_TIMEOUT);
            break;
        }
        const int st = k & 1;
        if (tid == 0) {
            const int nxt = atomicAdd(a.next, 1);
            int issued = 0;
            if (nxt < a.nitems && dep_met(a, a.passes[a.items[nxt].pass])) {
                issue_item(a, nxt, stage(st ^ 1), &bar[st ^ 1]);
                issued = 1;
            }
            ctl[1] = nxt;
            ctl[2] = issued;
        }
        const BatchItem item = a.items[cur];
        const BatchPass &ps = a.passes[item.pass];
        for (int i = tid; i < ps.ncoef; i += kThreadsBatched) cs[i] = a.coefs[ps.coef + i];
        const bool landed = mbar_wait_bounded(&bar[st], (k >> 1) & 1, a.wait_ns);
        if (__syncthreads_or(!landed)) {
            if (tid == 0) {
                record_status(a.status, DEV_TIMEOUT);
                if (ctl[2]) mbar_wait_bounded(&bar[st ^ 1], ((k + 1) >> 1) & 1, a.wait_ns);
            }
            break;
        }
        const int tx = item.tile % ps.tiles_x, ty = item.tile / ps.tiles_x;
        const TileOut o{ps.dst, ps.dst_py, ps.nx, ps.ny, ps.dst_gw, ps.dst_vec4};
        run_variant(ps.variant, stage(st), w0, w1, a.tile_y, ps.H, ps.HX, ps.b, SmemCoef{cs}, o,
                    tx * kTileX2D - ps.HX, ty * a.tile_y - ps.H);
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(&a.done[item.pass], 1);  // publish this tile
            const int nxt = ctl[1];
            int ok = 1;
            if (nxt < a.nitems && !ctl[2]) {
                ok = dep_wait(a, a.passes[a.items[nxt].pass]) ? 1 : 0;
                if (ok) issue_item(a, nxt, stage(st ^ 1), &bar[st ^ 1]);
            }
            ctl[0] = nxt;
            ctl[3] = ok;
        }
        __syncthreads();
    }
}

}  // namespace

bool batched_variant_supported(int rb, int m, int pattern)
{
    // folded stencils of at most 41 taps: the kernel runs 512 threads per CTA
    return rb == 1 && m >= 1 && ((pattern == PAT_STAR && m <= 4) || (pattern == PAT_BOX && m <= 2));
}

size_t batched_smem_bytes(int buf_floats)
{
    // two stages and two work buffers
    return 128 + round_up(kMaxTaps2D * 4, 128) + (size_t)4 * buf_floats * 4 + 2 * BUF_PAD * 4;
}

cudaError_t launch_batched(const BatchArgs &a, int grid, size_t smem, cudaStream_t s)
{
    static cudaError_t once = [] {
        int dev = 0, maxs = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&maxs, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        return cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
    }();
    if (once != cudaSuccess) return once;
    k_batched<<<grid, kThreadsBatched, smem, s>>>(a);
    return cudaGetLastError();
}

int batched_ctas_per_sm(size_t smem)
{
    int n = 0;
    cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batched, kThreadsBatched, smem) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace sg
