// Batched persistent sweep: many independent 2D grids of uneven size,
// stencil (star / box) and step count advance in ONE launch.
//
// The host flattens every grid's time loop (its folded passes of b fused
// sweeps, then its plain remainder passes, Section 3.4) into passes, and the
// passes into a work list of (pass, tile) items ordered round by round: all
// grids' first passes, then all grids' second passes, and so on.
//
// A CTA is 15 consumer warps (or 7, two CTAs per SM) that run the tile body
// and one producer warp (one active lane) that feeds them:
//   producer: pop an item from the device queue (one atomic counter), wait
//             (bounded) until every tile of the grid's previous pass is
//             counted done, write the item's description into one of two
//             slots and request the grid's folded weights (bulk copy) and,
//             once the TMA stage is free, the tile (2D TMA box), all on the
//             slot's "full" mbarrier;
//   consumers: wait on "full", run the TMA-staged, register-window,
//             temporally blocked tile body (the same one as the single-grid
//             sweep, weights from shared memory), release the stage after the
//             tile's first sweep (the later ones read only work buffers) and
//             the slot when the tile is done;
//   producer: once a slot is released, publish its item (release fence and
//             an atomic add on the pass's done counter).
// With one stage refilled after the first sweep, the next tile's copy overlaps
// the current tile's later sweeps, and the buffers left over allow tiles of up
// to 128 rows.  Batches of single sweeps keep two stages instead.
// Scheduling therefore never stalls the consumers.  Items only wait for items
// earlier in the list, every CTA is resident, and a producer that waits on a
// dependency keeps publishing the item its consumers are finishing, so the
// queue cannot deadlock.  Every wait is bounded; on expiry the CTA records a
// timeout, lets its requested copies land and exits.
#include "sweep2d_tile.cuh"

namespace sg {
namespace {

using namespace tile2d;

// Two CTA shapes, both at 128 registers a thread: 15 consumer warps and the
// producer (512 threads, one CTA per SM), or 7 consumer warps and the producer
// (256 threads, two CTAs per SM, each with half the shared memory).
constexpr int kConsumersWide = 480;  // threads that run the tile body
constexpr int kConsumersHalf = 224;
constexpr int kCoefSlot = 96;  // floats of weights per stage (>= 81)

// One stage's work description, written by the producer before its arrive on
// the stage's full barrier.
struct StageMeta {
    float *dst;
    long long dst_py;
    int nx, ny, dst_gw, dst_vec4;
    int variant, b, H, HX;
    int gx0, gy0, vx, vy;
    int stop;  // 0: an item; 1: the queue is empty; 2: a dependency wait ran out
};
static_assert(64 + 2 * sizeof(StageMeta) <= 256, "stage slots overlap the weights");

struct SmemCoef {
    const float *c;
    __device__ __forceinline__ float operator()(int k) const { return c[k]; }
};

// A tile's weights copied from its slot into registers once: read through the
// slot pointer, every tap of every row would be a shared-memory load (the
// compiler cannot prove the slot apart from the work buffers the sweep
// stores to).  Only the taps the pattern uses are ever read, so the copies of
// the others are dropped.  Patterns of up to 25 taps take this form; the
// 41-tap star (m = 4) keeps its weights in shared memory, where its registers
// would otherwise spill.
template <int N>
struct RegCoef {
    float w[N];
    __device__ __forceinline__ explicit RegCoef(const float *c)
    {
#pragma unroll
        for (int k = 0; k < N; ++k) w[k] = c[k];
    }
    __device__ __forceinline__ float operator()(int k) const { return w[k]; }
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

// OR of a predicate over the NC consumer threads (named barrier 1).
template <int NC>
__device__ __forceinline__ bool consumers_any(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(NC)
        : "memory");
    return r != 0;
}

__host__ __device__ constexpr int variant_code(int rb, int m, int pattern)
{
    return (rb - 1) * 16 + pattern * 8 + m;
}

// Runs the tile body of the variant (base radius, pattern, m) on the consumer
// threads that Sync names.
template <class Sync, class Hook>
__device__ __forceinline__ void run_variant(const StageMeta &md, const float *stage, float *w0,
                                            float *w1, int TY, const SmemCoef &cf,
                                            const Hook &stage_free)
{
    const TileOut o{md.dst, md.dst_py, md.nx, md.ny, md.dst_gw, md.dst_vec4};
#define SG_BATCHED_CASE(RB_, P_, M_)                                                            \
    case variant_code(RB_, M_, P_): {                                                           \
        if constexpr (Strip<RB_, M_, P_>::NNZ <= 25) {                                          \
            const RegCoef<(2 * M_ * RB_ + 1) * (2 * M_ * RB_ + 1)> rc(cf.c);                    \
            process_tile<RB_, M_, P_, Sync>(stage, w0, w1, TY, md.H, md.HX, md.b, rc,   \
                                                    o, md.gx0, md.gy0, md.vx, md.vy,            \
                                                    stage_free);                                \
        } else {                                                                                \
            process_tile<RB_, M_, P_, Sync>(stage, w0, w1, TY, md.H, md.HX, md.b, cf,   \
                                                    o, md.gx0, md.gy0, md.vx, md.vy,            \
                                                    stage_free);                                \
        }                                                                                       \
        break;                                                                                  \
    }
    switch (md.variant) {
        SG_BATCHED_CASE(1, PAT_STAR, 1)
        SG_BATCHED_CASE(1, PAT_STAR, 2)
        SG_BATCHED_CASE(1, PAT_STAR, 3)
        SG_BATCHED_CASE(1, PAT_STAR, 4)
        SG_BATCHED_CASE(1, PAT_BOX, 1)
        SG_BATCHED_CASE(1, PAT_BOX, 2)
        SG_BATCHED_CASE(2, PAT_STAR, 1)
        SG_BATCHED_CASE(2, PAT_STAR, 2)
        SG_BATCHED_CASE(2, PAT_BOX, 1)
    default: break;
    }
#undef SG_BATCHED_CASE
}

// The producer: one thread.  The CTA's k-th item uses description/weight slot
// p = k & 1 (barriers full[p], done[p]) and TMA stage k % S (barrier
// sfree[k % S]).  A stage is released after the item's first sweep when the
// item fuses two or more (the later sweeps read only work buffers), else when
// the item ends; a slot is released when the item ends.
__device__ __forceinline__ void produce(const BatchArgs &a, uint64_t *full, uint64_t *done_bar,
                                        uint64_t *sfree, StageMeta *meta, float *cslot,
                                        float *stage0)
{
    const int S = a.nstage;
    // per slot: the pass of the item it holds, not yet published (-1: none),
    // and that item's number k (registers, selected by slot)
    int pp0 = -1, pp1 = -1, pk0 = 0, pk1 = 0;
    auto pend_pass = [&](int p) { return p ? pp1 : pp0; };
    auto pend_k = [&](int p) { return p ? pk1 : pk0; };
    auto hold = [&](int p, int pass, int k) {
        if (p) {
            pp1 = pass;
            pk1 = k;
        } else {
            pp0 = pass;
            pk0 = k;
        }
    };
    auto publish = [&](int p) {
        __threadfence();  // the consumers' stores, acquired through the done barrier
        atomicAdd(&a.done[pend_pass(p)], 1);
        hold(p, -1, pend_k(p));
    };
    bool ok = true;
    for (int k = 0;; ++k) {
        const int p = k & 1;
        if (k >= 2) {
            // reuse slot p only after the consumers finished item k - 2
            if (!mbar_wait_bounded(&done_bar[p], ((k - 2) >> 1) & 1, a.wait_ns)) {
                ok = false;
                break;
            }
            if (pend_pass(p) >= 0) publish(p);
        }
        StageMeta &md = meta[p];
        const int idx = atomicAdd(a.next, 1);
        if (idx >= a.nitems) {
            md.stop = 1;
            mbar_arrive(&full[p]);
            break;
        }
        const BatchItem item = a.items[idx];
        const BatchPass &ps = a.passes[item.pass];
        if (ps.dep >= 0) {
            const int need = a.passes[ps.dep].ntiles;
            const int *cnt = &a.done[ps.dep];
            const uint64_t t0 = globaltimer_ns();
            // the test hook treats every dependency as unmet, so this wait
            // runs out (bounded) exactly as a lost completion would
            while (a.fault_withhold_dep || ld_acquire(cnt) < need) {
                // the item the consumers are finishing may be one this item waits for
                const int o = p ^ 1;
                if (pend_pass(o) >= 0 && mbar_test_wait(&done_bar[o], (pend_k(o) >> 1) & 1)) publish(o);
                if (globaltimer_ns() - t0 > a.wait_ns) {
                    ok = false;
                    break;
                }
            }
            if (!ok) {
                md.stop = 2;
                mbar_arrive(&full[p]);
                break;
            }
        }
        const int tx = item.tile % ps.tiles_x, ty = item.tile / ps.tiles_x;
        md.dst = ps.dst;
        md.dst_py = ps.dst_py;
        md.nx = ps.nx;
        md.ny = ps.ny;
        md.dst_gw = ps.dst_gw;
        md.dst_vec4 = ps.dst_vec4;
        md.variant = ps.variant;
        md.b = ps.b;
        md.H = ps.H;
        md.HX = ps.HX;
        md.gx0 = tx * kTileX2D - ps.HX;
        md.gy0 = ty * a.tile_y - ps.H;
        md.vx = min(kTileX2D, ps.nx - tx * kTileX2D);
        md.vy = min(a.tile_y, ps.ny - ty * a.tile_y);
        md.stop = 0;
        const uint32_t tile_bytes =
            (uint32_t)((kTileX2D + 2 * ps.HX) * (a.tile_y + 2 * ps.H) * 4);
        const uint32_t coef_bytes = (uint32_t)(((ps.ncoef + 3) & ~3) * 4);
        mbar_arrive_expect_tx(&full[p], tile_bytes + coef_bytes);
        bulk_load(cslot + p * kCoefSlot, a.coefs + ps.coef, coef_bytes, &full[p]);
        // the stage must have been released by item k - S.  After a timeout
        // the copy is still requested (the results are void by then): the
        // slot's barrier then completes, and the drain below lets every
        // requested copy land before the CTA exits
        const int st = k % S;
        const bool stage_ok =
            k < S || mbar_wait_bounded(&sfree[st], ((k - S) / S) & 1, a.wait_ns);
        fence_proxy_async_global();  // other CTAs' stores, acquired above, before the copy reads them
        tma_load_2d(stage0 + st * a.buf_floats, &a.maps[ps.map], &full[p],
                    ps.map_x0 + tx * kTileX2D - ps.HX, ps.map_y0 + ty * a.tile_y - ps.H);
        hold(p, item.pass, k);
        if (!stage_ok) {
            ok = false;
            break;
        }
    }
    if (!ok) record_status(a.status, DEV_TIMEOUT);
    // publish what the consumers still finish; if they stopped, let the
    // requested copies land before the CTA exits
    for (int p = 0; p < 2; ++p) {
        if (pend_pass(p) < 0) continue;
        const uint32_t par = (pend_k(p) >> 1) & 1;
        if (mbar_wait_bounded(&done_bar[p], par, a.wait_ns))
            publish(p);
        else
            mbar_wait_bounded(&full[p], par, a.wait_ns);
    }
}

template <int NC>
__global__ void __launch_bounds__(NC + 32, NC + 32 <= 256 ? 2 : 1)
    k_batched(const __grid_constant__ BatchArgs a)
{
    using ConsumerSync = NamedSync<NC>;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);  // full[2], done[2], sfree[2]
    uint64_t *done_bar = full + 2;
    uint64_t *sfree = full + 4;
    StageMeta *meta = reinterpret_cast<StageMeta *>(smem + 64);  // one per slot
    float *cslot = reinterpret_cast<float *>(smem + 256);      // kCoefSlot weights per slot
    float *base = reinterpret_cast<float *>(smem + 1024) + BUF_PAD;
    const int S = a.nstage;  // TMA stages at base, base + buf_floats
    // work buffers after the stages (a pass of b fused sweeps touches b - 1 of them)
    float *w0 = base + S * a.buf_floats;
    float *w1 = a.nwork >= 2 ? base + (S + 1) * a.buf_floats : w0;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&done_bar[i], 1);
            mbar_init(&sfree[i], 1);
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (tid >= NC) {
        if (tid == NC) produce(a, full, done_bar, sfree, meta, cslot, base);
        return;
    }
    for (int k = 0;; ++k) {
        const int p = k & 1;
        const bool landed = mbar_wait_bounded(&full[p], (k >> 1) & 1, a.wait_ns);
        if (consumers_any<NC>(!landed)) {
            if (tid == 0) record_status(a.status, DEV_TIMEOUT);
            break;
        }
        const StageMeta md = meta[p];
        if (md.stop) break;
        uint64_t *free_bar = &sfree[k % S];
        // b >= 2: the stage is free once the first sweep is done
        auto stage_free = [&]() {
            if (tid == 0) mbar_arrive(free_bar);
        };
        run_variant<ConsumerSync>(md, base + (k % S) * a.buf_floats, w0, w1, a.tile_y,
                    SmemCoef{cslot + p * kCoefSlot}, stage_free);
        ConsumerSync::sync();  // the item's buffers and slot are free again
        if (tid == 0) {
            if (md.b < 2) mbar_arrive(free_bar);
            mbar_arrive(&done_bar[p]);
        }
    }
}

}  // namespace

bool batched_variant_supported(int rb, int m, int pattern)
{
    // folded stencils of at most 41 taps (81 stored weights) within 128 registers
    if (m < 1) return false;
    if (rb == 1) return (pattern == PAT_STAR && m <= 4) || (pattern == PAT_BOX && m <= 2);
    if (rb == 2) return (pattern == PAT_STAR && m <= 2) || (pattern == PAT_BOX && m == 1);
    return false;
}

int batched_variant_id(int rb, int m, int pattern) { return variant_code(rb, m, pattern); }

size_t batched_smem_bytes(int buf_floats, int nwork, int nstage)
{
    // barriers, item slots and weights in the first KB; the stages and the
    // work buffers after it
    return 1024 + (size_t)(nstage + nwork) * buf_floats * 4 + 2 * BUF_PAD * 4;
}

cudaError_t launch_batched(const BatchArgs &a, int grid, size_t smem, int threads, cudaStream_t s)
{
    const bool half = threads == kConsumersHalf + 32;
    const void *fn = half ? (const void *)k_batched<kConsumersHalf> : (const void *)k_batched<kConsumersWide>;
    const cudaError_t e = smem_optin(fn);
    if (e != cudaSuccess) return e;
    if (half)
        k_batched<kConsumersHalf><<<grid, threads, smem, s>>>(a);
    else
        k_batched<kConsumersWide><<<grid, kConsumersWide + 32, smem, s>>>(a);
    return cudaGetLastError();
}

int batched_threads(int cta_threads) { return cta_threads == 256 ? kConsumersHalf + 32 : kConsumersWide + 32; }

int batched_ctas_per_sm(size_t smem, int threads)
{
    const bool half = threads == kConsumersHalf + 32;
    const void *fn = half ? (const void *)k_batched<kConsumersHalf> : (const void *)k_batched<kConsumersWide>;
    int n = 0;
    if (smem_optin(fn) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, half ? threads : kConsumersWide + 32, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

}  // namespace sg
