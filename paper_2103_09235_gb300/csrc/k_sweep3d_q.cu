// Multi-pass 3D CUDA-core sweep: ONE persistent launch runs npass single
// sweeps of one stencil (Section 1's time loop, ping-ponging between the
// plan's two padded grids, Section 3.3), with the z-streaming tile body of
// k_sweep3d.
//
// A pass is cut into pieces (a 64 x 16 column of the grid and a chunk of z
// planes).  Launched one pass per kernel, a small grid runs about two pieces
// per CTA per pass and the SMs idle through each pass's last wave.  Here the
// items (pass t, piece) form one list, handed to the resident CTAs round
// robin (CTA c takes items c, c + G, c + 2G, ...), and an item of pass t only
// waits until every piece whose cells it reads -- or whose cells of pass t-1
// it overwrites -- has finished pass t-1 (a per-piece counter of finished
// passes).  So the next pass's pieces fill the SMs while the last pieces of
// the current pass drain.  Pass t visits the z chunks starting at chunk t, so
// a piece's neighbours across the periodic z boundary finished early in the
// previous pass.
//
// Roles: 8 consumer warps run the tile body; the producer warp waits for an
// item's neighbours (one counter per lane, acquire loads) and requests its
// input planes four at a time (3D TMA boxes) into a ring that runs on across
// items.  After an item's outputs are stored and its ghost band refreshed,
// thread 0 publishes the item (release fence, atomic add on its counter).
//
// Items wait only for items earlier in the list, every CTA is resident and a
// CTA finishes its items in order, so the earliest unfinished item can always
// proceed.  Every wait is bounded; on expiry the CTA records a timeout, lets
// its requested copies land and exits.
#include "sweep3d_common.cuh"

namespace sg {
namespace {

using namespace sweep3d;

// 8 consumer warps and the producer warp.  Radius-1 instances are held to 72
// registers, three CTAs per SM: at four (56 registers) they spill and ran
// slower on GB300 (256^3 box 382 against 449 GS/s).
constexpr int NCQ = 256, NTQ = NCQ + 32;
constexpr int kMinBlocksQ1 = 3;

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_proxy_async_global3()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Item k of the list: pass t, position s within the pass; pass t visits the
// z chunks in the order t, t+1, ... (mod the chunk count), the xy tiles of a
// chunk in order.
struct QItem {
    int t, tx, ty, zc, piece;
};

__device__ __forceinline__ QItem decode_item(const Sweep3DArgs &a, int k)
{
    QItem it;
    it.t = k / a.ntiles;
    const int s = k - it.t * a.ntiles;
    const int sb = s / a.ntiles_xy, txy = s - sb * a.ntiles_xy;
    it.zc = (sb + it.t) % a.zchunks;
    it.tx = txy % a.tiles_x;
    it.ty = txy / a.tiles_x;
    it.piece = txy + it.zc * a.ntiles_xy;
    return it;
}

template <int RB, int M, int PAT>
__global__ void __launch_bounds__(NTQ, Taps3<RB, M, PAT>::R == 1 ? kMinBlocksQ1 : 2)
    k_sweep3d_q(const __grid_constant__ CUtensorMap map_e, const __grid_constant__ CUtensorMap map_o,
                const __grid_constant__ Sweep3DArgs a, const __grid_constant__ Sweep3DQueue q)
{
    using TP = Taps3<RB, M, PAT>;
    constexpr int R = TP::R, W = TP::W, RP = TP::RP;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    const int NST = a.nst;  // TMA stages (2 or 3)
    uint64_t *empty = full + NST;
    float *stages = reinterpret_cast<float *>(smem + 1024);
    const int HX = a.halo_x;
    const int SP = TX3 + 2 * HX;  // shared row pitch
    const int plane = SP * (TY3 + 2 * R);
    const uint32_t chunk_bytes = (uint32_t)(plane * ZC * 4);
    const int nitems = q.npass * a.ntiles;
    const int tid = threadIdx.x;
    if (tid == 0) {
        prefetch_tensormap(&map_e);
        prefetch_tensormap(&map_o);
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCQ / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (tid >= NCQ) {
        // ---- producer warp
        const int lane = tid - NCQ;
        int gc = 0;  // chunks requested so far (stage gc % NST)
        bool ok = true;
        for (int k = blockIdx.x; k < nitems && ok; k += gridDim.x) {
            const QItem it = decode_item(a, k);
            if (it.t > 0) {
                // every neighbour piece must have finished pass t - 1: lane l
                // watches the neighbours l, l + 32, ... of the per-axis lists
                const int *lx = q.dep + it.tx * kDep3;
                const int *ly = q.dep + q.dep_y + it.ty * kDep3;
                const int *lz = q.dep + q.dep_z + it.zc * kDep3;
                bool mine = true;
                const uint64_t t0 = globaltimer_ns();
                for (int l = lane; l < kDep3 * kDep3 * kDep3 && mine; l += 32) {
                    const int jx = lx[l % kDep3], jy = ly[(l / kDep3) % kDep3],
                              jz = lz[l / (kDep3 * kDep3)];
                    if (jx < 0 || jy < 0 || jz < 0) continue;
                    const int *cnt = q.done + jx + jy * a.tiles_x + jz * a.ntiles_xy;
                    // (the test hook treats every dependency as unmet, so this
                    // wait runs out, bounded, as a lost completion would)
                    while (q.fault_withhold_dep || ld_acquire_gpu(cnt) < it.t) {
                        if (globaltimer_ns() - t0 > a.wait_ns) {
                            mine = false;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                ok = __all_sync(0xffffffffu, mine);
                if (!ok) break;
            }
            if (lane == 0) {
                // other CTAs' stores, acquired above, before the copies read them
                fence_proxy_async_global3();
                const CUtensorMap *map = (it.t & 1) ? &map_o : &map_e;
                const int z0 = it.zc * a.zchunk, z1 = min(a.nz, z0 + a.zchunk);
                const int zin0 = z0 - R, nch = ((z1 - z0) + 2 * R + ZC - 1) / ZC;
                for (int c = 0; c < nch; ++c, ++gc) {
                    const int s = gc % NST;
                    if (gc >= NST && !mbar_wait_bounded(&empty[s], ((gc / NST) - 1) & 1, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    // (test hook: the CTA's first chunk is never requested)
                    if (gc == 0 && a.fault_withhold_copy) continue;
                    mbar_arrive_expect_tx(&full[s], chunk_bytes);
                    tma_load_3d(stages + s * a.buf_floats, map, &full[s], a.map_x0 + it.tx * TX3 - HX,
                                a.map_y0 + it.ty * TY3 - R, a.map_z0 + zin0 + c * ZC);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
        }
        if (lane == 0) {
            if (!ok) record_status(a.status, DEV_TIMEOUT);
            // the copies still in flight land before the CTA may exit
            for (int g = max(0, gc - NST); g < gc; ++g)
                mbar_wait_bounded(&full[g % NST], (g / NST) & 1, a.wait_ns);
        }
        return;
    }

    // ---- consumers: thread -> (4-column strip, row) of the piece
    const int strip = tid % (TX3 / 4), yr = tid / (TX3 / 4);
    int gc = 0;  // chunks consumed so far
    bool failed = false;
    for (int k = blockIdx.x; k < nitems; k += gridDim.x) {
        const QItem it = decode_item(a, k);
        // the last pass writes the launch's destination, the others the
        // padded grid the next pass reads
        const bool last = it.t == q.npass - 1;
        const Dst3 d = last ? dst_of(a) : Dst3{(it.t & 1) ? q.dst[1] : q.dst[0], q.py, q.pz, q.gw};
        const int z0 = it.zc * a.zchunk, nin = min(a.nz - z0, a.zchunk) + 2 * R;
        const int X = it.tx * TX3 + 4 * strip, Y = it.ty * TY3 + yr;
        const bool live = (Y < a.ny) && (X < a.nx);
        const bool vec4 = (!last || a.dst_vec4) && X + 3 < a.nx;
        float *const orow = d.p + (int64_t)Y * d.py + X;  // this thread's output row, plane 0
        float acc[W][4];
#pragma unroll
        for (int i = 0; i < W; ++i)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[i][v] = 0.f;
        // input plane p (from z0 - R) completes output plane z0 - 2R + p
        int zo = z0 - 2 * R;
        for (int p0 = 0; p0 < nin; p0 += ZC, ++gc) {
            const int s = gc % NST;
            // the warp decides together, so that it reaches __syncwarp whole
            const bool landed = __all_sync(0xffffffffu, mbar_wait_bounded(&full[s], (gc / NST) & 1, a.wait_ns));
            if (!landed) {
                record_status(a.status, DEV_TIMEOUT);
                failed = true;
                break;
            }
            const float *chunk = stages + s * a.buf_floats + 4 * strip + HX - RP;
            const int np = min(ZC, nin - p0);
#pragma unroll 1
            for (int qq = 0; qq < np; ++qq, ++zo) {
                add_plane3<RB, M, PAT>(acc, chunk + qq * plane, yr, SP, a);
                if (zo >= z0 && live) {
                    float *o = orow + (int64_t)zo * d.pz;
                    if (vec4) {
                        *reinterpret_cast<float4 *>(o) = make_float4(acc[0][0], acc[0][1], acc[0][2], acc[0][3]);
                    } else {
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            if (X + v < a.nx) o[v] = acc[0][v];
                    }
                }
#pragma unroll
                for (int i = 0; i < W - 1; ++i)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[i][v] = acc[i + 1][v];
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[W - 1][v] = 0.f;
            }
            __syncwarp();  // this warp is done with stage s
            if ((tid & 31) == 0) mbar_arrive(&empty[s]);
        }
        // barrier over the consumers: the item's outputs are stored
        if (consumers_any3<NCQ>(failed)) break;
        if (d.gw > 0) {
            refresh_ghosts3<NCQ>(a, d, it.tx * TX3, it.ty * TY3, z0, min(a.nz, z0 + a.zchunk), tid);
            NamedBarrier<NCQ>::sync();
        }
        if (tid == 0) {
            __threadfence();  // the consumers' stores, ordered by the barrier
            atomicAdd(q.done + it.piece, 1);
        }
    }
}

template <int RB, int M, int PAT>
cudaError_t prepare_q()
{
    return smem_optin((const void *)k_sweep3d_q<RB, M, PAT>);
}

template <int RB, int M, int PAT>
cudaError_t launch_q(const CUtensorMap &map_e, const CUtensorMap &map_o, const Sweep3DArgs &a,
                     const Sweep3DQueue &q, int grid, size_t smem, cudaStream_t s)
{
    cudaError_t e = prepare_q<RB, M, PAT>();
    if (e != cudaSuccess) return e;
    k_sweep3d_q<RB, M, PAT><<<grid, NTQ, smem, s>>>(map_e, map_o, a, q);
    return cudaGetLastError();
}

template <int RB, int M, int PAT>
int occ_q(size_t smem)
{
    if (prepare_q<RB, M, PAT>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep3d_q<RB, M, PAT>, NTQ, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

#define SG_SWEEP3DQ_LIST(X)                                                                \
    X(1, 1, PAT_STAR) X(1, 2, PAT_STAR) X(1, 3, PAT_STAR) X(1, 4, PAT_STAR) X(2, 1, PAT_STAR) \
    X(2, 2, PAT_STAR) X(1, 1, PAT_BOX) X(1, 2, PAT_BOX) X(2, 1, PAT_BOX)

}  // namespace

bool sweep3d_q_supported(int rb, int m, int pattern)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_) return true;
    SG_SWEEP3DQ_LIST(SG_X)
#undef SG_X
    return false;
}

int sweep3d_q_ctas_per_sm(int rb, int m, int pattern, size_t smem)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_) return occ_q<RB_, M_, P_>(smem);
    SG_SWEEP3DQ_LIST(SG_X)
#undef SG_X
    return 0;
}

cudaError_t launch_sweep3d_q(int rb, int m, int pattern, const CUtensorMap &map_e,
                             const CUtensorMap &map_o, const Sweep3DArgs &a,
                             const Sweep3DQueue &q, int grid, size_t smem, cudaStream_t s)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_) return launch_q<RB_, M_, P_>(map_e, map_o, a, q, grid, smem, s);
    SG_SWEEP3DQ_LIST(SG_X)
#undef SG_X
    return cudaErrorInvalidValue;
}

}  // namespace sg
