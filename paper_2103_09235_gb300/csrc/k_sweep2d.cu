// 2D CUDA-core stencil sweeps: plain (m = 1), folded (m > 1) and temporally
// blocked (b folded sweeps per HBM round trip).
//
// One persistent CTA walks its share of 128 x tile_y output tiles.  For every
// tile one TMA box brings the tile plus a halo of H = b*m*r cells (columns
// rounded up to 4) from the padded source grid into shared memory; a ring of
// 2-6 stages (one mbarrier each) keeps the next tiles' boxes in flight while
// this one is computed.  Sweeps 1..b-1 run shared memory to shared memory on a
// region that shrinks by R per sweep (overlapped tiles: the rim is computed
// redundantly, the GPU analogue of Section 3.4's time-loop fusion inside a
// tile); the last sweep writes the tile to global memory with 16-byte stores
// and refreshes the ghost band of the destination.
//
// Inside a sweep each thread owns a strip of 4 columns and walks down a run
// of rows with a register sliding window: input row j is read once (16-byte
// shared loads) and added, with the weights of row offset a, into the
// accumulators of output rows j - a.  These accumulators are the column
// partial sums the paper calls counterparts (Section 3.3, Eq. vfold); the
// shift of the window is the register form of its shifts reusing
// (Section 3.4).  Weights live in the kernel parameter block, so every
// multiply-add takes its weight from the constant bank.
#include "sweep2d_tile.cuh"

namespace sg {
namespace {

using namespace tile2d;

// Threads per CTA and resident CTAs per SM of each instance: plain radius-1
// sweeps are memory-bound and keep three 256-thread CTAs per SM; folded
// sweeps of at most 41 taps fit 512 threads (<= 128 registers each) in the
// one CTA per SM their shared memory allows, doubling the warps that hide
// FMA and shared-load latency; wider stencils keep 256 threads.
// Counterpart sweeps (two 1D folds per sweep) keep at most 2R+1 x 4
// accumulators and run 512 threads.
template <int RB, int M, int PAT>
constexpr int threads2d()
{
    if constexpr (PAT >= PAT_CP1) return 512;
    else return RB * M == 1 ? 256 : (Strip<RB, M, PAT>::NNZ <= 41 ? 512 : 256);
}
template <int RB, int M>
constexpr int min_blocks() { return RB * M == 1 ? 3 : 1; }

template <int RB, int M, int PAT>
__global__ void __launch_bounds__(threads2d<RB, M, PAT>(), min_blocks<RB, M>())
    k_sweep2d(const __grid_constant__ CUtensorMap map, const __grid_constant__ Sweep2DArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *base = reinterpret_cast<float *>(smem + 1024) + BUF_PAD;
    // buffers: NS TMA stages, then work 0 and work 1 (intermediate sweeps)
    const int NS = a.nstages;
    auto buf = [&](int k) { return base + k * a.buf_floats; };

    const int TY = a.tile_y, H = a.halo, HX = a.halo_x;
    const int SP = TX + 2 * HX, ROWS = TY + 2 * H;
    const uint32_t box_bytes = static_cast<uint32_t>(SP) * ROWS * 4u;
    const int tid = threadIdx.x;

    // the item split of each sweep of a full tile, worked out once per CTA
    // (bytes 512.. of the control block; the barriers use the first 48)
    SweepGeom *geom = reinterpret_cast<SweepGeom *>(smem + 512);
    if (tid < a.b) full_tile_geom<RB * M>(geom, tid, a.b, a.tile_y, a.halo, a.halo_x, blockDim.x);
    if (tid == 0) {
        prefetch_tensormap(&map);
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int tile, int s) {
        const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
        mbar_arrive_expect_tx(&bars[s], box_bytes);
        tma_load_2d(buf(s), &map, &bars[s], a.map_x0 + tx * TX - HX, a.map_y0 + ty * TY - H);
    };

    int tile = blockIdx.x;
    // b == 1: the only sweep reads the stage, so NS-1 tiles are in flight
    // while one is computed and a stage is refilled once its tile is done.
    // b >= 2: the stage is free after the tile's first sweep, so it is
    // refilled with the tile NS ahead right then (NS tiles in flight, and a
    // single stage already overlaps the copy with sweeps 2..b).  The
    // counterpart form frees it after its first vertical fold, for any b.
    const bool early = a.b >= 2 || PAT >= PAT_CP1;
    // (fault_withhold_copy is a test hook: the first copy is never issued, so
    // the bounded wait below must run out and report a timeout)
    if (tid == 0)
        for (int k = 0; k < (early ? NS : NS - 1); ++k) {
            const int t = tile + k * gridDim.x;
            if (t < a.ntiles && !(k == 0 && a.fault_withhold_copy)) issue(t, k);
        }

    for (int i = 0; tile < a.ntiles; ++i, tile += gridDim.x) {
        if (!early) {
            // request the tile NS-1 ahead into the stage the previous tile released
            const int ahead = tile + (NS - 1) * gridDim.x;
            if (tid == 0 && ahead < a.ntiles) issue(ahead, (i + NS - 1) % NS);
        }

        const bool ok = mbar_wait_bounded(&bars[i % NS], (i / NS) & 1, a.wait_ns);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                record_status(a.status, DEV_TIMEOUT);
                // let the copies already requested land before exiting: in
                // both modes those are the tiles i+1 .. i+NS-1 of this CTA
                for (int k = 1; k < NS; ++k) {
                    const int q = i + k;
                    if (tile + k * gridDim.x < a.ntiles)
                        mbar_wait_bounded(&bars[q % NS], (q / NS) & 1, a.wait_ns);
                }
            }
            return;
        }

        const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
        const TileOut o{a.dst, a.dst_py, a.nx, a.ny, a.dst_gw, a.dst_vec4};
        const int refill = tile + NS * gridDim.x;
        const int st = i % NS;
        auto stage_free = [&]() {
            if (tid == 0 && refill < a.ntiles) issue(refill, st);
        };
        // counterpart buffers (counterpart patterns only) follow the work buffers
        const int nwork = a.b >= 3 ? 2 : (a.b == 2 ? 1 : 0);
        process_tile<RB, M, PAT>(buf(st), buf(NS), buf(NS + 1), TY, H, HX, a.b, ParamCoef{a.c},
                                 o, tx * TX - HX, ty * TY - H, min(TX, a.nx - tx * TX),
                                 min(TY, a.ny - ty * TY), stage_free, buf(NS + nwork),
                                 a.buf_floats, geom);
        __syncthreads();
    }
}

// Opt every instantiation into the largest dynamic shared memory, once per
// device (the attribute is per device).
template <int RB, int M, int PAT>
cudaError_t prepare_t()
{
    return smem_optin((const void *)k_sweep2d<RB, M, PAT>);
}

// Threads per CTA of a launch: the instance's own count, or 256 when asked
// for and the instance runs 512 (the tile body adapts to its block size; two
// 256-thread CTAs per SM then keep their barriers independent).
template <int RB, int M, int PAT>
int threads_t(int want)
{
    constexpr int full = threads2d<RB, M, PAT>();
    return (want == 256 && full == 512) ? 256 : full;
}

template <int RB, int M, int PAT>
cudaError_t launch_t(const CUtensorMap &map, const Sweep2DArgs &a, int grid, size_t smem,
                     int threads, cudaStream_t s)
{
    cudaError_t e = prepare_t<RB, M, PAT>();
    if (e != cudaSuccess) return e;
    k_sweep2d<RB, M, PAT><<<grid, threads_t<RB, M, PAT>(threads), smem, s>>>(map, a);
    return cudaGetLastError();
}

template <int RB, int M, int PAT>
int occupancy_t(size_t smem, int threads)
{
    if (prepare_t<RB, M, PAT>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep2d<RB, M, PAT>,
                                                      threads_t<RB, M, PAT>(threads), smem) !=
        cudaSuccess)
        return 0;
    return n;
}

// The instantiated (rb, m, pattern) combinations.
// (counterpart instances are (1, R, PAT_CPk): folded radius R, k separable terms)
#define SG_SWEEP2D_LIST(X)                                                                     \
    X(1, 1, PAT_STAR) X(1, 2, PAT_STAR) X(1, 3, PAT_STAR) X(1, 4, PAT_STAR) X(2, 1, PAT_STAR) \
    X(2, 2, PAT_STAR) X(1, 1, PAT_BOX) X(1, 2, PAT_BOX) X(1, 3, PAT_BOX) X(1, 4, PAT_BOX)     \
    X(2, 1, PAT_BOX) X(2, 2, PAT_BOX) X(3, 1, PAT_BOX) X(4, 1, PAT_BOX)                       \
    X(1, 1, PAT_CP1) X(1, 2, PAT_CP1) X(1, 3, PAT_CP1) X(1, 4, PAT_CP1) X(1, 6, PAT_CP1)      \
    X(1, 8, PAT_CP1) X(1, 1, PAT_CP2) X(1, 2, PAT_CP2) X(1, 3, PAT_CP2) X(1, 4, PAT_CP2)      \
    X(1, 6, PAT_CP2) X(1, 8, PAT_CP2)

}  // namespace

bool sweep2d_supported(int rb, int m, int pattern)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_) return true;
    SG_SWEEP2D_LIST(SG_X)
#undef SG_X
    return false;
}

size_t sweep2d_smem_bytes(int tile_y, int b, int R, int *buf_floats, int nstages, int cp_bufs)
{
    const int H = b * R, HX = round_up(H, 4);
    const int SP = TX + 2 * HX, ROWS = tile_y + 2 * H;
    const int bf = round_up(SP * ROWS + 2 * BUF_PAD, 32);
    const int nbuf = nstages + (b >= 3 ? 2 : (b == 2 ? 1 : 0)) + cp_bufs;
    if (buf_floats) *buf_floats = bf;
    return 1024 + static_cast<size_t>(nbuf) * bf * 4;
}

int sweep2d_ctas_per_sm(int rb, int m, int pattern, size_t smem, int threads)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_) return occupancy_t<RB_, M_, P_>(smem, threads);
    SG_SWEEP2D_LIST(SG_X)
#undef SG_X
    return 0;
}

int sweep2d_block_threads(int rb, int m, int pattern, int threads)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_) return threads_t<RB_, M_, P_>(threads);
    SG_SWEEP2D_LIST(SG_X)
#undef SG_X
    return 0;
}

cudaError_t launch_sweep2d(int rb, int m, int pattern, const CUtensorMap &map,
                           const Sweep2DArgs &a, int grid, size_t smem, int threads,
                           cudaStream_t s)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_)  \
        return launch_t<RB_, M_, P_>(map, a, grid, smem, threads, s);
    SG_SWEEP2D_LIST(SG_X)
#undef SG_X
    return cudaErrorInvalidValue;
}

}  // namespace sg
