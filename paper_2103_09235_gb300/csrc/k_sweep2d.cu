// 2D CUDA-core stencil sweeps: plain (m = 1), folded (m > 1) and temporally
// blocked (b folded sweeps per HBM round trip).
//
// One persistent CTA walks its share of 128 x tile_y output tiles.  For every
// tile one TMA box brings the tile plus a halo of H = b*m*r cells (columns
// rounded up to 4) from the padded source grid into shared memory; the next
// tile's box is already in flight while this one is computed (two stages,
// one mbarrier each).  Sweeps 1..b-1 run shared memory to shared memory on a
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
#include "device_common.cuh"
#include "internal.h"

namespace sg {
namespace {

constexpr int TX = kTileX2D;
constexpr int NT = kThreads2D;
constexpr int BUF_PAD = 32;  // floats of slack before and after every buffer

__host__ __device__ constexpr int cabs_div(int v, int d) { return ((v < 0 ? -v : v) + d - 1) / d; }

template <int RB, int M, int PAT>
struct Taps {
    static constexpr int R = RB * M;
    static constexpr int W = 2 * R + 1;
    static constexpr int RP = (R + 3) / 4 * 4;  // halo columns loaded per side, 16-byte aligned
    __host__ __device__ static constexpr bool nz(int a, int b)
    {
        return PAT == PAT_BOX ? true : (cabs_div(a, RB) + cabs_div(b, RB) <= M);
    }
};

__device__ __forceinline__ void store_point(float *dst, int64_t py, int nx, int ny, int gw, int X,
                                            int Y, float v)
{
    dst[Y * py + X] = v;
    if (gw > 0) {
        const bool xl = X < gw, xh = X >= nx - gw, yl = Y < gw, yh = Y >= ny - gw;
        if (xl) dst[Y * py + X + nx] = v;
        if (xh) dst[Y * py + X - nx] = v;
        if (yl) {
            dst[(Y + ny) * py + X] = v;
            if (xl) dst[(Y + ny) * py + X + nx] = v;
            if (xh) dst[(Y + ny) * py + X - nx] = v;
        }
        if (yh) {
            dst[(Y - ny) * py + X] = v;
            if (xl) dst[(Y - ny) * py + X + nx] = v;
            if (xh) dst[(Y - ny) * py + X - nx] = v;
        }
    }
}

template <int RB, int M, int PAT>
struct Strip {
    using TP = Taps<RB, M, PAT>;
    static constexpr int R = TP::R, W = TP::W, RP = TP::RP;
    static constexpr int NSEG = 4 + 2 * RP;
    static constexpr int NNZ = [] {
        int n = 0;
        for (int a = -R; a <= R; ++a)
            for (int b = -R; b <= R; ++b) n += TP::nz(a, b) ? 1 : 0;
        return n;
    }();
    // rows of the steady loop unrolled together: a full turn of the window
    // when the row's multiply-adds are few, so the window shift is renamed away
    static constexpr int UNR = NNZ * 4 <= 200 ? W : 1;

    __device__ __forceinline__ static void load(const float *rowp, float (&seg)[NSEG])
    {
        const float4 *rp = reinterpret_cast<const float4 *>(rowp);
#pragma unroll
        for (int q = 0; q < NSEG / 4; ++q) {
            const float4 t = rp[q];
            seg[4 * q + 0] = t.x;
            seg[4 * q + 1] = t.y;
            seg[4 * q + 2] = t.z;
            seg[4 * q + 3] = t.w;
        }
    }

    // input row into window slot i (output row j - R + i, row offset a = R - i)
    __device__ __forceinline__ static void slot(float (&acc)[W][4], const float (&seg)[NSEG],
                                                const Sweep2DArgs &a, int i)
    {
        const int aa = R - i;
#pragma unroll
        for (int bb = -R; bb <= R; ++bb) {
            if (TP::nz(aa, bb)) {
                const float w = a.c[(aa + R) * W + (bb + R)];
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[i][v] = fmaf(w, seg[v + bb + RP], acc[i][v]);
            }
        }
    }

    __device__ __forceinline__ static void shift(float (&acc)[W][4])
    {
#pragma unroll
        for (int i = 0; i < W - 1; ++i)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[i][v] = acc[i + 1][v];
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[W - 1][v] = 0.f;
    }
};

__device__ __noinline__ void store_ghosts4(const Sweep2DArgs &a, int X, int Y, float v0, float v1,
                                           float v2, float v3)
{
    const float v[4] = {v0, v1, v2, v3};
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (X + k < a.nx) store_point(a.dst, a.dst_py, a.nx, a.ny, a.dst_gw, X + k, Y, v[k]);
}

// One sweep over output rows [r0, r1) and 4-column strips [k0, k1) of a
// shared-memory buffer S (row pitch SP).  FINAL writes to global memory;
// otherwise the outputs go to the same coordinates of buffer D.
//
// A strip of rows [ya, yb) reads input rows ya-R .. yb+R-1.  The first 2R
// rows only feed window slots whose output row is >= ya and the last 2R only
// slots whose output row is < yb, so every output gets exactly its taps.
template <int RB, int M, int PAT, bool FINAL>
__device__ __forceinline__ void sweep_region(const float *__restrict__ S, float *__restrict__ D,
                                             int SP, int r0, int r1, int k0, int k1,
                                             const Sweep2DArgs &a, int gx0, int gy0)
{
    using ST = Strip<RB, M, PAT>;
    constexpr int R = ST::R, W = ST::W, RP = ST::RP, NSEG = ST::NSEG;
    const int nsx = k1 - k0;
    const int nr = r1 - r0;
    if (nsx <= 0 || nr <= 0) return;
    // row groups: as many as the threads allow, each at least 2R rows tall
    int G = NT / nsx;
    G = max(1, min(G, nr / (2 * R)));
    const int items = nsx * G;

    for (int it = threadIdx.x; it < items; it += NT) {
        const int k = k0 + it % nsx;
        const int g = it / nsx;
        const int ya = r0 + (g * nr) / G;
        const int yb = r0 + ((g + 1) * nr) / G;
        const int cx = 4 * k;
        const float *col = S + cx - RP;

        float acc[W][4];
#pragma unroll
        for (int i = 0; i < W; ++i)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[i][v] = 0.f;

        auto emit = [&](int y) {
            if constexpr (FINAL) {
                const int X = gx0 + cx, Y = gy0 + y;
                if (Y < a.ny && X < a.nx) {
                    float *row = a.dst + Y * a.dst_py;
                    if (a.dst_vec4 && X + 3 < a.nx) {
                        *reinterpret_cast<float4 *>(row + X) =
                            make_float4(acc[0][0], acc[0][1], acc[0][2], acc[0][3]);
                    } else {
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            if (X + v < a.nx) row[X + v] = acc[0][v];
                    }
                    if (a.dst_gw > 0 && (X < a.dst_gw || X + 3 >= a.nx - a.dst_gw ||
                                         Y < a.dst_gw || Y >= a.ny - a.dst_gw))
                        store_ghosts4(a, X, Y, acc[0][0], acc[0][1], acc[0][2], acc[0][3]);
                }
            } else {
                *reinterpret_cast<float4 *>(D + y * SP + cx) =
                    make_float4(acc[0][0], acc[0][1], acc[0][2], acc[0][3]);
            }
        };

        int j = ya - R;
        if (yb - ya >= 2 * R) {
            // ramp-up: rows ya-R .. ya+R-1 feed only slots i >= 2R - u
#pragma unroll
            for (int u = 0; u < 2 * R; ++u, ++j) {
                float seg[NSEG];
                ST::load(col + j * SP, seg);
#pragma unroll
                for (int i = 0; i < W; ++i)
                    if (i >= 2 * R - u) ST::slot(acc, seg, a, i);
                ST::shift(acc);
            }
            // steady rows: every slot, one finished output row each
            const int jm = yb - R;
#pragma unroll ST::UNR
            for (; j < jm; ++j) {
                float seg[NSEG];
                ST::load(col + j * SP, seg);
#pragma unroll
                for (int i = 0; i < W; ++i) ST::slot(acc, seg, a, i);
                emit(j - R);
                ST::shift(acc);
            }
            // ramp-down: the last 2R rows feed only slots i <= v
#pragma unroll
            for (int v = 2 * R - 1; v >= 0; --v, ++j) {
                float seg[NSEG];
                ST::load(col + j * SP, seg);
#pragma unroll
                for (int i = 0; i < W; ++i)
                    if (i <= v) ST::slot(acc, seg, a, i);
                emit(j - R);
                ST::shift(acc);
            }
        } else {
            // short strip: plain window over all rows
#pragma unroll 1
            for (; j < yb + R; ++j) {
                float seg[NSEG];
                ST::load(col + j * SP, seg);
#pragma unroll
                for (int i = 0; i < W; ++i) ST::slot(acc, seg, a, i);
                if (j - R >= ya) emit(j - R);
                ST::shift(acc);
            }
        }
    }
}

// Plain radius-1 sweeps are memory-bound: keep three CTAs per SM resident.
template <int RB, int M>
constexpr int min_blocks() { return RB * M == 1 ? 3 : 1; }

template <int RB, int M, int PAT>
__global__ void __launch_bounds__(NT, min_blocks<RB, M>())
    k_sweep2d(const __grid_constant__ CUtensorMap map, const __grid_constant__ Sweep2DArgs a)
{
    constexpr int R = RB * M;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *base = reinterpret_cast<float *>(smem + 1024) + BUF_PAD;
    // buffers: stage 0, stage 1 (TMA targets), work 0, work 1 (intermediate sweeps)
    auto buf = [&](int k) { return base + k * a.buf_floats; };

    const int TY = a.tile_y, H = a.halo, HX = a.halo_x;
    const int SP = TX + 2 * HX, ROWS = TY + 2 * H;
    const uint32_t box_bytes = static_cast<uint32_t>(SP) * ROWS * 4u;
    const int tid = threadIdx.x;

    if (tid == 0) {
        prefetch_tensormap(&map);
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int tile, int s) {
        const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
        mbar_arrive_expect_tx(&bars[s], box_bytes);
        tma_load_2d(buf(s), &map, &bars[s], a.map_x0 + tx * TX - HX, a.map_y0 + ty * TY - H);
    };

    int tile = blockIdx.x;
    // (fault_withhold_copy is a test hook: the first copy is never issued, so
    // the bounded wait below must run out and report a timeout)
    if (tid == 0 && tile < a.ntiles && !a.fault_withhold_copy) issue(tile, 0);

    for (int i = 0; tile < a.ntiles; ++i, tile += gridDim.x) {
        const int nxt = tile + gridDim.x;
        if (tid == 0 && nxt < a.ntiles) issue(nxt, (i + 1) & 1);

        const bool ok = mbar_wait_bounded(&bars[i & 1], (i >> 1) & 1, a.wait_ns);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                record_status(a.status, DEV_TIMEOUT);
                // let the copy already issued for the next tile land before exiting
                if (nxt < a.ntiles) mbar_wait_bounded(&bars[(i + 1) & 1], ((i + 1) >> 1) & 1, a.wait_ns);
            }
            return;
        }

        const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
        const int gx0 = tx * TX - HX;  // interior x of shared column 0
        const int gy0 = ty * TY - H;   // interior y of shared row 0
        const float *src = buf(i & 1);
        for (int s = 0; s < a.b - 1; ++s) {
            const int sh = (s + 1) * R;
            const int c0 = HX - H + sh, c1 = SP - (HX - H) - sh;
            float *dst = buf(2 + (s & 1));
            sweep_region<RB, M, PAT, false>(src, dst, SP, sh, ROWS - sh, c0 / 4, (c1 + 3) / 4, a,
                                            gx0, gy0);
            __syncthreads();
            src = dst;
        }
        sweep_region<RB, M, PAT, true>(src, nullptr, SP, H, H + TY, HX / 4, (HX + TX) / 4, a, gx0,
                                       gy0);
        __syncthreads();
    }
}

// Opt every instantiation into the largest dynamic shared memory once, so
// launches need no attribute call.
template <int RB, int M, int PAT>
cudaError_t prepare_t()
{
    static cudaError_t once = [] {
        int dev = 0, maxs = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&maxs, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        return cudaFuncSetAttribute(k_sweep2d<RB, M, PAT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
    }();
    return once;
}

template <int RB, int M, int PAT>
cudaError_t launch_t(const CUtensorMap &map, const Sweep2DArgs &a, int grid, size_t smem,
                     cudaStream_t s)
{
    cudaError_t e = prepare_t<RB, M, PAT>();
    if (e != cudaSuccess) return e;
    k_sweep2d<RB, M, PAT><<<grid, NT, smem, s>>>(map, a);
    return cudaGetLastError();
}

template <int RB, int M, int PAT>
int occupancy_t(size_t smem)
{
    if (prepare_t<RB, M, PAT>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep2d<RB, M, PAT>, NT, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

// The instantiated (rb, m, pattern) combinations.
#define SG_SWEEP2D_LIST(X)                                                                     \
    X(1, 1, PAT_STAR) X(1, 2, PAT_STAR) X(1, 3, PAT_STAR) X(1, 4, PAT_STAR) X(2, 1, PAT_STAR) \
    X(2, 2, PAT_STAR) X(1, 1, PAT_BOX) X(1, 2, PAT_BOX) X(1, 3, PAT_BOX) X(1, 4, PAT_BOX)     \
    X(2, 1, PAT_BOX) X(2, 2, PAT_BOX) X(3, 1, PAT_BOX) X(4, 1, PAT_BOX)

}  // namespace

bool sweep2d_supported(int rb, int m, int pattern)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_) return true;
    SG_SWEEP2D_LIST(SG_X)
#undef SG_X
    return false;
}

size_t sweep2d_smem_bytes(int tile_y, int b, int R, int *buf_floats)
{
    const int H = b * R, HX = round_up(H, 4);
    const int SP = TX + 2 * HX, ROWS = tile_y + 2 * H;
    const int bf = round_up(SP * ROWS + 2 * BUF_PAD, 32);
    const int nbuf = 2 + (b >= 3 ? 2 : (b == 2 ? 1 : 0));
    if (buf_floats) *buf_floats = bf;
    return 1024 + static_cast<size_t>(nbuf) * bf * 4;
}

int sweep2d_ctas_per_sm(int rb, int m, int pattern, size_t smem)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_) return occupancy_t<RB_, M_, P_>(smem);
    SG_SWEEP2D_LIST(SG_X)
#undef SG_X
    return 0;
}

cudaError_t launch_sweep2d(int rb, int m, int pattern, const CUtensorMap &map,
                           const Sweep2DArgs &a, int grid, size_t smem, cudaStream_t s)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_) return launch_t<RB_, M_, P_>(map, a, grid, smem, s);
    SG_SWEEP2D_LIST(SG_X)
#undef SG_X
    return cudaErrorInvalidValue;
}

}  // namespace sg
