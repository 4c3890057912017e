// 3D CUDA-core stencil sweeps (plain m = 1 and folded m > 1), streaming along z.
//
// A CTA owns a 64 x 16 (x, y) column of the grid and a chunk of z planes.
// Input planes arrive four at a time: one 3D TMA box (x-HX .. x+64+HX,
// y-R .. y+16+R, four planes) per stage of a three-stage ring, so the CTA
// synchronises once per four planes.  Each thread owns a 4-point strip of one row and keeps a
// register window of 2R+1 output planes: input plane z is read once from
// shared memory and added, with the weights of plane offset a, into the
// partial sums of output planes z - a (the counterparts of Section 3.3,
// taken along z: the paper handles a 3D grid as a stack of 2D slices);
// output plane z - R is then complete and stored.  The input plane's slot is
// free as soon as it has been read, so the ring needs only the prefetch depth.
#include "sweep3d_common.cuh"

namespace sg {
namespace {

using namespace sweep3d;

// 8 consumer warps (one 4-column strip of one row per thread) and one
// producer warp that keeps the ring full.
constexpr int NC3 = 256, NT3 = NC3 + 32;

template <int RB, int M, int PAT>
__global__ void __launch_bounds__(NT3)
    k_sweep3d(const __grid_constant__ CUtensorMap map, const __grid_constant__ Sweep3DArgs a)
{
    using TP = Taps3<RB, M, PAT>;
    constexpr int R = TP::R, W = TP::W, RP = TP::RP;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *stages = reinterpret_cast<float *>(smem + 1024);
    const int HX = a.halo_x;
    const int SP = TX3 + 2 * HX;   // shared row pitch
    const int ROWS = TY3 + 2 * R;
    const int plane = SP * ROWS;   // floats of one staged plane
    const uint32_t chunk_bytes = (uint32_t)(plane * ZC * 4);
    const int tid = threadIdx.x;

    const int tile = blockIdx.x;
    const int txy = tile % a.ntiles_xy, zc = tile / a.ntiles_xy;
    const int tx = txy % a.tiles_x, ty = txy / a.tiles_x;
    const int x0 = tx * TX3, y0 = ty * TY3;
    const int z0 = zc * a.zchunk, z1 = min(a.nz, z0 + a.zchunk);
    const int zin0 = z0 - R, nin = (z1 - z0) + 2 * R;  // input planes streamed
    const int nchunks = (nin + ZC - 1) / ZC;

    const int NST = a.nst;          // TMA stages (2 or 3)
    uint64_t *empty = bars + NST;  // released by the 8 consumer warps
    if (tid == 0) {
        prefetch_tensormap(&map);
        for (int s = 0; s < NST; ++s) {
            mbar_init(&bars[s], 1);
            mbar_init(&empty[s], NC3 / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (tid >= NC3) {
        // producer: chunk c (input planes 4c .. 4c+3 of this CTA) into stage
        // c % NST once the consumers released the chunk NST earlier
        if (tid != NC3) return;
        int c = 0;
        for (; c < nchunks; ++c) {
            const int s = c % NST;
            if (c >= NST && !mbar_wait_bounded(&empty[s], ((c / NST) - 1) & 1, a.wait_ns)) {
                record_status(a.status, DEV_TIMEOUT);
                break;
            }
            // (fault_withhold_copy is a test hook: the first chunk is never
            // requested, so the consumers' bounded waits and then this
            // warp's must run out and report a timeout)
            if (c == 0 && a.fault_withhold_copy) continue;
            mbar_arrive_expect_tx(&bars[s], chunk_bytes);
            tma_load_3d(stages + s * a.buf_floats, &map, &bars[s], a.map_x0 + x0 - HX,
                        a.map_y0 + y0 - R, a.map_z0 + zin0 + c * ZC);
        }
        // the copies still in flight land before the CTA may exit
        for (int q = max(0, c - NST); q < c; ++q)
            mbar_wait_bounded(&bars[q % NST], (q / NST) & 1, a.wait_ns);
        return;
    }

    // thread -> (4-column strip, row) of the tile
    const int strip = tid % (TX3 / 4), yr = tid / (TX3 / 4);
    const int X = x0 + 4 * strip, Y = y0 + yr;
    const bool live = (Y < a.ny) && (X < a.nx);
    const bool vec4 = a.dst_vec4 && X + 3 < a.nx;  // one 16-byte store per plane
    const Dst3 dst = dst_of(a);

    float acc[W][4];
#pragma unroll
    for (int i = 0; i < W; ++i)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[i][v] = 0.f;

    bool failed = false;
    for (int c = 0; c < nchunks; ++c) {
        const int s = c % NST;
        if (!mbar_wait_bounded(&bars[s], (c / NST) & 1, a.wait_ns)) {
            record_status(a.status, DEV_TIMEOUT);
            failed = true;
            break;
        }
        const float *chunk = stages + s * a.buf_floats + 4 * strip + HX - RP;
#pragma unroll 1
        for (int q = 0; q < ZC; ++q) {
            const int p = c * ZC + q;
            if (p >= nin) break;
            // this input plane feeds output plane z - R + i with plane offset R - i
            add_plane3<RB, M, PAT>(acc, chunk + q * plane, yr, SP, a);
            const int zo = zin0 + p - R;  // output plane completed by this input plane
            emit_plane3<W>(acc, dst, X, Y, zo, a.nx, zo >= z0 && live, vec4);
        }
        __syncwarp();  // this warp is done with stage s
        if ((tid & 31) == 0) mbar_arrive(&empty[s]);
    }
    // every consumer gets here (all waits are bounded); the ghost band is
    // refreshed once all of the CTA's outputs are stored
    if (consumers_any3<NC3>(failed) || a.dst_gw <= 0) return;
    refresh_ghosts3<NC3>(a, dst, x0, y0, z0, z1, tid);
}

template <int RB, int M, int PAT>
cudaError_t prepare3()
{
    return smem_optin((const void *)k_sweep3d<RB, M, PAT>);
}

template <int RB, int M, int PAT>
cudaError_t launch3(const CUtensorMap &map, const Sweep3DArgs &a, int grid, size_t smem,
                   cudaStream_t s)
{
    cudaError_t e = prepare3<RB, M, PAT>();
    if (e != cudaSuccess) return e;
    k_sweep3d<RB, M, PAT><<<grid, NT3, smem, s>>>(map, a);
    return cudaGetLastError();
}

template <int RB, int M, int PAT>
int occ3(size_t smem)
{
    if (prepare3<RB, M, PAT>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep3d<RB, M, PAT>, NT3, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

#define SG_SWEEP3D_LIST(X)                                                                 \
    X(1, 1, PAT_STAR) X(1, 2, PAT_STAR) X(1, 3, PAT_STAR) X(1, 4, PAT_STAR) X(2, 1, PAT_STAR) \
    X(2, 2, PAT_STAR) X(1, 1, PAT_BOX) X(1, 2, PAT_BOX) X(2, 1, PAT_BOX)

}  // namespace

bool sweep3d_supported(int rb, int m, int pattern)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_) return true;
    SG_SWEEP3D_LIST(SG_X)
#undef SG_X
    return false;
}

size_t sweep3d_smem_bytes(int tile_y, int R, int *buf_floats, int nst)
{
    (void)tile_y;
    const int HX = round_up(R, 4);
    const int bf = round_up((TX3 + 2 * HX) * (TY3 + 2 * R) * ZC, 32);
    if (buf_floats) *buf_floats = bf;
    return 1024 + (size_t)nst * bf * 4;
}

int sweep3d_ctas_per_sm(int rb, int m, int pattern, size_t smem)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_) return occ3<RB_, M_, P_>(smem);
    SG_SWEEP3D_LIST(SG_X)
#undef SG_X
    return 0;
}

cudaError_t launch_sweep3d(int rb, int m, int pattern, const CUtensorMap &map,
                           const Sweep3DArgs &a, int grid, size_t smem, cudaStream_t s)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_) return launch3<RB_, M_, P_>(map, a, grid, smem, s);
    SG_SWEEP3D_LIST(SG_X)
#undef SG_X
    return cudaErrorInvalidValue;
}

}  // namespace sg
