// 3D CUDA-core sweeps with temporal blocking: two fused sweeps of the
// (folded) stencil per HBM round trip, the time-loop fusion of Section 3.4
// taken along the streaming axis.
//
// A CTA owns a 64 x 16 (x, y) output column and a chunk of z planes, as in
// the single-sweep kernel, and input planes arrive through the same
// ring of 4-plane TMA boxes fed by a producer warp (two stages here).  The
// boxes carry 2R rows and 8 columns of halo per side.  For every chunk of four
// input planes:
//   1. the first sweep, over the tile plus a rim of R cells (18 strips of 4
//      columns by 16+2R rows, one per consumer thread), adds each plane into
//      a register window along z; every intermediate plane the window
//      completes goes to a ring of eight shared-memory plane buffers;
//   2. after one barrier over the consumer warps, the second sweep (16 x 16
//      strips) reads those intermediate planes' neighbours from the ring into
//      its own window along z and stores every output plane it completes.
// One barrier per four planes: the ring holds two chunks, so the next chunk's
// first sweep writes only slots the second sweep finished before the barrier.
// The rim's intermediate values come from the ghost-padded input (the band is
// 2R wide), so they are the periodic values; only the tile is stored, and the
// CTA then refreshes the ghost band of its output block as the single-sweep
// kernel does.
#include "sweep3d_common.cuh"

namespace sg {
namespace {

using namespace sweep3d;

constexpr int NCT = 384, NTT = NCT + 32;  // 12 consumer warps and the producer warp
constexpr int HXT = 8;                     // input halo columns per side (>= 2R, 16-byte aligned)
constexpr int S1X = TX3 / 4 + 2;           // first-sweep strips: the tile plus 4 columns per side
constexpr int SPT = TX3 + 2 * HXT;         // staged row pitch (floats)
constexpr int SPP = TX3 + 8;               // intermediate-plane row pitch: x0-4 .. x0+68
constexpr int NSTT = 2;                    // TMA stages (4 planes each)
constexpr int NPS = 2 * ZC;                // intermediate-plane ring: two chunks' worth

template <int RB, int M, int PAT>
__global__ void __launch_bounds__(NTT)
    k_sweep3d_tb(const __grid_constant__ CUtensorMap map, const __grid_constant__ Sweep3DArgs a)
{
    using TP = Taps3<RB, M, PAT>;
    constexpr int R = TP::R, W = TP::W, RP = TP::RP;
    constexpr int NSEG = 4 + 2 * RP;
    static_assert(RP <= 4 && S1X * (TY3 + 2 * R) <= NCT, "first sweep needs one thread per strip");
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);  // full[NSTT], then empty[NSTT]
    uint64_t *empty = bars + NSTT;
    float *stages = reinterpret_cast<float *>(smem + 1024);
    constexpr int ROWS_IN = TY3 + 4 * R, ROWS_P = TY3 + 2 * R;
    constexpr int plane_in = SPT * ROWS_IN;
    constexpr int plane_p = (SPP * ROWS_P + 31) / 32 * 32;
    float *pbuf = stages + NSTT * a.buf_floats;  // ring of NPS intermediate planes
    const uint32_t chunk_bytes = (uint32_t)(plane_in * ZC * 4);
    const int tid = threadIdx.x;

    const int tile = blockIdx.x;
    const int txy = tile % a.ntiles_xy, zc = tile / a.ntiles_xy;
    const int tx = txy % a.tiles_x, ty = txy / a.tiles_x;
    const int x0 = tx * TX3, y0 = ty * TY3;
    const int z0 = zc * a.zchunk, z1 = min(a.nz, z0 + a.zchunk);
    const int zin0 = z0 - 2 * R, nin = (z1 - z0) + 4 * R;  // input planes streamed
    const int nchunks = (nin + ZC - 1) / ZC;

    if (tid == 0) {
        prefetch_tensormap(&map);
        for (int s = 0; s < NSTT; ++s) {
            mbar_init(&bars[s], 1);
            mbar_init(&empty[s], 1);
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (tid >= NCT) {
        // producer: chunk c (input planes 4c .. 4c+3) into stage c % NSTT once
        // the consumers released the chunk NSTT earlier
        if (tid != NCT) return;
        int c = 0;
        for (; c < nchunks; ++c) {
            const int s = c % NSTT;
            if (c >= NSTT && !mbar_wait_bounded(&empty[s], ((c / NSTT) - 1) & 1, a.wait_ns)) {
                record_status(a.status, DEV_TIMEOUT);
                break;
            }
            // (fault_withhold_copy is a test hook: the first chunk is never
            // requested, so the consumers' bounded waits and then this
            // warp's must run out and report a timeout)
            if (c == 0 && a.fault_withhold_copy) continue;
            mbar_arrive_expect_tx(&bars[s], chunk_bytes);
            tma_load_3d(stages + s * a.buf_floats, &map, &bars[s], a.map_x0 + x0 - HXT,
                        a.map_y0 + y0 - 2 * R, a.map_z0 + zin0 + c * ZC);
        }
        for (int q = max(0, c - NSTT); q < c; ++q)
            mbar_wait_bounded(&bars[q % NSTT], (q / NSTT) & 1, a.wait_ns);
        return;
    }

    // first sweep: strip s1 of row r1 of the intermediate block, whose column 0
    // is x0-4 and row 0 is y0-R
    const bool do1 = tid < S1X * ROWS_P;
    const int s1 = tid % S1X, r1 = tid / S1X;
    // second sweep: strip s2 of row r2 of the output tile
    const bool do2 = tid < (TX3 / 4) * TY3;
    const int s2 = tid % (TX3 / 4), r2 = tid / (TX3 / 4);
    const int X = x0 + 4 * s2, Y = y0 + r2;
    const bool live = do2 && Y < a.ny && X < a.nx;
    const bool vec4 = a.dst_vec4 && X + 3 < a.nx;

    float w1[W][4], w2[W][4];
#pragma unroll
    for (int i = 0; i < W; ++i)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            w1[i][v] = 0.f;
            w2[i][v] = 0.f;
        }

    // adds one plane (rows base_row-R .. base_row+R of `pl`, columns from
    // `col`) into the window slots
    auto accumulate = [&](float (&w)[W][4], const float *pl, int pitch, int base_row) {
#pragma unroll
        for (int dy = -R; dy <= R; ++dy) {
            float seg[NSEG];
            const float4 *rp = reinterpret_cast<const float4 *>(pl + (base_row + dy) * pitch);
#pragma unroll
            for (int k = 0; k < NSEG / 4; ++k) {
                const float4 t = rp[k];
                seg[4 * k] = t.x;
                seg[4 * k + 1] = t.y;
                seg[4 * k + 2] = t.z;
                seg[4 * k + 3] = t.w;
            }
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const int az = R - i;
#pragma unroll
                for (int dx = -R; dx <= R; ++dx) {
                    if (TP::nz(az, dy, dx)) {
                        const float wt = a.c[((az + R) * W + (dy + R)) * W + (dx + R)];
#pragma unroll
                        for (int v = 0; v < 4; ++v) w[i][v] = fmaf(wt, seg[v + dx + RP], w[i][v]);
                    }
                }
            }
        }
    };
    auto shift = [&](float (&w)[W][4]) {
#pragma unroll
        for (int i = 0; i < W - 1; ++i)
#pragma unroll
            for (int v = 0; v < 4; ++v) w[i][v] = w[i + 1][v];
#pragma unroll
        for (int v = 0; v < 4; ++v) w[W - 1][v] = 0.f;
    };

    bool failed = false;
    for (int c = 0; c < nchunks; ++c) {
        const int s = c % NSTT;
        const bool landed = mbar_wait_bounded(&bars[s], (c / NSTT) & 1, a.wait_ns);
        if (consumers_any3<NCT>(!landed)) {
            if (!landed) record_status(a.status, DEV_TIMEOUT);
            failed = true;
            break;
        }
        const float *chunk = stages + s * a.buf_floats;
        const int pend = min(ZC, nin - c * ZC);  // planes of this chunk
        // 1. first sweep over the chunk's planes: input plane p into w1; the
        // intermediate plane p - 2R completes once 2R+1 input planes are in,
        // and goes to slot (p - 2R) mod 8 of the plane ring
        if (do1) {
#pragma unroll 1
            for (int q = 0; q < pend; ++q) {
                const int p = c * ZC + q;
                // staged column of intermediate column 4*s1 is 4*s1 + 4; the
                // strip's loads start RP columns to its left
                accumulate(w1, chunk + q * plane_in + 4 * s1 + 4 - RP, SPT, r1 + R);
                if (p >= 2 * R) {
                    float *dst = pbuf + ((p - 2 * R) & (NPS - 1)) * plane_p + r1 * SPP + 4 * s1;
                    *reinterpret_cast<float4 *>(dst) = make_float4(w1[0][0], w1[0][1], w1[0][2], w1[0][3]);
                }
                shift(w1);
            }
        }
        // the chunk's intermediate planes are in the ring and its stage has
        // been read by every consumer
        NamedBarrier<NCT>::sync();
        if (tid == 0) mbar_arrive(&empty[s]);
        // 2. second sweep over the same planes: intermediate plane qi into w2;
        // output plane z0 - 2R + qi completes once 2R+1 of them are in.  The
        // slots written by the next chunk were last read before this barrier.
        if (do2) {
#pragma unroll 1
            for (int q = 0; q < pend; ++q) {
                const int qi = c * ZC + q - 2 * R;
                if (qi < 0) continue;
                accumulate(w2, pbuf + (qi & (NPS - 1)) * plane_p + 4 * s2 + 4 - RP, SPP, r2 + R);
                const int zo = z0 - 2 * R + qi;
                if (zo >= z0 && live) {
                    float *row = a.dst + zo * a.dst_pz + Y * a.dst_py;
                    if (vec4) {
                        *reinterpret_cast<float4 *>(row + X) =
                            make_float4(w2[0][0], w2[0][1], w2[0][2], w2[0][3]);
                    } else {
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            if (X + v < a.nx) row[X + v] = w2[0][v];
                    }
                }
                shift(w2);
            }
        }
    }
    if (consumers_any3<NCT>(failed) || a.dst_gw <= 0) return;
    refresh_ghosts3<NCT>(a, dst_of(a), x0, y0, z0, z1, tid);
}

}  // namespace

namespace {

template <int RB, int M, int PAT>
cudaError_t prepare_tb()
{
    return smem_optin((const void *)k_sweep3d_tb<RB, M, PAT>);
}

template <int RB, int M, int PAT>
cudaError_t launch_tb(const CUtensorMap &map, const Sweep3DArgs &a, int grid, size_t smem,
                      cudaStream_t s)
{
    cudaError_t e = prepare_tb<RB, M, PAT>();
    if (e != cudaSuccess) return e;
    k_sweep3d_tb<RB, M, PAT><<<grid, NTT, smem, s>>>(map, a);
    return cudaGetLastError();
}

// Fused pairs of sweeps: folded radius R = m*r <= 2 (one thread per
// first-sweep strip of the tile plus its rim).
#define SG_SWEEP3D_TB_LIST(X) X(1, 1, PAT_STAR) X(1, 2, PAT_STAR) X(1, 1, PAT_BOX) X(1, 2, PAT_BOX) \
    X(2, 1, PAT_STAR) X(2, 1, PAT_BOX)

}  // namespace

bool sweep3d_tb_supported(int rb, int m, int pattern)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_) return true;
    SG_SWEEP3D_TB_LIST(SG_X)
#undef SG_X
    return false;
}

size_t sweep3d_tb_smem_bytes(int R, int *buf_floats)
{
    const int bf = round_up(SPT * (TY3 + 4 * R) * ZC, 32);
    const int pp = round_up(SPP * (TY3 + 2 * R), 32);
    if (buf_floats) *buf_floats = bf;
    return 1024 + ((size_t)NSTT * bf + (size_t)NPS * pp) * 4;
}

int sweep3d_tb_halo_x() { return HXT; }

cudaError_t launch_sweep3d_tb(int rb, int m, int pattern, const CUtensorMap &map,
                              const Sweep3DArgs &a, int grid, size_t smem, cudaStream_t s)
{
#define SG_X(RB_, M_, P_) \
    if (rb == RB_ && m == M_ && pattern == P_) return launch_tb<RB_, M_, P_>(map, a, grid, smem, s);
    SG_SWEEP3D_TB_LIST(SG_X)
#undef SG_X
    return cudaErrorInvalidValue;
}

}  // namespace sg
