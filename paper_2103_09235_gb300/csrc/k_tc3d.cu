// Folded 3D box sweep on the tcgen05 tensor cores (BF16 hi/lo, FP32 accumulate).
//
// One sweep applies the folded weights c^(m) (radius R = m*r, Section 3.2) of a
// 3D stencil.  Section 3.3 treats a 3D grid as layers of 2D planes: output
// plane z is the sum over the plane offsets dz of 2D folded stencils, the
// weights c^(m)[dz][.][.], applied to input plane z+dz.  Each of those is the
// banded-Toeplitz contraction of the 2D kernel (k_tc2d.cu):
//   out[z][y][x0+n] = sum_dz sum_dy sum_k X[z+dz][y+dy][x0-R+k] * T_{dz,dy}[n][k],
// so a tile (128 rows x 32 columns of one output plane) runs 2R+1 plane
// steps, each a staged tile of plane z+dz times the 2R+1 Toeplitz panels of
// that plane offset, all accumulated in one tensor-memory accumulator.
//
// Stages: the producer warp loads, per plane step, the FP32 tile of plane
// z+dz (3D TMA box) into a staging slot, and the step's 2R+1 panels (a bulk
// copy from the plan's panel array, L2-resident) into a panel slot; the
// converters centre and split the tile into BF16 hi/lo A operands; the MMA
// issuer runs the step's (2R+1) x 3 K steps x 2 MMAs and releases the A
// operand and the panel slot with commits; after the last plane step it
// commits the accumulator to the epilogue, which adds mu * sum(c), stores the
// tile and, into a padded destination, its periodic ghost copies.
//
// Warp roles (384 threads) and bounded waits as in k_tc2d.cu.
#include <cuda_bf16.h>

#include <vector>

#include "device_common.cuh"
#include "tc_common.cuh"
#include "internal.h"

namespace sg {
namespace {

using namespace tcore;

constexpr int NT = kTcThreads;
constexpr int PANEL_BYTES = kTcPanelElems * 2;  // one (dz, dy): [T_hi ; T_lo], 64 rows x 48 K
constexpr int LBO_B = 64 * 16;
constexpr uint32_t TMEM_COLS = 128;             // two 64-column accumulators

struct Ctl {
    uint64_t stage_full[2], stage_empty[2], pan_full[2], pan_empty[2];
    uint64_t a_full[2], a_empty[2], d_full[2], d_empty[2];
    uint32_t tmem_base;
    int abort;
    int epi_ok[2][4];
};

// Shared-memory layout: control block | A operands (2 buffers x hi/lo) |
// FP32 staging (2 slots) | panel slots (2 x (2R+1) panels).
struct Tc3Layout {
    uint32_t a_bytes, off_a, stage_bytes, off_stage, pan_bytes, off_pan, total;
};

__host__ __device__ inline Tc3Layout tc3_layout(int R, int rows, int rows_p, int box_w)
{
    Tc3Layout L;
    L.a_bytes = (uint32_t)(kTcKC * rows_p * 16);
    L.off_a = 1024;
    L.off_stage = (L.off_a + 4 * L.a_bytes + 127) / 128 * 128;
    L.stage_bytes = ((uint32_t)(rows * box_w * 4) + 127) / 128 * 128;
    L.pan_bytes = (uint32_t)(2 * R + 1) * PANEL_BYTES;
    L.off_pan = L.off_stage + 2 * L.stage_bytes;
    L.total = L.off_pan + 2 * L.pan_bytes;
    return L;
}

// The periodic copies of output (X, Y, Z) across the destination's ghost band.
__device__ __forceinline__ void store_point_3d(const TC3DArgs &a, int X, int Y, int Z, float v)
{
    const int nx = a.t.nx, ny = a.t.ny, nz = a.nz, gw = a.t.dst_gw;
    // the periodic image shift along each axis: 0, +n (near the low edge) or
    // -n (near the high edge); at most one of the two for gw <= n / 2
    const int ex = X < gw ? nx : (X >= nx - gw ? -nx : 0);
    const int ey = Y < gw ? ny : (Y >= ny - gw ? -ny : 0);
    const int ez = Z < gw ? nz : (Z >= nz - gw ? -nz : 0);
    for (int iz = 0; iz < 2; ++iz) {
        if (iz && !ez) break;
        for (int iy = 0; iy < 2; ++iy) {
            if (iy && !ey) break;
            for (int ix = 0; ix < 2; ++ix) {
                if (ix && !ex) break;
                if (ix || iy || iz)
                    a.t.dst[(int64_t)(Z + iz * ez) * a.dst_pz + (int64_t)(Y + iy * ey) * a.t.dst_py +
                            X + ix * ex] = v;
            }
        }
    }
}

__global__ void __launch_bounds__(NT, 1)
    k_tc3d(const __grid_constant__ CUtensorMap map, const __grid_constant__ TC3DArgs a3)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const TC2DArgs &a = a3.t;
    Ctl *ctl = reinterpret_cast<Ctl *>(smem);
    const int R = a.R, W = 2 * R + 1;
    const Tc3Layout L = tc3_layout(R, a.rows, a.rows_p, a.box_w);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_u32(smem);

    if (tid == 0) {
        prefetch_tensormap(&map);
        for (int s = 0; s < 2; ++s) {
            mbar_init(&ctl->stage_full[s], 1);
            mbar_init(&ctl->stage_empty[s], 128);
            mbar_init(&ctl->pan_full[s], 1);
            mbar_init(&ctl->pan_empty[s], 1);
            mbar_init(&ctl->a_full[s], 128);
            mbar_init(&ctl->a_empty[s], 1);
            mbar_init(&ctl->d_full[s], 1);
            mbar_init(&ctl->d_empty[s], 128);
        }
        ctl->abort = 0;
        // self-check: the layout the operands' descriptors address must lie
        // inside the shared memory this launch has
        uint32_t dyn = 0;
        asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        if (dyn < L.total) {
            record_status(a.status, DEV_CHECK);
            ctl->abort = 1;
        }
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&ctl->tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;
    const int first = blockIdx.x, step = gridDim.x;
    const int tiles_xy = a.tiles_x * a3.tiles_y;
    const bool skip = *(volatile int *)&ctl->abort != 0;  // the self-check failed

    if (skip) {
        // nothing but the tensor-memory release below
    } else if (warp == 0) {
        // ---- producer: per plane step, the tile of plane z+dz and the step's panels
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)(a.rows * a.box_w * 4);
            int j = 0, last = -1;  // j counts plane steps
            bool ok = true;
            for (int tile = first; tile < a.ntiles && ok; tile += step) {
                const int z = tile / tiles_xy, rem = tile % tiles_xy;
                const int ty = rem / a.tiles_x, tx = rem % a.tiles_x;
                for (int dz = 0; dz < W; ++dz, ++j) {
                    const int s = j & 1, k = j >> 1;
                    if (!wait_or_abort(&ctl->stage_empty[s], (k & 1) ^ 1, ctl, a) ||
                        !wait_or_abort(&ctl->pan_empty[s], (k & 1) ^ 1, ctl, a)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&ctl->stage_full[s], bytes);
                    tma_load_3d(smem + L.off_stage + s * L.stage_bytes, &map, &ctl->stage_full[s],
                                a.map_x0 + tx * kTcN - a.halo_x, a.map_y0 + ty * kTcM - R,
                                a3.map_z0 + z + dz - R);
                    mbar_arrive_expect_tx(&ctl->pan_full[s], L.pan_bytes);
                    bulk_load(smem + L.off_pan + s * L.pan_bytes,
                              reinterpret_cast<const unsigned char *>(a.panels) +
                                  (size_t)dz * L.pan_bytes,
                              L.pan_bytes, &ctl->pan_full[s]);
                    last = j;
                }
            }
            if (ctl->abort && last >= 0) {
                drain_wait(&ctl->stage_full[last & 1], (last >> 1) & 1, a);
                drain_wait(&ctl->pan_full[last & 1], (last >> 1) & 1, a);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            const uint32_t id64 = idesc_bf16(kTcM, 64), id32 = idesc_bf16(kTcM, 32);
            const uint32_t lbo_a = (uint32_t)a.rows_p * 16;
            const uint32_t kstep_a = (2 * lbo_a) >> 4, kstep_b = (2 * LBO_B) >> 4;
            int i = 0, j = 0, last_j = -1;  // last_j: the last plane step committed
            bool ok = true;
            for (int tile = first; tile < a.ntiles && ok; tile += step, ++i) {
                const int sd = i & 1, kd = i >> 1;
                if (a.fault_withhold_mma) break;  // test hook, as in k_tc2d.cu
                if (!wait_or_abort(&ctl->d_empty[sd], (kd & 1) ^ 1, ctl, a)) break;
                const uint32_t dt = tmem + (uint32_t)(sd * 64);
                for (int dz = 0; dz < W; ++dz, ++j) {
                    const int s = j & 1, k = j >> 1;
                    if (!wait_or_abort(&ctl->a_full[s], k & 1, ctl, a) ||
                        !wait_or_abort(&ctl->pan_full[s], k & 1, ctl, a)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_hi = sbase + L.off_a + (2 * s) * L.a_bytes;
                    const uint64_t dh0 = smem_desc(a_hi, lbo_a, 128);
                    const uint64_t dl0 = smem_desc(a_hi + L.a_bytes, lbo_a, 128);
                    const uint64_t db0 = smem_desc(sbase + L.off_pan + s * L.pan_bytes, LBO_B, 128);
                    for (int ai = 0; ai < W; ++ai) {
                        const uint32_t oa = (uint32_t)ai, ob = (uint32_t)ai * (PANEL_BYTES >> 4);
#pragma unroll
                        for (int kk = 0; kk < kTcK / 16; ++kk) {
                            const uint64_t d_a = oa + kk * kstep_a, d_b = ob + kk * kstep_b;
                            const uint32_t acc = (dz == 0 && ai == 0 && kk == 0) ? 0u : 1u;
                            if (a.terms == 3) {
                                mma_bf16(dt, dh0 + d_a, db0 + d_b, id64, acc);
                                mma_bf16(dt, dl0 + d_a, db0 + d_b, id32, 1u);
                            } else {
                                mma_bf16(dt, dh0 + d_a, db0 + d_b, id32, acc);
                            }
                        }
                    }
                    mma_commit(&ctl->a_empty[s]);
                    mma_commit(&ctl->pan_empty[s]);
                    last_j = j;
                }
                if (!ok) break;
                mma_commit(&ctl->d_full[sd]);
            }
            // a commit tracks every MMA issued before it: after an abort, the
            // last plane step's commit covers all MMAs still in flight
            if (ctl->abort && last_j >= 0)
                drain_wait(&ctl->a_empty[last_j & 1], (last_j >> 1) & 1, a);
        }
    } else if (warp >= 4 && warp < 8) {
        // ---- converters: FP32 staging -> centred BF16 hi/lo operands
        const int ct = tid - 128;
        const float mu = a.mean_sum ? (float)(a.mean_sum[0] * a.inv_n) : 0.f;
        const int off = a.halo_x - R;
        const uint32_t lbo_a = (uint32_t)a.rows_p * 16;
        int j = 0;
        bool ok = true;
        for (int tile = first; tile < a.ntiles && ok; tile += step) {
            for (int dz = 0; dz < W; ++dz, ++j) {
                const int s = j & 1, k = j >> 1;
                bool w = wait_or_abort(&ctl->stage_full[s], k & 1, ctl, a);
                w = w && wait_or_abort(&ctl->a_empty[s], (k & 1) ^ 1, ctl, a);
                if (!__all_sync(0xffffffffu, w)) {
                    ok = false;
                    break;
                }
                const float *st =
                    reinterpret_cast<const float *>(smem + L.off_stage + s * L.stage_bytes);
                unsigned char *ahi = smem + L.off_a + (2 * s) * L.a_bytes;
                unsigned char *alo = ahi + L.a_bytes;
                for (int it = ct; it < a.rows * kTcKC; it += 128) {
                    const int kc = it % kTcKC, r = it / kTcKC;
                    const float *src = st + r * a.box_w + kc * 8 + off;
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = src[e] - mu;
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * e]);
                        const __nv_bfloat16 h1 = __float2bfloat16_rn(v[2 * e + 1]);
                        const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * e] - __bfloat162float(h0));
                        const __nv_bfloat16 l1 =
                            __float2bfloat16_rn(v[2 * e + 1] - __bfloat162float(h1));
                        hw[e] = (uint32_t)__bfloat16_as_ushort(h0) |
                                ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                        lw[e] = (uint32_t)__bfloat16_as_ushort(l0) |
                                ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                    }
                    const uint32_t o = kc * lbo_a + r * 16;
                    *reinterpret_cast<uint4 *>(ahi + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4 *>(alo + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
                fence_proxy_async_smem();
                mbar_arrive(&ctl->stage_empty[s]);
                mbar_arrive(&ctl->a_full[s]);
            }
        }
    } else if (warp >= 8) {
        // ---- epilogue: tensor memory -> registers -> global memory
        const int q = warp - 8;
        const float mu = a.mean_sum ? (float)(a.mean_sum[0] * a.inv_n) : 0.f;
        const float musum = mu * a.sum_c;
        int i = 0;
        for (int tile = first; tile < a.ntiles; tile += step, ++i) {
            const int s = i & 1, k = i >> 1;
            __syncwarp();  // the warp is converged before its aligned tensor-memory loads
            bool ok = wait_or_abort(&ctl->d_full[s], k & 1, ctl, a);
            ok = __all_sync(0xffffffffu, ok);
            if (lane == 0) ctl->epi_ok[s][q] = ok ? 1 : 0;
            __syncwarp();
            epi_barrier();
            const volatile int *votes = ctl->epi_ok[s];
            if (!(votes[0] && votes[1] && votes[2] && votes[3])) break;
            tc_fence_after();
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(s * 64);
            float v0[32], v1[32];
            tmem_ld32(taddr, v0);
            if (a.terms == 3) tmem_ld32(taddr + 32, v1);
            tmem_ld_wait();
            tc_fence_before();
            mbar_arrive(&ctl->d_empty[s]);
            const int z = tile / tiles_xy, rem = tile % tiles_xy;
            const int ty = rem / a.tiles_x, tx = rem % a.tiles_x;
            const int Y = ty * kTcM + 32 * q + lane;
            const int X0 = tx * kTcN;
            if (Y < a.ny) {
                float o[32];
#pragma unroll
                for (int n = 0; n < 32; ++n) o[n] = v0[n] + (a.terms == 3 ? v1[n] : 0.f) + musum;
                float *row = a.dst + (int64_t)z * a3.dst_pz + (int64_t)Y * a.dst_py + X0;
                if (a.dst_vec4 && X0 + 32 <= a.nx) {
#pragma unroll
                    for (int n = 0; n < 32; n += 4)
                        *reinterpret_cast<float4 *>(row + n) =
                            make_float4(o[n], o[n + 1], o[n + 2], o[n + 3]);
                } else {
#pragma unroll
                    for (int n = 0; n < 32; ++n)
                        if (X0 + n < a.nx) row[n] = o[n];
                }
                const int gw = a.dst_gw;
                if (gw > 0 && (X0 < gw || X0 + 32 > a.nx - gw || Y < gw || Y >= a.ny - gw ||
                               z < gw || z >= a3.nz - gw)) {
#pragma unroll
                    for (int n = 0; n < 32; ++n)
                        if (X0 + n < a.nx) store_point_3d(a3, X0 + n, Y, z, o[n]);
                }
            }
            __syncwarp();
        }
    }

    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

bool tc3d_supported(int R) { return R >= 1 && R <= kTc3MaxR; }

void tc3d_geometry(int R, int *rows, int *rows_p, int *box_w, int *halo_x)
{
    *halo_x = round_up(R, 4);
    *rows = kTcM + 2 * R;
    *rows_p = *rows | 1;
    *box_w = round_up(kTcK + *halo_x - R, 4);
}

size_t tc3d_smem_bytes(int R)
{
    int rows, rows_p, box_w, hx;
    tc3d_geometry(R, &rows, &rows_p, &box_w, &hx);
    return tc3_layout(R, rows, rows_p, box_w).total;
}

size_t tc3d_panel_elems(int R) { return (size_t)(2 * R + 1) * (2 * R + 1) * kTcPanelElems; }

double tc3d_build_panels(const double *cm, int R, uint16_t *out)
{
    const int W = 2 * R + 1, N = W * W * W;
    auto rnd = [](double v) { return (double)__bfloat162float(__double2bfloat16(v)); };
    std::vector<double> hi(N), lo(N);
    double target = 0.0, got = 0.0;
    for (int i = 0; i < N; ++i) {
        hi[i] = rnd(cm[i]);
        lo[i] = rnd(cm[i] - hi[i]);
        target += cm[i];
        got += hi[i] + lo[i];
    }
    // mass correction: the centre tap's lo absorbs the rounding of the sum
    const int c = (R * W + R) * W + R;
    lo[c] = rnd(lo[c] + (target - got));
    // panels ordered (dz, dy): the 2R+1 panels of one plane offset are contiguous
    for (int dz = 0; dz < W; ++dz)
        for (int dy = 0; dy < W; ++dy) {
            uint16_t *panel = out + ((size_t)dz * W + dy) * kTcPanelElems;
            for (int n = 0; n < 64; ++n) {
                const int nn = n & 31;
                const std::vector<double> &src = n < 32 ? hi : lo;
                for (int k = 0; k < kTcK; ++k) {
                    const int b = k - nn - R;  // column offset
                    double w = 0.0;
                    if (b >= -R && b <= R) w = src[(dz * W + dy) * W + (b + R)];
                    panel[((k / 8) * 64 + n) * 8 + (k % 8)] =
                        __bfloat16_as_ushort(__double2bfloat16(w));
                }
            }
        }
    return target;
}

cudaError_t launch_tc3d(const CUtensorMap &map, const TC3DArgs &a, int grid, size_t smem,
                        cudaStream_t s)
{
    const cudaError_t e = smem_optin((const void *)k_tc3d);
    if (e != cudaSuccess) return e;
    k_tc3d<<<grid, NT, smem, s>>>(map, a);
    return cudaGetLastError();
}

}  // namespace sg
