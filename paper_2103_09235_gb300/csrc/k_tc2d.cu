// Folded 2D box sweep on the tcgen05 tensor cores: BF16 hi/lo (kind::f16) or
// TF32 hi/lo (kind::tf32) operands, FP32 accumulation.
//
// One sweep applies the folded weights c^(m) (radius R = m*r, Section 3.2):
//   out[y][x0+n] = sum_{a=-R..R} sum_k X[y+a][x0-R+k] * T_a[n][k],
// where T_a is the banded Toeplitz matrix holding row a of c^(m)
// (T_a[n][k] = c[a][k-n-R] for 0 <= k-n <= 2R).  This is the paper's vertical
// and horizontal folding (Section 3.3, Eq. vfold and Eq. horifold) written as
// 2R+1 dense contractions over the tile's 48-column window, one per row
// offset a; the partial sums the paper keeps in vector registers accumulate
// in tensor memory instead.
//
// Tile: M = 128 grid rows (the MMA's M) x 32 output columns.  The FP32 tile
// plus R halo rows arrives by TMA; converter warps subtract the grid mean mu,
// split v = x - mu into v_hi = rnd(v) and v_lo = rnd(v - v_hi) (rnd: BF16 or
// TF32) and write both in the no-swizzle K-major core-matrix layout, in which
// every row is 16 bytes away from the next within a 16-byte K chunk.  The
// operand "rows y+a" for offset a is then the same matrix with its descriptor
// start moved by 16*(a+R) bytes, so no shifted copies are made.  An MMA takes
// 32 bytes of K per row (16 BF16 or 8 TF32 values); per (a, K step) one MMA of
// N = 64 multiplies v_hi by [T_a,hi ; T_a,lo] and one of N = 32 multiplies
// v_lo by T_a,hi; the two halves of the accumulator are added in the epilogue
// together with mu * sum(c).  Toeplitz panels stay resident in shared memory.
// TF32 operands take twice the bytes: its A operand is single-buffered so that
// the panels of R <= 4 still fit, and it has no single-product variant.
//
// Warp roles (384 threads): warp 0 issues TMA loads, warp 1 owns tensor
// memory and issues the MMAs (one thread), warps 4-7 convert, warps 8-11
// drain the accumulator to global memory.  Every wait is bounded; a wait that
// runs out records a timeout, raises an abort flag that ends the other roles'
// waits, lets in-flight copies and MMAs land, frees tensor memory and returns.
#include <cuda_bf16.h>
#include <string.h>

#include <vector>

#include "device_common.cuh"
#include "tc_common.cuh"
#include "internal.h"

namespace sg {
namespace {

using namespace tcore;

constexpr int NT = kTcThreads;
constexpr int LBO_B = 64 * 16;       // K-chunk stride of a panel (64 rows x 16 B)
constexpr uint32_t TMEM_COLS = 128;  // two 64-column accumulators

// Operand format: EB bytes per element (2: BF16, 4: TF32).
template <int EB>
struct Fmt {
    static constexpr int KCH = kTcK * EB / 16;      // 16-byte K chunks per row of the window
    static constexpr int KSTEPS = kTcK * EB / 32;   // MMAs per (row offset, term)
    static constexpr int PANEL_BYTES = 64 * kTcK * EB;
    static constexpr int NSA = EB == 2 ? 2 : 1;     // A-operand buffers
};

// kind::tf32 instruction descriptor: FP32 accumulator, TF32 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

template <int EB>
__device__ __forceinline__ void mma_fmt(uint32_t d, uint64_t a, uint64_t b, uint32_t id,
                                        uint32_t acc)
{
    if constexpr (EB == 2) mma_bf16(d, a, b, id, acc);
    else mma_tf32(d, a, b, id, acc);
}

// FP32 -> TF32 (round to nearest, ties away), as a 32-bit pattern.
__device__ __forceinline__ uint32_t to_tf32(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

// Barriers, tensor-memory address and abort flag shared by the warp roles.
struct Ctl {
    uint64_t stage_full[2], stage_empty[2], a_full[2], a_empty[2], d_full[2], d_empty[2];
    uint32_t tmem_base;
    int abort;
    int epi_ok[2][4];  // per-iteration votes of the four epilogue warps
};

// Shared-memory layout (bytes from the 1024-aligned base):
//   [0, 1024)           control block (barriers, tensor-memory address, abort flag)
//   A operands          buffer s, part h (0 = hi, 1 = lo) at off_a + (2s+h)*a_bytes
//   FP32 staging        stage s at off_stage + s*stage_bytes (TMA boxes)
//   Toeplitz panels     (2R+1) * PANEL_BYTES
//   output tile         128 x 32 FP32, 128-byte swizzled (only with the TMA store)
struct TcLayout {
    uint32_t a_bytes, off_a, stage_bytes, off_stage, off_b, off_out, total;
};

template <int EB>
__host__ __device__ inline TcLayout tc_layout(int R, int rows, int rows_p, int box_w, int tma_store)
{
    using F = Fmt<EB>;
    TcLayout L;
    L.a_bytes = (uint32_t)(F::KCH * rows_p * 16);
    L.off_a = 1024;
    L.off_stage = (L.off_a + 2 * F::NSA * L.a_bytes + 127) / 128 * 128;
    L.stage_bytes = ((uint32_t)(rows * box_w * 4) + 127) / 128 * 128;
    L.off_b = L.off_stage + 2 * L.stage_bytes;
    L.off_out = (L.off_b + (uint32_t)(2 * R + 1) * F::PANEL_BYTES + 1023) / 1024 * 1024;
    L.total = tma_store ? L.off_out + kTcM * kTcN * 4
                        : L.off_b + (uint32_t)(2 * R + 1) * F::PANEL_BYTES;
    return L;
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(smem_u32(src)), "r"(x), "r"(y)
        : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Eight staged FP32 values of row r starting at column c0 (off: the window's
// shift inside the staged box), minus mu.
__device__ __forceinline__ void load8(const float *src, int off, float mu, float (&v)[8])
{
    if (off == 0) {  // 16-byte aligned: two vector loads
        const float4 p0 = reinterpret_cast<const float4 *>(src)[0];
        const float4 p1 = reinterpret_cast<const float4 *>(src)[1];
        v[0] = p0.x; v[1] = p0.y; v[2] = p0.z; v[3] = p0.w;
        v[4] = p1.x; v[5] = p1.y; v[6] = p1.z; v[7] = p1.w;
    } else if ((off & 1) == 0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 p = reinterpret_cast<const float2 *>(src)[e];
            v[2 * e] = p.x;
            v[2 * e + 1] = p.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = src[e];
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] -= mu;
}

template <int EB>
__global__ void __launch_bounds__(NT, 1)
    k_tc2d(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap dmap,
           const __grid_constant__ TC2DArgs a)
{
    using F = Fmt<EB>;
    extern __shared__ __align__(1024) unsigned char smem[];
    Ctl *ctl = reinterpret_cast<Ctl *>(smem);
    const TcLayout L = tc_layout<EB>(a.R, a.rows, a.rows_p, a.box_w, a.tma_store);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_u32(smem);
    const int R = a.R;

    if (tid == 0) {
        prefetch_tensormap(&map);
        for (int s = 0; s < 2; ++s) {
            mbar_init(&ctl->stage_full[s], 1);
            mbar_init(&ctl->stage_empty[s], 128);
            mbar_init(&ctl->a_full[s], 128);
            mbar_init(&ctl->a_empty[s], 1);
            mbar_init(&ctl->d_full[s], 1);
            mbar_init(&ctl->d_empty[s], 128);
        }
        ctl->abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&ctl->tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    {  // resident Toeplitz panels
        const int n16 = (2 * R + 1) * F::PANEL_BYTES / 16;
        const uint4 *gp = reinterpret_cast<const uint4 *>(a.panels);
        uint4 *sp = reinterpret_cast<uint4 *>(smem + L.off_b);
        for (int i = tid; i < n16; i += NT) sp[i] = gp[i];
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;
    const int first = blockIdx.x, step = gridDim.x;

    if (warp == 0) {
        // ---- producer: FP32 tile + halo by TMA
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)(a.rows * a.box_w * 4);
            int i = 0, last = -1;
            for (int tile = first; tile < a.ntiles; tile += step, ++i) {
                const int s = i & 1, k = i >> 1;
                if (!wait_or_abort(&ctl->stage_empty[s], (k & 1) ^ 1, ctl, a)) break;
                const int per_plane = a.tiles_x * a.tiles_y;
                const int pl = tile / per_plane, t2 = tile % per_plane;
                const int tx = t2 % a.tiles_x, ty = t2 / a.tiles_x;
                // rows of the source plane dz away from the output plane (2D: pl = dz = 0)
                const int y_src = a.map_y0 + (int)((int64_t)(pl + a.dz) * a.src_plane_rows) +
                                  ty * kTcM - R;
                mbar_arrive_expect_tx(&ctl->stage_full[s], bytes);
                tma_load_2d(smem + L.off_stage + s * L.stage_bytes, &map, &ctl->stage_full[s],
                            a.map_x0 + tx * kTcN - a.halo_x, y_src);
                last = i;
            }
            if (ctl->abort && last >= 0)
                drain_wait(&ctl->stage_full[last & 1], (last >> 1) & 1, a);
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            const uint32_t id64 = EB == 2 ? idesc_bf16(kTcM, 64) : idesc_tf32(kTcM, 64);
            const uint32_t id32 = EB == 2 ? idesc_bf16(kTcM, 32) : idesc_tf32(kTcM, 32);
            const uint32_t lbo_a = (uint32_t)a.rows_p * 16;
            int i = 0, last = -1;
            for (int tile = first; tile < a.ntiles; tile += step, ++i) {
                const int s = i & 1, k = i >> 1;                       // accumulator
                const int sa = i % F::NSA, ka = i / F::NSA;            // A operand
                // (fault_withhold_mma is a test hook: the issuer stops before its
                // first MMA, as if its completions were lost, so every other
                // role's bounded wait must run out and report a timeout)
                if (a.fault_withhold_mma) break;
                if (!wait_or_abort(&ctl->a_full[sa], ka & 1, ctl, a)) break;
                if (!wait_or_abort(&ctl->d_empty[s], (k & 1) ^ 1, ctl, a)) break;
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(s * 64);
                const uint32_t a_hi = sbase + L.off_a + (2 * sa) * L.a_bytes;
                // descriptors of the first (row offset, K step); the others differ
                // only in the start-address field, by whole 16-byte units
                const uint64_t dh0 = smem_desc(a_hi, lbo_a, 128);
                const uint64_t dl0 = smem_desc(a_hi + L.a_bytes, lbo_a, 128);
                const uint64_t db0 = smem_desc(sbase + L.off_b, LBO_B, 128);
                const uint32_t kstep_a = (2 * lbo_a) >> 4, kstep_b = (2 * LBO_B) >> 4;
                if (a.terms == 3) {
                    mma_fmt<EB>(dt, dh0, db0, id64, 0u);
                    mma_fmt<EB>(dt, dl0, db0, id32, 1u);
                    for (int ai = 0; ai <= 2 * R; ++ai) {
                        const uint32_t oa = (uint32_t)ai, ob = (uint32_t)ai * (F::PANEL_BYTES >> 4);
#pragma unroll
                        for (int kk = (ai == 0 ? 1 : 0); kk < F::KSTEPS; ++kk) {
                            const uint64_t d_a = oa + kk * kstep_a, d_b = ob + kk * kstep_b;
                            mma_fmt<EB>(dt, dh0 + d_a, db0 + d_b, id64, 1u);
                            mma_fmt<EB>(dt, dl0 + d_a, db0 + d_b, id32, 1u);
                        }
                    }
                } else {
                    mma_fmt<EB>(dt, dh0, db0, id32, 0u);
                    for (int ai = 0; ai <= 2 * R; ++ai) {
                        const uint32_t oa = (uint32_t)ai, ob = (uint32_t)ai * (F::PANEL_BYTES >> 4);
#pragma unroll
                        for (int kk = (ai == 0 ? 1 : 0); kk < F::KSTEPS; ++kk)
                            mma_fmt<EB>(dt, dh0 + oa + kk * kstep_a, db0 + ob + kk * kstep_b, id32,
                                        1u);
                    }
                }
                mma_commit(&ctl->a_empty[sa]);
                mma_commit(&ctl->d_full[s]);
                last = i;
            }
            if (ctl->abort && last >= 0) drain_wait(&ctl->d_full[last & 1], (last >> 1) & 1, a);
        }
    } else if (warp >= 4 && warp < 8) {
        // ---- converters: FP32 staging -> centred hi/lo operands
        const int ct = tid - 128;
        const float mu = a.mean_sum ? (float)(a.mean_sum[0] * a.inv_n) : 0.f;
        const int off = a.halo_x - R;
        const uint32_t lbo_a = (uint32_t)a.rows_p * 16;
        constexpr int VPC = 16 / EB;        // values per 16-byte chunk
        constexpr int CPI = 8 / VPC;        // chunks per item of 8 values
        constexpr int ITEMS = kTcK / 8;     // items of 8 values per row
        int i = 0;
        for (int tile = first; tile < a.ntiles; tile += step, ++i) {
            const int s = i & 1, k = i >> 1;
            const int sa = i % F::NSA, ka = i / F::NSA;
            bool ok = wait_or_abort(&ctl->stage_full[s], k & 1, ctl, a);
            ok = ok && wait_or_abort(&ctl->a_empty[sa], (ka & 1) ^ 1, ctl, a);
            if (!__all_sync(0xffffffffu, ok)) break;
            const float *st = reinterpret_cast<const float *>(smem + L.off_stage + s * L.stage_bytes);
            unsigned char *ahi = smem + L.off_a + (2 * sa) * L.a_bytes;
            unsigned char *alo = ahi + L.a_bytes;
            for (int it = ct; it < a.rows * ITEMS; it += 128) {
                const int kc8 = it % ITEMS, r = it / ITEMS;
                float v[8];
                load8(st + r * a.box_w + kc8 * 8 + off, off, mu, v);
                if constexpr (EB == 2) {
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
                    const uint32_t o = kc8 * lbo_a + r * 16;
                    *reinterpret_cast<uint4 *>(ahi + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4 *>(alo + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                } else {
                    uint32_t hw[8], lw[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        hw[e] = to_tf32(v[e]);
                        lw[e] = to_tf32(v[e] - __uint_as_float(hw[e]));
                    }
#pragma unroll
                    for (int c = 0; c < CPI; ++c) {
                        const uint32_t o = (kc8 * CPI + c) * lbo_a + r * 16;
                        *reinterpret_cast<uint4 *>(ahi + o) =
                            make_uint4(hw[4 * c], hw[4 * c + 1], hw[4 * c + 2], hw[4 * c + 3]);
                        *reinterpret_cast<uint4 *>(alo + o) =
                            make_uint4(lw[4 * c], lw[4 * c + 1], lw[4 * c + 2], lw[4 * c + 3]);
                    }
                }
            }
            fence_proxy_async_smem();
            mbar_arrive(&ctl->stage_empty[s]);
            mbar_arrive(&ctl->a_full[sa]);
        }
    } else if (warp >= 8) {
        // ---- epilogue: tensor memory -> registers -> global memory
        const int q = warp - 8;
        const float mu = a.mean_sum ? (float)(a.mean_sum[0] * a.inv_n) : 0.f;
        const float musum = mu * a.sum_c;
        int i = 0;
        for (int tile = first; tile < a.ntiles; tile += step, ++i) {
            const int s = i & 1, k = i >> 1;
            bool ok = wait_or_abort(&ctl->d_full[s], k & 1, ctl, a);
            ok = __all_sync(0xffffffffu, ok);
            // the four epilogue warps decide together, so that none of them is
            // left waiting at a named barrier the others never reach
            if (lane == 0) ctl->epi_ok[s][q] = ok ? 1 : 0;
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
            const int per_plane = a.tiles_x * a.tiles_y;
            const int pl = tile / per_plane, t2 = tile % per_plane;
            const int tx = t2 % a.tiles_x, ty = t2 / a.tiles_x;
            const int Y = ty * kTcM + 32 * q + lane;
            const int X0 = tx * kTcN;
            float o[32];
#pragma unroll
            for (int n = 0; n < 32; ++n) o[n] = v0[n] + (a.terms == 3 ? v1[n] : 0.f) + musum;
            float *const dplane = a.dst + (int64_t)pl * a.dst_pz;
            if (a.accumulate && Y < a.ny) {
                // add the partial result of the other plane offsets (stacked
                // grids take direct stores, never the TMA store)
                const float *row = dplane + Y * a.dst_py + X0;
                if (a.dst_vec4 && X0 + 32 <= a.nx) {
#pragma unroll
                    for (int n = 0; n < 32; n += 4) {
                        const float4 t = *reinterpret_cast<const float4 *>(row + n);
                        o[n] += t.x;
                        o[n + 1] += t.y;
                        o[n + 2] += t.z;
                        o[n + 3] += t.w;
                    }
                } else {
#pragma unroll
                    for (int n = 0; n < 32; ++n)
                        if (X0 + n < a.nx) o[n] += row[n];
                }
            }
            // Only tiles wholly inside the grid leave by TMA store.  A store box
            // clipped by the grid edge in x and y at once (a 97 x 203 grid)
            // gave wrong values beside the clipped tile, so ragged tiles take
            // the direct stores.  The decision is the same for the four
            // epilogue warps, which all reach the barriers of the store path.
            const bool via_tma = a.tma_store && a.nplanes == 1 && !a.accumulate &&
                                 X0 + kTcN <= a.nx && (ty + 1) * kTcM <= a.ny;
            if (via_tma) {
                // row 32q+lane of the swizzled tile: 16-byte chunk j lands at j ^ (row & 7)
                const int row = 32 * q + lane;
                unsigned char *tile_s = smem + L.off_out;
                if (tid == 256) bulk_wait_read();  // previous tile's store has read the buffer
                epi_barrier();
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    *reinterpret_cast<float4 *>(tile_s + row * 128 + ((j ^ (row & 7)) * 16)) =
                        make_float4(o[4 * j], o[4 * j + 1], o[4 * j + 2], o[4 * j + 3]);
                fence_proxy_async_smem();
                epi_barrier();
                if (tid == 256) tma_store_2d(&dmap, tile_s, X0, ty * kTcM);
            }
            if (Y < a.ny) {
                float *row = dplane + Y * a.dst_py + X0;
                if (via_tma) {
                    // the bulk store wrote the interior; only ghost copies remain
                } else if (a.dst_vec4 && X0 + 32 <= a.nx) {
#pragma unroll
                    for (int n = 0; n < 32; n += 4)
                        *reinterpret_cast<float4 *>(row + n) =
                            make_float4(o[n], o[n + 1], o[n + 2], o[n + 3]);
                } else {
#pragma unroll
                    for (int n = 0; n < 32; ++n)
                        if (X0 + n < a.nx) row[n] = o[n];
                }
                if (a.dst_gw > 0 && a.nplanes == 1 && (X0 < a.dst_gw || X0 + 32 > a.nx - a.dst_gw ||
                                     Y < a.dst_gw || Y >= a.ny - a.dst_gw)) {
#pragma unroll
                    for (int n = 0; n < 32; ++n)
                        if (X0 + n < a.nx) store_point_tc(a, X0 + n, Y, o[n]);
                }
            }
        }
    }

    __syncwarp();  // every warp reconverges after its role before the block barrier
    if (a.tma_store && tid == 256) bulk_wait_all();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

// Host-side rounding of a double to the nearest TF32 (ties away from zero,
// as the converters' cvt.rna does): keep 10 mantissa bits of the float.
float tf32_round(double v)
{
    const float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

}  // namespace

bool tc2d_supported(int R) { return R >= 1 && R <= kTcMaxR; }
bool tc2d_tf32_supported(int R) { return R >= 1 && R <= kTcMaxRTf32; }

static void tc_geometry(int R, int *rows, int *rows_p, int *box_w, int *halo_x)
{
    *halo_x = round_up(R, 4);
    *rows = kTcM + 2 * R;
    *rows_p = *rows | 1;  // odd: consecutive K chunks fall in different bank groups
    *box_w = round_up(kTcK + *halo_x - R, 4);
}

size_t tc2d_smem_bytes(int R, bool tma_store, bool tf32)
{
    int rows, rows_p, box_w, hx;
    tc_geometry(R, &rows, &rows_p, &box_w, &hx);
    return tf32 ? tc_layout<4>(R, rows, rows_p, box_w, tma_store ? 1 : 0).total
                : tc_layout<2>(R, rows, rows_p, box_w, tma_store ? 1 : 0).total;
}

size_t tc2d_panel_bytes(int R, bool tf32)
{
    return (size_t)(2 * R + 1) * (tf32 ? Fmt<4>::PANEL_BYTES : Fmt<2>::PANEL_BYTES);
}

// The hi/lo split of the folded weights with the mass correction: the centre
// tap's lo absorbs the rounding of the sum.  rnd rounds a double to the
// operand format and back.
template <class Rnd>
static double split_weights(const double *cm, int R, Rnd rnd, std::vector<double> &hi,
                            std::vector<double> &lo)
{
    const int W = 2 * R + 1;
    hi.assign(W * W, 0.0);
    lo.assign(W * W, 0.0);
    double target = 0.0, got = 0.0;
    for (int i = 0; i < W * W; ++i) {
        hi[i] = rnd(cm[i]);
        lo[i] = rnd(cm[i] - hi[i]);
        target += cm[i];
        got += hi[i] + lo[i];
    }
    const int c = R * W + R;
    lo[c] = rnd(lo[c] + (target - got));
    return target;
}

double tc2d_build_panels(const double *cm, int R, void *host_out, bool tf32)
{
    const int W = 2 * R + 1;
    std::vector<double> hi, lo;
    double target;
    if (tf32)
        target = split_weights(cm, R, [](double v) { return (double)tf32_round(v); }, hi, lo);
    else
        target = split_weights(
            cm, R, [](double v) { return (double)__bfloat162float(__double2bfloat16(v)); }, hi, lo);
    for (int ai = 0; ai < W; ++ai) {
        for (int n = 0; n < 64; ++n) {
            const int nn = n & 31;
            const std::vector<double> &src = n < 32 ? hi : lo;
            for (int k = 0; k < kTcK; ++k) {
                const int b = k - nn - R;  // column offset
                double w = 0.0;
                if (b >= -R && b <= R) w = src[ai * W + (b + R)];
                // K-major core-matrix layout: 16-byte chunk (k / per-chunk) of row n
                if (tf32) {
                    uint32_t *panel = static_cast<uint32_t *>(host_out) +
                                      (size_t)ai * (Fmt<4>::PANEL_BYTES / 4);
                    const float f = tf32_round(w);
                    uint32_t u;
                    memcpy(&u, &f, 4);
                    panel[((k / 4) * 64 + n) * 4 + (k % 4)] = u;
                } else {
                    uint16_t *panel = static_cast<uint16_t *>(host_out) +
                                      (size_t)ai * (Fmt<2>::PANEL_BYTES / 2);
                    panel[((k / 8) * 64 + n) * 8 + (k % 8)] =
                        __bfloat16_as_ushort(__double2bfloat16(w));
                }
            }
        }
    }
    // The epilogue adds mu * (sum of the exact folded weights): the mean the
    // exact stencil carries forward.  The split weights then act only on the
    // centred values x - mu, whose mean stays near zero, so their residual
    // mass error does not make the grid mean drift sweep after sweep.
    return target;
}

cudaError_t launch_tc2d(const CUtensorMap &map, const CUtensorMap &dmap, const TC2DArgs &a,
                        int grid, size_t smem, cudaStream_t s, bool tf32)
{
    if (tf32) {
        const cudaError_t e = smem_optin((const void *)k_tc2d<4>);
        if (e != cudaSuccess) return e;
        k_tc2d<4><<<grid, NT, smem, s>>>(map, dmap, a);
    } else {
        const cudaError_t e = smem_optin((const void *)k_tc2d<2>);
        if (e != cudaSuccess) return e;
        k_tc2d<2><<<grid, NT, smem, s>>>(map, dmap, a);
    }
    return cudaGetLastError();
}

}  // namespace sg
