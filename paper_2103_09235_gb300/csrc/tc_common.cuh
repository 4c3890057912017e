// tcgen05 and control helpers shared by the two tensor-core sweep kernels
// (k_tc2d.cu: one MMA per row offset; k_tc2d_grouped.cu: four row offsets
// per MMA): operand and instruction descriptors, the MMA issue and commit,
// tensor-memory loads and fences, the bounded role waits, and the periodic
// ghost copies of an output.
#pragma once

#include <cuda_bf16.h>

#include "device_common.cuh"
#include "internal.h"

namespace sg {
namespace tcore {

// Shared-memory matrix descriptor of a no-swizzle K-major operand.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    // start address, leading (K-chunk) and stride (8-row group) byte offsets,
    // all >> 4; bit 46 = descriptor version 1; swizzle mode 0 (none)
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

// One tcgen05.mma of kind::f16 into tensor-memory address d_tmem;
// accumulate = 0 overwrites the accumulator.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate)
{
    // no memory clobber: ordering with the operand writes comes from the
    // mbarrier waits and fences around the issue loop
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive accumulator columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// A bounded wait that also ends when another role has raised the control
// block's abort flag; running out raises it and records a timeout.
template <class Ctl>
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, Ctl *ctl,
                                              const TC2DArgs &a)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*(volatile int *)&ctl->abort) return false;
        if (globaltimer_ns() - t0 > a.wait_ns) {
            *(volatile int *)&ctl->abort = 1;
            record_status(a.status, DEV_TIMEOUT);
            return false;
        }
    }
}

// A final bounded wait used while winding down after an abort.
__device__ __forceinline__ void drain_wait(uint64_t *bar, uint32_t parity, const TC2DArgs &a)
{
    mbar_wait_bounded(bar, parity, a.wait_ns);
}

// Barrier over the four epilogue warps (named barrier 1).
__device__ __forceinline__ void epi_barrier() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// The periodic copies of output (X, Y) across the destination's ghost band.
__device__ __forceinline__ void store_point_tc(const TC2DArgs &a, int X, int Y, float v)
{
    float *dst = a.dst;
    const int64_t py = a.dst_py;
    const int nx = a.nx, ny = a.ny, gw = a.dst_gw;
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

}  // namespace tcore
}  // namespace sg
