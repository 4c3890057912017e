// Pieces shared by the 3D sweep kernels: the tap pattern of a folded star or
// box, the periodic copies of an output across the ghost band, the batched
// ghost refresh of a CTA's output block, and a vote over the consumer warps.
#pragma once

#include <climits>

#include "device_common.cuh"
#include "internal.h"

namespace sg {
namespace sweep3d {

// Output tile of a 3D CTA (columns x rows), planes per TMA chunk, stages.
constexpr int TX3 = 64, TY3 = 16, ZC = 4, NST = 3;

__host__ __device__ constexpr int cabs_div3(int v, int d) { return ((v < 0 ? -v : v) + d - 1) / d; }

template <int RB, int M, int PAT>
struct Taps3 {
    static constexpr int R = RB * M;
    static constexpr int W = 2 * R + 1;
    static constexpr int RP = (R + 3) / 4 * 4;
    __host__ __device__ static constexpr bool nz(int a, int b, int c)
    {
        return PAT == PAT_BOX ? true : (cabs_div3(a, RB) + cabs_div3(b, RB) + cabs_div3(c, RB) <= M);
    }
};

// Where a sweep's outputs go: the origin (interior point 0) of a grid, its
// row and plane pitches and the ghost band to refresh (0 = none).
struct Dst3 {
    float *p;
    int64_t py, pz;
    int gw;
};

__device__ __forceinline__ Dst3 dst_of(const Sweep3DArgs &a) { return {a.dst, a.dst_py, a.dst_pz, a.dst_gw}; }

// Copies of output (X, Y, Z) across every edge of the ghost band it lies
// within (up to seven: faces, edges and corners of the periodic box).
__device__ __forceinline__ void mirror3(const Sweep3DArgs &a, const Dst3 &d, int X, int Y, int Z,
                                        float v)
{
    const int gw = d.gw;
    // per axis: the cell itself, its copy past the high edge, past the low edge
    const int xs[3] = {X, X < gw ? X + a.nx : INT_MIN, X >= a.nx - gw ? X - a.nx : INT_MIN};
    const int ys[3] = {Y, Y < gw ? Y + a.ny : INT_MIN, Y >= a.ny - gw ? Y - a.ny : INT_MIN};
    const int zs[3] = {Z, Z < gw ? Z + a.nz : INT_MIN, Z >= a.nz - gw ? Z - a.nz : INT_MIN};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if ((i | j | k) && zs[i] != INT_MIN && ys[j] != INT_MIN && xs[k] != INT_MIN)
                    d.p[zs[i] * d.pz + ys[j] * d.py + xs[k]] = v;
}

// Ghost band of a padded destination, for the CTA's block of outputs
// (columns x0.., rows y0.., planes z0..z1): after a barrier over the consumer
// threads, the outputs within gw cells of an edge are read back (the CTA's own
// stores) and mirrored, one thread per cell.  The cells are the x/y band of
// every plane, then every cell of the planes in the z band; all planes are
// handled at once, each thread loading four cells before it stores.  Only
// CTAs that touch the band have work; a cell in two bands is handled twice,
// writing the same values.
template <int NC>
__device__ __forceinline__ void refresh_ghosts3(const Sweep3DArgs &a, const Dst3 &d, int x0,
                                                int y0, int z0, int z1, int tid)
{
    const int gw = d.gw, nx = a.nx, ny = a.ny, nz = a.nz;
    const int vx = min(TX3, nx - x0), vy = min(TY3, ny - y0);
    const int nt = y0 < gw ? min(y0 + vy, gw) - y0 : 0;  // band rows and columns of the tile
    const int yb0 = max(y0, ny - gw), nb = y0 + vy > yb0 ? y0 + vy - yb0 : 0;
    const int nl = x0 < gw ? min(x0 + vx, gw) - x0 : 0;
    const int xr0 = max(x0, nx - gw), nr = x0 + vx > xr0 ? x0 + vx - xr0 : 0;
    const int n_rows = (nt + nb) * vx, n_xy = n_rows + vy * (nl + nr);
    const int zl = max(0, min(z1, gw) - z0);           // planes z0 .. z0+zl-1 in the low z band
    const int zh0 = max(z0, nz - gw), zh = max(0, z1 - zh0);
    const int total1 = (z1 - z0) * n_xy, total = total1 + (zl + zh) * vx * vy;
    constexpr int U = 4;
    for (int base = tid; base < total; base += U * NC) {
        float v[U];
        int X[U], Y[U], Z[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int it = base + u * NC;
            if (it >= total) continue;
            if (it < total1) {
                const int c = it % n_xy;
                Z[u] = z0 + it / n_xy;
                if (c < nt * vx) {
                    Y[u] = y0 + c / vx;
                    X[u] = x0 + c % vx;
                } else if (c < n_rows) {
                    Y[u] = yb0 + (c - nt * vx) / vx;
                    X[u] = x0 + (c - nt * vx) % vx;
                } else if (c < n_rows + vy * nl) {
                    Y[u] = y0 + (c - n_rows) / nl;
                    X[u] = x0 + (c - n_rows) % nl;
                } else {
                    Y[u] = y0 + (c - n_rows - vy * nl) / nr;
                    X[u] = xr0 + (c - n_rows - vy * nl) % nr;
                }
            } else {
                const int j = it - total1, pl = j / (vx * vy), c = j % (vx * vy);
                Z[u] = pl < zl ? z0 + pl : zh0 + (pl - zl);
                Y[u] = y0 + c / vx;
                X[u] = x0 + c % vx;
            }
            v[u] = d.p[Z[u] * d.pz + Y[u] * d.py + X[u]];
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (base + u * NC < total) mirror3(a, d, X[u], Y[u], Z[u], v[u]);
    }
}

// Adds one staged input plane into a thread's register window of W output
// planes (4 columns each): with the weights of plane offset R - i, into the
// partial sums of output plane i of the window.  `pl` points at the thread's
// strip in the plane's first staged row, RP columns before its first output
// column; rows are SP floats apart and the thread's row is yr.
template <int RB, int M, int PAT>
__device__ __forceinline__ void add_plane3(float (&acc)[Taps3<RB, M, PAT>::W][4], const float *pl,
                                           int yr, int SP, const Sweep3DArgs &a)
{
    using TP = Taps3<RB, M, PAT>;
    constexpr int R = TP::R, W = TP::W, RP = TP::RP;
    constexpr int NSEG = 4 + 2 * RP;
#pragma unroll
    for (int dy = -R; dy <= R; ++dy) {
        float seg[NSEG];
        const float4 *rp = reinterpret_cast<const float4 *>(pl + (yr + R + dy) * SP);
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
                    const float w = a.c[((az + R) * W + (dy + R)) * W + (dx + R)];
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[i][v] = fmaf(w, seg[v + dx + RP], acc[i][v]);
                }
            }
        }
    }
}

// Stores the window's completed plane (acc[0]: 4 columns from X of row Y)
// when `store`, then shifts the window by one plane.
template <int W>
__device__ __forceinline__ void emit_plane3(float (&acc)[W][4], const Dst3 &d, int X, int Y,
                                            int zo, int nx, bool store, bool vec4)
{
    if (store) {
        float *row = d.p + zo * d.pz + Y * d.py;
        if (vec4) {
            *reinterpret_cast<float4 *>(row + X) = make_float4(acc[0][0], acc[0][1], acc[0][2], acc[0][3]);
        } else {
#pragma unroll
            for (int v = 0; v < 4; ++v)
                if (X + v < nx) row[X + v] = acc[0][v];
        }
    }
#pragma unroll
    for (int i = 0; i < W - 1; ++i)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[i][v] = acc[i + 1][v];
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[W - 1][v] = 0.f;
}

// OR of a predicate over the consumer threads (named barrier 1); also orders
// their memory accesses like a barrier.
template <int NC>
__device__ __forceinline__ bool consumers_any3(bool v)
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

// Barrier over the first NC threads (the consumer warps) on named barrier 1.
template <int NC>
struct NamedBarrier {
    __device__ static void sync() { asm volatile("bar.sync 1, %0;" ::"n"(NC) : "memory"); }
};

}  // namespace sweep3d
}  // namespace sg
