// Per-tile body of the 2D CUDA-core sweep, shared by the single-grid kernel
// and the batched persistent kernel: the register-window strip sweep over a
// shared-memory tile (see k_sweep2d.cu) and the b-sweep temporal block.
#pragma once

#include <climits>

#include "device_common.cuh"
#include "internal.h"

namespace sg {
namespace tile2d {

// Where a tile's final sweep writes: a padded grid (with a ghost band to
// refresh) or a dense grid.
struct TileOut {
    float *dst;      // interior origin
    int64_t dst_py;  // row stride (elements)
    int nx, ny;
    int dst_gw;      // ghost band to refresh (0 = dense)
    int dst_vec4;    // rows allow 16-byte stores
};

// Weight accessors: from the kernel parameter block (constant bank) or from
// shared memory.
struct ParamCoef {
    const float *c;
    __device__ __forceinline__ float operator()(int k) const { return c[k]; }
};

// Barrier over the threads that run the tile body: the whole CTA, or the
// first N threads on named barrier 1 when the CTA has warps with other roles.
struct CtaSync {
    __device__ static int nthr() { return blockDim.x; }
    __device__ static void sync() { __syncthreads(); }
};
template <int N>
struct NamedSync {
    __device__ static constexpr int nthr() { return N; }
    __device__ static void sync() { asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory"); }
};

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
    // rows of the steady loop unrolled together.  Rolled (1), the window shift
    // costs register moves; a full turn (W) renames them away but multiplies
    // the code, and instruction-cache misses then cost more.  Measured on
    // GB300: the plain 9-point box runs faster unrolled (737 vs 672 GS/s at
    // 8192^2), every other instance rolled (plain star 778 vs 735, folded
    // sweeps 1-11 % faster).
    static constexpr int UNR = (PAT == PAT_BOX && R == 1) ? W : 1;

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
    template <class Coef>
    __device__ __forceinline__ static void slot(float (&acc)[W][4], const float (&seg)[NSEG],
                                                const Coef &cf, int i)
    {
        const int aa = R - i;
#pragma unroll
        for (int bb = -R; bb <= R; ++bb) {
            if (TP::nz(aa, bb)) {
                const float w = cf((aa + R) * W + (bb + R));
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

// Four outputs of row Y starting at column X of a row that ends at column nx
// or is not 16-byte aligned: only the columns inside the grid are stored.
// Out of line, with scalar arguments: only the last strip of a ragged tile
// (or an unaligned destination) comes here, and the caller's descriptor stays
// in registers.
static __device__ __noinline__ void store_masked4(float *dst, int64_t py, int nx, int vec4, int X,
                                                  int Y, float v0, float v1, float v2, float v3)
{
    float *row = dst + Y * py;
    if (vec4 && X + 3 < nx) {
        *reinterpret_cast<float4 *>(row + X) = make_float4(v0, v1, v2, v3);
        return;
    }
    if (X < nx) row[X] = v0;
    if (X + 1 < nx) row[X + 1] = v1;
    if (X + 2 < nx) row[X + 2] = v2;
    if (X + 3 < nx) row[X + 3] = v3;
}

// The thread-to-item split of one sweep of a full tile, the same for every
// full tile of a launch, so each CTA works it out once: nsx strips by G row
// groups over nr rows, with q / nsx = umulhi(q, mn) and q / G = umulhi(q, mg)
// (mn = ceil(2^32 / nsx), mg = ceil(2^32 / G); exact for q below 2^17 with
// divisors below 2^9, since q * (m * d - 2^32) < 2^32 then).
struct SweepGeom {
    int nsx_G;    // nsx | G << 16
    uint32_t mn, mg;
    int nr;
};

__host__ __device__ inline uint32_t div_magic(uint32_t d)
{
    return (uint32_t)((0x100000000ull + d - 1) / d);
}

// One sweep over output rows [r0, r1) and 4-column strips [k0, k1) of a
// shared-memory buffer S (row pitch SP).  FINAL writes to global memory;
// otherwise the outputs go to the same coordinates of buffer D.  gm, when
// given, is the precomputed split of this sweep (full tiles).
//
// A strip of rows [ya, yb) reads input rows ya-R .. yb+R-1.  The first 2R
// rows only feed window slots whose output row is >= ya and the last 2R only
// slots whose output row is < yb, so every output gets exactly its taps.
template <int RB, int M, int PAT, bool FINAL, class Sync, class Coef>
__device__ __forceinline__ void sweep_region(const float *__restrict__ S, float *__restrict__ D,
                                             int SP, int r0, int r1, int k0, int k1,
                                             const Coef &cf, const TileOut &a, int gx0, int gy0,
                                             const SweepGeom *gm = nullptr)
{
    using ST = Strip<RB, M, PAT>;
    constexpr int R = ST::R, W = ST::W, RP = ST::RP, NSEG = ST::NSEG;
    const int nsx = k1 - k0;
    const int nr = r1 - r0;
    if (nsx <= 0 || nr <= 0) return;
    // row groups: as many as the threads allow, each at least 2R rows tall
    const int nthr = Sync::nthr();  // the threads running the tile body (224 to 512)
    int G;
    uint32_t mn = 0, mg = 0;
    if (gm && gm->nsx_G == 0) gm = nullptr;  // a split without a usable reciprocal
    if (gm) {
        G = gm->nsx_G >> 16;
        mn = gm->mn;
        mg = gm->mg;
    } else {
        G = nthr / nsx;
        G = max(1, min(G, nr / (2 * R)));
    }
    const int items = nsx * G;

    for (int it = threadIdx.x; it < items; it += nthr) {
        int k, g, ya, yb;
        if (gm) {
            g = (int)__umulhi((uint32_t)it, mn);
            k = k0 + it - g * nsx;
            ya = r0 + (int)__umulhi((uint32_t)(g * nr), mg);
            yb = r0 + (int)__umulhi((uint32_t)((g + 1) * nr), mg);
        } else {
            k = k0 + it % nsx;
            g = it / nsx;
            ya = r0 + (g * nr) / G;
            yb = r0 + ((g + 1) * nr) / G;
        }
        const int cx = 4 * k;
        const float *col = S + cx - RP;

        float acc[W][4];
#pragma unroll
        for (int i = 0; i < W; ++i)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[i][v] = 0.f;

        // Output rows are emitted in order ya, ya+1, ...: a strip whose four
        // columns lie inside the grid (all but a ragged tile's last strip)
        // stores each row with one 16-byte store and a pointer step.
        float *orow = nullptr;
        bool fast = false;
        if constexpr (FINAL) {
            // rows [ya, yb) all lie inside the grid (the region is clipped to it)
            const int X = gx0 + cx, Y0 = gy0 + ya;
            fast = a.dst_vec4 && X + 3 < a.nx;
            orow = a.dst + (int64_t)Y0 * a.dst_py + X;
        } else {
            orow = D + ya * SP + cx;
        }
        auto emit = [&](int y) {
            if constexpr (FINAL) {
                if (fast)
                    *reinterpret_cast<float4 *>(orow) =
                        make_float4(acc[0][0], acc[0][1], acc[0][2], acc[0][3]);
                else
                    store_masked4(a.dst, a.dst_py, a.nx, a.dst_vec4, gx0 + cx, gy0 + y, acc[0][0],
                                  acc[0][1], acc[0][2], acc[0][3]);
                orow += a.dst_py;
            } else {
                (void)y;
                *reinterpret_cast<float4 *>(orow) =
                    make_float4(acc[0][0], acc[0][1], acc[0][2], acc[0][3]);
                orow += SP;
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
                    if (i >= 2 * R - u) ST::slot(acc, seg, cf, i);
                ST::shift(acc);
            }
            // steady rows: every slot, one finished output row each
            const int jm = yb - R;
#pragma unroll ST::UNR
            for (; j < jm; ++j) {
                float seg[NSEG];
                ST::load(col + j * SP, seg);
#pragma unroll
                for (int i = 0; i < W; ++i) ST::slot(acc, seg, cf, i);
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
                    if (i <= v) ST::slot(acc, seg, cf, i);
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
                for (int i = 0; i < W; ++i) ST::slot(acc, seg, cf, i);
                if (j - R >= ya) emit(j - R);
                ST::shift(acc);
            }
        }
    }
}

// Ghost band of a padded destination: every output within gw cells of an edge
// is repeated across that edge (across both at a corner), so that the next
// pass's TMA boxes read periodic neighbours without wrapping.  Run after the
// tile's final sweep by the tiles that touch the band: the outputs are read
// back from the destination after a barrier (the CTA's own stores) and copied
// with one thread per band cell.  A cell in a row band and a column band is
// handled twice, writing the same values.
template <class Sync>
__device__ __forceinline__ void refresh_ghosts(const TileOut &o, int x0, int y0, int vx, int vy)
{
    const int gw = o.dst_gw, nx = o.nx, ny = o.ny;
    if (gw <= 0) return;
    const int nt = y0 < gw ? min(y0 + vy, gw) - y0 : 0;                  // top band rows
    const int yb0 = max(y0, ny - gw), nb = y0 + vy > yb0 ? y0 + vy - yb0 : 0;
    const int nl = x0 < gw ? min(x0 + vx, gw) - x0 : 0;                  // left band columns
    const int xr0 = max(x0, nx - gw), nr = x0 + vx > xr0 ? x0 + vx - xr0 : 0;
    const int n_rows = (nt + nb) * vx, total = n_rows + vy * (nl + nr);
    if (total == 0) return;  // the same for every thread of the tile
    Sync::sync();
    float *d = o.dst;
    const int64_t py = o.dst_py;
    for (int it = threadIdx.x; it < total; it += Sync::nthr()) {
        int X, Y;
        if (it < nt * vx) {
            Y = y0 + it / vx;
            X = x0 + it % vx;
        } else if (it < n_rows) {
            const int j = it - nt * vx;
            Y = yb0 + j / vx;
            X = x0 + j % vx;
        } else if (it < n_rows + vy * nl) {
            const int j = it - n_rows;
            Y = y0 + j / nl;
            X = x0 + j % nl;
        } else {
            const int j = it - n_rows - vy * nl;
            Y = y0 + j / nr;
            X = xr0 + j % nr;
        }
        const float v = d[Y * py + X];
        const int xs[2] = {X < gw ? X + nx : INT_MIN, X >= nx - gw ? X - nx : INT_MIN};
        const int ys[2] = {Y < gw ? Y + ny : INT_MIN, Y >= ny - gw ? Y - ny : INT_MIN};
#pragma unroll
        for (int i = 0; i < 2; ++i)
            if (xs[i] != INT_MIN) d[Y * py + xs[i]] = v;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (ys[j] == INT_MIN) continue;
            d[ys[j] * py + X] = v;
#pragma unroll
            for (int i = 0; i < 2; ++i)
                if (xs[i] != INT_MIN) d[ys[j] * py + xs[i]] = v;
        }
    }
}

// ---- counterpart form (Section 3.3, Eq. vfold and Eq. horifold; Section 3.5)
// When the folded weights factor as c^(m) = sum_{k<K} u_k (x) v_k (u_k over
// row offsets, v_k over column offsets), a sweep is a vertical fold of the
// input with each u_k -- the counterparts V_k -- followed by a horizontal
// fold that combines the counterparts with the v_k:
//   V_k[y][x] = sum_a u_k[a] S[y+a][x],   out[y][x] = sum_k sum_b v_k[b] V_k[y][x+b],
// 2K(2R+1) multiply-adds per point instead of one per nonzero of c^(m).
// The weights sit in the parameter block as u_0 .. u_{K-1}, then v_0 .. v_{K-1}.

// Vertical fold of rows [r0, r1) and columns [x0, x1) (multiples of 4) of S
// into the counterpart buffers V + k*vstride (same coordinates as S): a
// register window of 2R+1 output rows per strip of CW columns, one
// counterpart at a time, with the same trimmed ramps as sweep_region.  A
// window needs runs of at least 2R rows, so wide folds (R >= 6) take
// 2-column strips to keep every thread busy on the same region.
template <int R, int K, class Sync, class Coef>
__device__ __forceinline__ void vfold_region(const float *__restrict__ S, float *__restrict__ V,
                                             int vstride, int SP, int r0, int r1, int x0, int x1,
                                             const Coef &cf)
{
    constexpr int W = 2 * R + 1;
    constexpr int CW = R >= 6 ? 2 : 4;
    const int k0 = x0 / CW, k1 = x1 / CW;
    const int nsx = k1 - k0, nr = r1 - r0;
    if (nsx <= 0 || nr <= 0) return;
    const int nthr = Sync::nthr();
    int G = nthr / nsx;
    G = max(1, min(G, nr / (2 * R)));
    const int items = nsx * G;
    for (int it = threadIdx.x; it < items; it += nthr) {
        const int k = k0 + it % nsx, g = it / nsx;
        const int ya = r0 + (g * nr) / G, yb = r0 + ((g + 1) * nr) / G;
        const float *col = S + CW * k;
#pragma unroll 1
        for (int q = 0; q < K; ++q) {
            float acc[W][CW];
#pragma unroll
            for (int i = 0; i < W; ++i)
#pragma unroll
                for (int v = 0; v < CW; ++v) acc[i][v] = 0.f;
            float *orow = V + q * vstride + ya * SP + CW * k;
            // input row j feeds slot i (output row j - R + i) with weight u_q[R - i]
            auto feed = [&](int j, int ilo, int ihi) {
                float x[CW];
                if constexpr (CW == 4) {
                    const float4 t = *reinterpret_cast<const float4 *>(col + j * SP);
                    x[0] = t.x;
                    x[1] = t.y;
                    x[2] = t.z;
                    x[3] = t.w;
                } else {
                    const float2 t = *reinterpret_cast<const float2 *>(col + j * SP);
                    x[0] = t.x;
                    x[1] = t.y;
                }
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    if (i < ilo || i > ihi) continue;
                    const float w = cf(q * W + (W - 1 - i));
#pragma unroll
                    for (int v = 0; v < CW; ++v) acc[i][v] = fmaf(w, x[v], acc[i][v]);
                }
            };
            auto emit_shift = [&](bool emit) {
                if (emit) {
                    if constexpr (CW == 4)
                        *reinterpret_cast<float4 *>(orow) =
                            make_float4(acc[0][0], acc[0][1], acc[0][2], acc[0][3]);
                    else
                        *reinterpret_cast<float2 *>(orow) = make_float2(acc[0][0], acc[0][1]);
                    orow += SP;
                }
#pragma unroll
                for (int i = 0; i < W - 1; ++i)
#pragma unroll
                    for (int v = 0; v < CW; ++v) acc[i][v] = acc[i + 1][v];
#pragma unroll
                for (int v = 0; v < CW; ++v) acc[W - 1][v] = 0.f;
            };
            int j = ya - R;
            if (yb - ya >= 2 * R) {
#pragma unroll
                for (int u = 0; u < 2 * R; ++u, ++j) {
                    feed(j, 2 * R - u, W - 1);
                    emit_shift(false);
                }
                const int jm = yb - R;
#pragma unroll 1
                for (; j < jm; ++j) {
                    feed(j, 0, W - 1);
                    emit_shift(true);
                }
#pragma unroll
                for (int v = 2 * R - 1; v >= 0; --v, ++j) {
                    feed(j, 0, v);
                    emit_shift(true);
                }
            } else {
#pragma unroll 1
                for (; j < yb + R; ++j) {
                    feed(j, 0, W - 1);
                    emit_shift(j - R >= ya);
                }
            }
        }
    }
}

// Horizontal fold of the counterparts into rows [r0, r1) and strips [k0, k1)
// of D (or, FINAL, of the global destination), one output row at a time.
template <int R, int K, bool FINAL, class Sync, class Coef>
__device__ __forceinline__ void hfold_region(const float *__restrict__ V, int vstride,
                                             float *__restrict__ D, int SP, int r0, int r1, int k0,
                                             int k1, const Coef &cf, const TileOut &a, int gx0,
                                             int gy0)
{
    constexpr int W = 2 * R + 1;
    constexpr int RP = (R + 3) / 4 * 4, NSEG = 4 + 2 * RP;
    const int nsx = k1 - k0, nr = r1 - r0;
    if (nsx <= 0 || nr <= 0) return;
    const int nthr = Sync::nthr();
    int G = nthr / nsx;
    G = max(1, min(G, nr));
    const int items = nsx * G;
    for (int it = threadIdx.x; it < items; it += nthr) {
        const int k = k0 + it % nsx, g = it / nsx;
        const int ya = r0 + (g * nr) / G, yb = r0 + ((g + 1) * nr) / G;
        const int cx = 4 * k;
        float *orow;
        bool fast = false;
        if constexpr (FINAL) {
            const int X = gx0 + cx;
            fast = a.dst_vec4 && X + 3 < a.nx;
            orow = a.dst + (int64_t)(gy0 + ya) * a.dst_py + X;
        } else {
            orow = D + ya * SP + cx;
        }
#pragma unroll 1
        for (int y = ya; y < yb; ++y) {
            float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < K; ++q) {
                float seg[NSEG];
                const float4 *rp = reinterpret_cast<const float4 *>(V + q * vstride + y * SP + cx - RP);
#pragma unroll
                for (int t = 0; t < NSEG / 4; ++t) {
                    const float4 x = rp[t];
                    seg[4 * t] = x.x;
                    seg[4 * t + 1] = x.y;
                    seg[4 * t + 2] = x.z;
                    seg[4 * t + 3] = x.w;
                }
#pragma unroll
                for (int bb = -R; bb <= R; ++bb) {
                    const float w = cf(K * W + q * W + bb + R);
#pragma unroll
                    for (int v = 0; v < 4; ++v) o[v] = fmaf(w, seg[v + bb + RP], o[v]);
                }
            }
            if constexpr (FINAL) {
                if (fast)
                    *reinterpret_cast<float4 *>(orow) = make_float4(o[0], o[1], o[2], o[3]);
                else
                    store_masked4(a.dst, a.dst_py, a.nx, a.dst_vec4, gx0 + cx, gy0 + y, o[0], o[1],
                                  o[2], o[3]);
                orow += a.dst_py;
            } else {
                *reinterpret_cast<float4 *>(orow) = make_float4(o[0], o[1], o[2], o[3]);
                orow += SP;
            }
        }
    }
}

// The item split of every sweep of a full tile (TX x TY outputs, halo H rows
// and HX columns, b sweeps of radius R) for blocks of nthr threads; sweep s
// goes to g[s].  Run by one thread per sweep (s = threadIdx.x < b).
template <int R>
__device__ __forceinline__ void full_tile_geom(SweepGeom *g, int s, int b, int TY, int H, int HX,
                                               int nthr)
{
    int nr, k0, k1;
    if (s < b - 1) {
        const int sh = (s + 1) * R;
        nr = 2 * H + TY - 2 * sh;
        k0 = (HX - H + sh) / 4;
        k1 = (HX + TX + H - sh + 3) / 4;
    } else {
        nr = TY;
        k0 = HX / 4;
        k1 = (HX + TX + 3) / 4;
    }
    const int nsx = k1 - k0;
    int G = nthr / nsx;
    G = max(1, min(G, nr / (2 * R)));
    // a divisor of 1 has no 32-bit reciprocal: such sweeps keep the divisions
    g[s].nsx_G = (nsx >= 2 && G >= 2) ? (nsx | (G << 16)) : 0;
    g[s].mn = div_magic((uint32_t)nsx);
    g[s].mg = div_magic((uint32_t)G);
    g[s].nr = nr;
}

// A callback that does nothing (see process_tile's stage_free).
struct NoHook {
    __device__ void operator()() const {}
};

// b fused sweeps of one staged tile: stage -> work buffers -> destination.
// The staged box covers rows [0, TY + 2H) and columns [0, TX + 2HX), with the
// output tile at rows [H, H + TY) and columns [HX, HX + TX).  Only the first
// vy rows and vx columns of the tile lie inside the grid (a ragged last tile):
// every sweep's region is clipped to what those outputs need.  When b >= 2
// only the first sweep reads the stage: stage_free() runs right after the
// barrier that ends it, so the caller can refill the stage during the others.
//
// Counterpart patterns (PAT_CP1, PAT_CP2: K = 1, 2) take the counterpart
// buffers at vbuf (K buffers, vstride floats apart); each sweep is a vertical
// fold into them and a horizontal fold out of them, so for any b the stage is
// free once the first vertical fold has read it.
template <int RB, int M, int PAT, class Sync = CtaSync, class Coef, class Hook = NoHook>
__device__ __forceinline__ void process_tile(const float *stage, float *work0, float *work1,
                                             int TY, int H, int HX, int b, const Coef &cf,
                                             const TileOut &o, int gx0, int gy0, int vx, int vy,
                                             const Hook &stage_free = Hook(),
                                             float *vbuf = nullptr, int vstride = 0,
                                             const SweepGeom *geom = nullptr)
{
    constexpr int R = RB * M;
    const int SP = TX + 2 * HX;
    (void)TY;
    const float *src = stage;
    if constexpr (PAT >= PAT_CP1) {
        constexpr int K = PAT - PAT_CP1 + 1;
        for (int s = 0; s < b; ++s) {
            // the region of sweep s: its rim shrinks by R per sweep down to the tile
            const int sh = (s + 1) * R;
            const int r0 = sh, r1 = 2 * H + vy - sh;
            const int c0 = HX - H + sh, c1 = HX + vx + H - sh;
            vfold_region<R, K, Sync>(src, vbuf, vstride, SP, r0, r1, (c0 - R) / 4 * 4,
                                     (c1 + R + 3) / 4 * 4, cf);
            Sync::sync();
            if (s == 0) stage_free();  // everything after this reads only the counterparts
            if (s == b - 1) {
                hfold_region<R, K, true, Sync>(vbuf, vstride, nullptr, SP, r0, r1, c0 / 4,
                                               (c1 + 3) / 4, cf, o, gx0, gy0);
            } else {
                float *dst = (s & 1) ? work1 : work0;
                hfold_region<R, K, false, Sync>(vbuf, vstride, dst, SP, r0, r1, c0 / 4,
                                                (c1 + 3) / 4, cf, o, gx0, gy0);
                Sync::sync();
                src = dst;
            }
        }
    } else {
        (void)vbuf;
        (void)vstride;
        // the precomputed item splits hold for full tiles only
        const SweepGeom *gm = (vx == TX && vy == TY) ? geom : nullptr;
        for (int s = 0; s < b - 1; ++s) {
            const int sh = (s + 1) * R;  // rim still needed: H - sh per side
            const int c0 = HX - H + sh, c1 = HX + vx + H - sh;
            float *dst = (s & 1) ? work1 : work0;
            sweep_region<RB, M, PAT, false, Sync>(src, dst, SP, sh, 2 * H + vy - sh, c0 / 4,
                                                  (c1 + 3) / 4, cf, o, gx0, gy0,
                                                  gm ? gm + s : nullptr);
            Sync::sync();
            if (s == 0) stage_free();
            src = dst;
        }
        sweep_region<RB, M, PAT, true, Sync>(src, nullptr, SP, H, H + vy, HX / 4,
                                             (HX + vx + 3) / 4, cf, o, gx0, gy0,
                                             gm ? gm + (b - 1) : nullptr);
    }
    refresh_ghosts<Sync>(o, gx0 + HX, gy0 + H, vx, vy);
}

}  // namespace tile2d
}  // namespace sg
