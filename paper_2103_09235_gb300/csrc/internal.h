// Host-side declarations shared by the library's translation units: device
// grid layouts, kernel argument blocks and launcher entry points.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace sg {

__host__ __device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int round_up(int a, int b) { return ceil_div(a, b) * b; }

// Ghost width allocated on every side of a padded 2D/3D grid.  Sweeps read
// their halo from these ghost cells instead of wrapping indices, so every
// tile (interior or boundary) is one rectangular TMA box.
constexpr int kGhost = 16;

// Largest folded radius R = m*r of a CUDA-core 2D/3D sweep kernel.
constexpr int kMaxR2D = 8;
constexpr int kMaxTaps2D = (2 * kMaxR2D + 1) * (2 * kMaxR2D + 1);
constexpr int kMaxR3D = 4;
constexpr int kMaxTaps3D = (2 * kMaxR3D + 1) * (2 * kMaxR3D + 1) * (2 * kMaxR3D + 1);
constexpr int kMaxR1D = 16;

// Tap patterns a kernel is specialised for.  A star of base radius rb folded
// m times keeps tap (a, b[, c]) iff sum ceil(|offset_i| / rb) <= m; a box
// keeps every tap.
// Tap patterns of the 2D/3D kernels.  PAT_CP1 and PAT_CP2 are 2D sweeps in
// counterpart form (c^(m) = sum of 1 or 2 separable terms).
enum Pattern : int { PAT_STAR = 0, PAT_BOX = 1, PAT_CP1 = 2, PAT_CP2 = 3 };

// FP32 grid in device memory surrounded by kGhost ghost cells per side.
// Interior point (x, y, z) lives at origin[z*pz + y*py + x].
struct Padded {
    float *alloc = nullptr;
    float *origin = nullptr;
    int ndim = 0;
    int nx = 1, ny = 1, nz = 1;
    int64_t py = 0, pz = 0;
    int gx = 0, gy = 0, gz = 0;
    size_t elems = 0;
};

// Rounds FP64 weights to FP32 and then moves the rounding of their sum into
// the centre tap (out[centre] absorbs sum(c) - sum(out), rounded once more),
// so that the FP32 weights carry the exact stencil's mass to within one
// rounding of the centre tap: the mean of the grid then does not drift by
// T/m roundings of the weight sum.
void round_f32_mass(const double *c, size_t n, size_t centre, float *out);

// Raises a kernel's dynamic shared-memory limit to the current device's
// opt-in maximum, once per (kernel, device); the attribute is per device, so
// a library used on several GPUs sets it on each.
cudaError_t smem_optin(const void *kernel);

// ---- 2D CUDA-core sweep (plain, folded, temporally blocked) ---------------
constexpr int kTileX2D = 128;   // output columns per CTA tile
constexpr int kThreads2D = 256;

struct Sweep2DArgs {
    int nx, ny;
    int tiles_x, ntiles;
    int tile_y;        // output rows per CTA tile
    int b;             // folded sweeps fused in this pass
    int halo;          // H = b * R rows/columns of halo
    int halo_x;        // H rounded up to a multiple of 4 (16-byte TMA column alignment)
    int map_x0, map_y0;  // tensor-map coordinates of the interior origin
    int buf_floats;    // floats between consecutive shared-memory buffers
    int nstages;       // TMA stages in flight per CTA (2..6)
    float *dst;        // destination interior origin
    int64_t dst_py;    // destination row stride (elements)
    int dst_gw;        // ghost band of the destination to refresh (0 = dense output)
    int dst_vec4;      // destination rows allow 16-byte stores
    int *status;
    unsigned long long wait_ns;
    int fault_withhold_copy;  // test hook: never issue the first tile's copy
    float c[kMaxTaps2D];  // folded weights, (2R+1)^2, row-major (dy, dx)
};

bool sweep2d_supported(int rb, int m, int pattern);
// cp_bufs: counterpart buffers of a counterpart-pattern pass (its K), else 0.
size_t sweep2d_smem_bytes(int tile_y, int b, int R, int *buf_floats, int nstages = 2,
                          int cp_bufs = 0);
// threads: 0 = the instance's own block size; 256 = two half-size CTAs for
// instances that run 512.
int sweep2d_ctas_per_sm(int rb, int m, int pattern, size_t smem, int threads = 0);
// Threads per CTA a launch of the instance runs (threads as for the launch).
int sweep2d_block_threads(int rb, int m, int pattern, int threads = 0);
cudaError_t launch_sweep2d(int rb, int m, int pattern, const CUtensorMap &map,
                           const Sweep2DArgs &a, int grid, size_t smem, int threads,
                           cudaStream_t s);

// ---- batched persistent 2D sweep --------------------------------------------
// One pass of one grid of a batched run.
struct BatchPass {
    int variant;        // batched_variant_id(base radius, m, pattern)
    int b, H, HX;       // fused sweeps, halo, halo rounded up to 4
    int tiles_x, ntiles;
    int map;            // index of the source tensor map
    int coef, ncoef;    // weights in the coefficient pool
    int dep;            // pass whose completion this one waits for (-1: none)
    int nx, ny;
    int map_x0, map_y0;
    float *dst;
    int64_t dst_py;
    int dst_gw;
    int dst_vec4;
};
struct BatchItem {
    int pass;
    int tile;
};
struct BatchArgs {
    const BatchItem *items;
    int nitems;
    const BatchPass *passes;
    const CUtensorMap *maps;  // 64-byte aligned, in global memory
    const float *coefs;
    int *done;                // tiles completed per pass (zeroed before the launch)
    int *next;                // queue head (zeroed before the launch)
    int tile_y;
    int buf_floats;
    int nwork;                // work buffers: 2 if a pass fuses >= 3 sweeps, 1 for 2, else 0
    int nstage;               // TMA stages: 1 (refilled after a tile's first sweep) or 2
    int *status;
    unsigned long long wait_ns;
    int fault_withhold_dep;   // test hook: dependencies never count as met, so the
                              // producer's bounded wait runs out (no fault)
};
// Radius-1 bases: star m <= 4, box m <= 2; radius-2 bases: star m <= 2, box m = 1.
bool batched_variant_supported(int rb, int m, int pattern);
// The kernel's code for (base radius, fold, pattern).
int batched_variant_id(int rb, int m, int pattern);
// nstage TMA stages plus nwork (0..2) work buffers of buf_floats each.
size_t batched_smem_bytes(int buf_floats, int nwork, int nstage);
// threads of the batched CTA for a plan's cta_threads option (256: the
// half-size CTA, two per SM; else the 512-thread CTA, one per SM)
int batched_threads(int cta_threads);
int batched_ctas_per_sm(size_t smem, int threads);
cudaError_t launch_batched(const BatchArgs &a, int grid, size_t smem, int threads, cudaStream_t s);

// ---- 3D CUDA-core sweep (streaming along z) -------------------------------
struct Sweep3DArgs {
    int nx, ny, nz;
    int tiles_x, tiles_y, ntiles_xy, zchunks, ntiles;
    int tile_y, zchunk;
    int fault_withhold_copy;    // test hook: k_sweep3d never issues a CTA's first chunk
    int halo_x;                 // R rounded up to a multiple of 4
    int map_x0, map_y0, map_z0;
    int buf_floats;             // floats per shared-memory plane slot
    int nst;                    // single sweeps: TMA stages of the ring (2 or 3)
    float *dst;
    int64_t dst_py, dst_pz;
    int dst_gw;
    int dst_vec4;
    int *status;
    unsigned long long wait_ns;
    float c[kMaxTaps3D];
};
bool sweep3d_supported(int rb, int m, int pattern);
size_t sweep3d_smem_bytes(int tile_y, int R, int *buf_floats, int nst = 3);
cudaError_t launch_sweep3d(int rb, int m, int pattern, const CUtensorMap &map,
                           const Sweep3DArgs &a, int grid, size_t smem, cudaStream_t s);
int sweep3d_ctas_per_sm(int rb, int m, int pattern, size_t smem);
// Multi-pass persistent 3D sweep (k_sweep3d_q): npass single sweeps in one
// launch, items (pass, piece) handed to the resident CTAs round robin, each
// waiting (bounded) for its neighbour pieces to finish the previous pass.
// Pass t reads the grid of map_e (t even) or map_o (t odd) and writes dst[t & 1]
// (padded, pitches py/pz, ghost band gw) except the last pass, which writes
// the Sweep3DArgs destination.
constexpr int kDep3 = 5;  // neighbour tiles per axis and tile, -1 padded
struct Sweep3DQueue {
    int npass;
    int *done;         // per piece: passes finished (zero before the launch)
    const int *dep;    // neighbour tiles: x table (tiles_x x kDep3), then y, then z
    int dep_y, dep_z;  // offsets of the y and z tables in dep
    float *dst[2];     // destinations of even and odd passes (padded grid origins)
    int64_t py, pz;
    int gw;
    int fault_withhold_dep;  // test hook: dependencies never count as met
};
bool sweep3d_q_supported(int rb, int m, int pattern);
int sweep3d_q_ctas_per_sm(int rb, int m, int pattern, size_t smem);
cudaError_t launch_sweep3d_q(int rb, int m, int pattern, const CUtensorMap &map_e,
                             const CUtensorMap &map_o, const Sweep3DArgs &a,
                             const Sweep3DQueue &q, int grid, size_t smem, cudaStream_t s);
// Two fused 3D sweeps per launch (temporal blocking, b = 2): folded radius <= 2.
// The staged boxes carry sweep3d_tb_halo_x() columns and 2R rows/planes of
// halo per side; a.halo_x must be set to sweep3d_tb_halo_x().
bool sweep3d_tb_supported(int rb, int m, int pattern);
size_t sweep3d_tb_smem_bytes(int R, int *buf_floats);
int sweep3d_tb_halo_x();
cudaError_t launch_sweep3d_tb(int rb, int m, int pattern, const CUtensorMap &map,
                              const Sweep3DArgs &a, int grid, size_t smem, cudaStream_t s);

// ---- 1D sweep (FP32/FP64, temporally blocked in shared memory) ------------
struct Sweep1DArgs {
    const void *src;
    void *dst;
    long long n;
    int tile;       // outputs per CTA
    int b;          // steps fused per launch
    double c[2 * kMaxR1D + 1];
};
bool sweep1d_supported(int R, bool f64);
cudaError_t launch_sweep1d(int R, bool f64, const Sweep1DArgs &a, cudaStream_t s);

// ---- FP64 2D/3D sweeps (k_sweep_f64.cu) -----------------------------------
constexpr int kMaxRF64_2D = 8;  // folded radius limits of the FP64 sweep
constexpr int kMaxRF64_3D = 4;
struct SweepF64Args {
    const double *src;
    double *dst;
    long long nx, ny, nz;
    int64_t src_py, src_pz, dst_py, dst_pz;  // row and plane strides (elements)
    int ndim, R;
    int tz;              // output planes per CTA (3D)
    int bx, by;          // CTAs along x and y
    int ntaps_dense;     // (2R+1)^ndim
    int nnz;             // nonzero weights
    double c[kMaxTaps3D];  // weights, dense, axis order (z, y, x)
};
size_t sweep_f64_smem_bytes(int ndim, int R, int tz, int nnz);
cudaError_t launch_sweep_f64(const SweepF64Args &a, cudaStream_t s);
int sweep_f64_block_x();
int sweep_f64_block_y();

// ---- 1D exact tessellate tiling (k_tess1d.cu, tess1d.h) --------------------
struct Tess1DArgs {
    const void *src;
    void *dst;
    void *par0, *par1;  // the two Jacobi arrays (n points each): edge values between stages
    long long n;
    int W;              // tile width; the last tile also takes n mod W
    int ntiles;         // max(1, n / W)
    int wmax;           // widest tile
    int b;              // steps per pass
    double c[2 * kMaxR1D + 1];
};
// Whether b steps of radius R tessellate n points in tiles of W.
bool tess1d_fits(long long n, int W, int b, int R);
// Both stages of one pass (two launches); radii as sweep1d_supported.
cudaError_t launch_tess1d(int R, bool f64, const Tess1DArgs &a, cudaStream_t s);

// ---- layout conversion, coefficient folding, error reduction --------------
// src: the user's grid, rows src_py and planes src_pz elements apart (0 =
// dense: nx and nx*ny).
// mean_sum: when given, the grid is stored centred: every value minus
// mu = (float)(mean_sum[0] * inv_n).
cudaError_t launch_import(const Padded &P, const float *src, int gw, cudaStream_t s,
                          int64_t src_py = 0, int64_t src_pz = 0,
                          const double *mean_sum = nullptr, double inv_n = 0.0);
// One 2D grid's import within a batch: padded rows [row0, row0 + ny + 2 gw)
// of the batch's row space.
struct ImportJob {
    float *origin;
    int64_t py;
    const float *src;
    int64_t src_py;  // row stride of the user's grid (elements)
    long long row0;
    int nx, ny, gw, vec4;
    // centred storage (k_center.cu): the grid's FP64 sum (null: not centred),
    // 1 / points, and the output the final bias mu * factor is added to
    double *mean_sum;
    double inv_n;
    float *out;
    int64_t out_py;
    double factor;
};
ImportJob make_import_job(const Padded &P, const float *src, int gw, long long row0,
                          int64_t src_py = 0);
// All jobs (device array, ordered by row0) in one launch; rows = the total.
cudaError_t launch_import_batch(const ImportJob *d_jobs, int njobs, long long rows, cudaStream_t s);
cudaError_t launch_export(const Padded &P, float *dst, cudaStream_t s);
// Centred storage (k_center.cu).  acc[0] += the FP64 sum of a caller-layout grid.
cudaError_t launch_grid_sum(const float *src, int nx, int ny, int nz, int64_t py, int64_t pz,
                            double *acc, cudaStream_t s);
// dst += (float)(mu * factor), mu = (float)(mean_sum[0] * inv_n), over a caller-layout grid.
cudaError_t launch_add_bias(float *dst, int nx, int ny, int nz, int64_t py, int64_t pz,
                            const double *mean_sum, double inv_n, double factor, cudaStream_t s);
// The same two steps for every job of a batch (rows as for launch_import_batch).
cudaError_t launch_grid_sum_batch(const ImportJob *d_jobs, int njobs, long long rows,
                                  cudaStream_t s);
cudaError_t launch_add_bias_batch(const ImportJob *d_jobs, int njobs, long long rows,
                                  cudaStream_t s);
// c^(m) by m-1 convolutions with c (FP64 on the GPU); work holds 2*(2mr+1)^ndim doubles.
cudaError_t launch_fold_power(int ndim, int r, int m, const double *d_c, double *d_out,
                              double *d_work, cudaStream_t s);
// Accumulates sum (y-r)^2, sum r^2, sum y, sum r into acc[4] (zeroed by the caller).
cudaError_t launch_rel_l2(const void *y, bool y_f64, const double *ref, long long n,
                          double *acc, cudaStream_t s);

// ---- tcgen05 folded 2D box sweep (BF16 hi/lo split) -----------------------
// A tile is 128 grid rows x 32 output columns.  The contraction dimension K
// is the 48-column window x0-R .. x0+32+R of the tile, padded with zero
// weights; R = m*r <= 8 keeps 32 + 2R <= 48.
constexpr int kTcM = 128;
constexpr int kTcN = 32;
constexpr int kTcK = 48;
constexpr int kTcKC = kTcK / 8;                 // 16-byte K chunks
constexpr int kTcMaxR = 8;
constexpr int kTcMaxRTf32 = 4;                  // TF32 panels take twice the bytes
constexpr int kTcPanelElems = 64 * kTcK;        // one row offset: C_hi (32 rows) over C_lo (32 rows)
constexpr int kTcGroup = 4;                     // grouped form: row offsets per MMA
constexpr int kTcOutRows = kTcM - (kTcGroup - 1);  // grouped form: output rows per tile
constexpr int kTcGroupedMinR = 6;               // folded radius from which the grouped form is used
constexpr int kTcThreads = 384;

struct TC2DArgs {
    int nx, ny;
    int tiles_x, ntiles;
    int R;                  // folded radius
    int halo_x;             // R rounded up to a multiple of 4
    int box_w;              // staging box width (floats)
    int rows;               // 128 + 2R staged rows
    int rows_p;             // A-operand rows per K chunk in shared memory (odd)
    int nstage;             // grouped form: FP32 staging slots (1 or 2)
    int terms;              // 3: hi*hi + hi*lo + lo*hi, 1: hi*hi
    int map_x0, map_y0;     // tensor-map coordinates of the interior origin
    const double *mean_sum; // grid sum; mu = mean_sum[0] * inv_n (null: mu = 0)
    double inv_n;
    float sum_c;            // FP64 sum of the folded weights (rounded to FP32)
    const uint16_t *panels; // (2R+1) panels, tc2d panel layout
    float *dst;
    int64_t dst_py;
    int dst_gw;
    int dst_vec4;
    int tma_store;          // 1: the output tile leaves through a swizzled smem tile and a TMA store
    int fault_withhold_mma; // test hook: the MMA issuer stops before its first MMA (no fault;
                            // the other roles' bounded waits run out)
    int *status;
    unsigned long long wait_ns;
    // Per-offset kernel only: a stack of nplanes 2D grids (the planes of a 3D
    // grid seen as one tall 2D array whose planes start src_plane_rows rows
    // apart), each tile reading the plane dz away from the one it writes;
    // outputs land dst_pz floats apart per plane and, with accumulate, are
    // added to what the destination holds.  2D: nplanes = 1, the rest 0.
    int tiles_y;            // tiles per plane in y
    int nplanes;
    int64_t src_plane_rows;
    int dz;
    int64_t dst_pz;
    int accumulate;
};
bool tc2d_supported(int R);
bool tc2d_tf32_supported(int R);
// tf32: TF32 hi/lo operands (kind::tf32) instead of BF16 hi/lo (kind::f16).
size_t tc2d_smem_bytes(int R, bool tma_store, bool tf32 = false);
size_t tc2d_panel_bytes(int R, bool tf32);
// Grouped form (k_tc2d_grouped.cu): four row offsets per MMA, 125 output rows
// of 32 columns per tile, direct stores.
size_t tc2dg_smem_bytes(int R, int nstage);
// Tile geometry of the grouped kernel: staged rows, A-operand row pitch (rows),
// FP32 staging row pitch (floats; also the TMA box width) and halo columns.
void tc2dg_geometry(int R, int *rows, int *rows_p, int *box_w, int *halo_x);
size_t tc2dg_panel_elems(int R);
double tc2dg_build_panels(const double *cm, int R, uint16_t *host_out);
cudaError_t launch_tc2dg(const CUtensorMap &map, const TC2DArgs &a, int grid, size_t smem,
                         cudaStream_t s);
// Builds the (2R+1) Toeplitz panels (BF16, or TF32 with tf32) of folded
// weights cm ((2R+1)^2, row-major (dy, dx)) with the hi/lo split and the mass
// correction into host_out (tc2d_panel_bytes bytes); returns the FP64 sum of
// cm, which the epilogue multiplies by mu.
double tc2d_build_panels(const double *cm, int R, void *host_out, bool tf32);
cudaError_t launch_tc2d(const CUtensorMap &map, const CUtensorMap &dmap, const TC2DArgs &a,
                        int grid, size_t smem, cudaStream_t s, bool tf32);
cudaError_t launch_grid_mean(const float *origin, int nx, int ny, int64_t py, double *acc,
                             cudaStream_t s);


// ---- tensor maps ------------------------------------------------------------
// Encodes a tiled FP32 tensor map over a padded grid's whole allocation.
// box has P.ndim entries (x first).  Returns false if the encoder refuses it.
bool encode_padded_map(CUtensorMap *map, const Padded &P, const int *box);
// Encodes a 2D FP32 store map over exactly nx x ny elements at base (row
// stride pitch elements) with 128-byte swizzle; false if unaligned or refused.
bool encode_store_map_2d(CUtensorMap *map, float *base, int nx, int ny, int64_t pitch, int box_x,
                         int box_y);

}  // namespace sg
