// Exact tessellate tiling of a 1D periodic line (Section 3.4, tessellate
// tiling): b steps of a radius-R stencil over tiles of width W, in two
// stages and with no point updated twice for the same time level.
//
//  - Stage 1 (triangles): every tile advances, at step s = 1..b, the points
//    whose distance to both of its edges is at least s*R -- the tile's
//    local indices [s*R, W - s*R).  Such a point only reads points of its
//    own tile that stage 1 brought to level s-1.
//  - Stage 2 (inverted triangles): around every tile boundary xb, at step
//    s = 1..b, the points with xb - s*R <= x < xb + s*R -- those stage 1
//    left below level s -- advance from level s-1 to s.
//
// A point at distance d from its tile's nearer edge thus takes
// min(b, floor(d / R)) steps in stage 1 and the rest in stage 2; for W = 9,
// b = 4, R = 1 the stage-1 counts are 0,1,2,3,4,3,2,1,0 and the stage-2
// counts 4,3,2,1,0,1,2,3,4, the profiles the paper draws.  Both stages use
// the two Jacobi arrays of the time loop: level s goes to array s mod 2, so
// every point's two latest levels stay readable.  Step s of stage 2 reads
// the points within (s+1)R of its boundary at level s-1; with W >= 2bR each
// of them is either one this boundary advanced itself or one stage 1 left at
// level s-1 or s (whose level s-1 is still in array (s-1) mod 2), and the two
// boundaries of a tile write disjoint points.  The window of 2(b+1)R points a
// boundary reads must also be distinct points of the line: n >= 2(b+1)R.
#pragma once

namespace sg {
namespace tess {

// Stage 1, step s: local indices [s*R, W - s*R) of a tile of width W.
__host__ __device__ inline int s1_lo(int s, int R) { return s * R; }
__host__ __device__ inline int s1_hi(int s, int R, int W) { return W - s * R; }

// Stage 2, step s: offsets t from the boundary with -s*R <= t < s*R.
__host__ __device__ inline int s2_lo(int s, int R) { return -s * R; }
__host__ __device__ inline int s2_hi(int s, int R) { return s * R; }

// Half-width of the window a stage-2 CTA loads around its boundary.
__host__ __device__ inline int s2_half(int b, int R) { return (b + 1) * R; }

// Smallest tile width for which the two stages stay apart.
__host__ __device__ inline int min_width(int b, int R) { return 2 * b * R; }

}  // namespace tess
}  // namespace sg
