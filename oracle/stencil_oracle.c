/*
 * Plain FP64 CPU oracle for constant-coefficient stencils on periodic grids.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may link,
 * load or call this file; only the tests, the smoke check and the bench's CPU
 * baseline leg do.  It shares no code with the CUDA path.
 *
 * What it computes is the problem definition of Section 1 of Li et al.,
 * "Reducing Redundancy in Data Organization and Arithmetic Calculation for
 * Stencil Computations": every point at time t+1 is the weighted sum of
 * itself and its neighbours at time t, swept T times over the whole grid.
 * Two arrays alternate between odd and even time steps, as in the Jacobi
 * scheme the paper uses (Section 3.3, "Weighted Transpose").
 *
 * Readings taken where the paper is silent:
 *  - orientation: out[x] = sum_o c[o] * in[(x + o) mod N] (correlation form);
 *  - boundary: periodic in every axis;
 *  - coefficient layout: dense (2r+1)^ndim array, axis order (z, y, x), each
 *    axis indexed by offset + r; a star stencil has zeros off the axes.
 * Arithmetic is double throughout; no folding, blocking or reordering.
 * Taps whose weight is zero (the off-axis taps of a star) are skipped.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* index of (i - r) wrapped into [0, n) for i in [0, n + 2r) */
static int64_t *wrap_table(int64_t n, int r)
{
    int64_t *t = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 2 * r));
    if (!t) return NULL;
    for (int64_t i = 0; i < n + 2 * r; ++i) {
        int64_t v = (i - r) % n;
        if (v < 0) v += n;
        t[i] = v;
    }
    return t;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Runs T plain steps.  shape has ndim entries, shape[0] slowest.  `in` and
 * `out` hold prod(shape) doubles and may alias.  nthreads <= 0 uses the
 * OpenMP default.  Returns 0, or -1 on a bad argument or allocation failure.
 */
int oracle_stencil_run(int ndim, const int64_t *shape, int radius,
                       const double *coeffs, const double *in, double *out,
                       int64_t T, int nthreads)
{
    if (ndim < 1 || ndim > 3 || radius < 0 || T < 0 || !shape || !coeffs ||
        !in || !out)
        return -1;
    int64_t nz = 1, ny = 1, nx;
    int rz = 0, ry = 0, rx = radius;
    if (ndim == 3) { nz = shape[0]; ny = shape[1]; nx = shape[2]; rz = radius; ry = radius; }
    else if (ndim == 2) { ny = shape[0]; nx = shape[1]; ry = radius; }
    else { nx = shape[0]; }
    if (nz < 1 || ny < 1 || nx < 1) return -1;
    const int64_t n = nz * ny * nx;
    const int wx = 2 * rx + 1, wy = 2 * ry + 1, wz = 2 * rz + 1;

    double *a = (double *)malloc(sizeof(double) * (size_t)n);
    double *b = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t *tz = wrap_table(nz, rz), *ty = wrap_table(ny, ry), *tx = wrap_table(nx, rx);
    if (!a || !b || !tz || !ty || !tx) {
        free(a); free(b); free(tz); free(ty); free(tx);
        return -1;
    }
    memcpy(a, in, sizeof(double) * (size_t)n);
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    (void)nthreads;
#endif

    for (int64_t t = 0; t < T; ++t) {
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads)
#endif
        for (int64_t z = 0; z < nz; ++z) {
            for (int64_t y = 0; y < ny; ++y) {
                for (int64_t x = 0; x < nx; ++x) {
                    double s = 0.0;
                    for (int dz = 0; dz < wz; ++dz) {
                        const int64_t zz = tz[z + dz];
                        for (int dy = 0; dy < wy; ++dy) {
                            const int64_t row = (zz * ny + ty[y + dy]) * nx;
                            const double *c = coeffs + ((int64_t)dz * wy + dy) * wx;
                            for (int dx = 0; dx < wx; ++dx)
                                if (c[dx] != 0.0) s += c[dx] * a[row + tx[x + dx]];
                        }
                    }
                    b[(z * ny + y) * nx + x] = s;
                }
            }
        }
        double *tmp = a; a = b; b = tmp;
    }
    memcpy(out, a, sizeof(double) * (size_t)n);
    free(a); free(b); free(tz); free(ty); free(tx);
    return 0;
}
