// Counterpart form of folded 2D weights (Section 3.3, Eq. vfold and
// Eq. horifold; Section 3.5's reuse of counterparts).
//
// The paper folds each column of a point square vertically into counterparts
// and combines them horizontally; in general (Section 3.5) a counterpart is
// a weighted sum of others plus a correction.  Written exactly, that is a
// factorisation of the (2R+1) x (2R+1) folded weights into separable terms,
//   c^(m)[a][b] = sum_{k<K} u_k[a] v_k[b],
// where the u_k fold columns (the counterparts) and the v_k combine them.
// Gaussian elimination with complete pivoting finds the smallest such K (the
// rank) and the factors: each step takes the largest remaining entry as the
// pivot, splits off the rank-one term through its row and column, and stops
// when what is left is zero to FP64 rounding.
#include <cmath>
#include <vector>

#include "plan.h"

namespace sg {

int cp_factor(const double *c, int W, int max_k, double *u, double *v)
{
    std::vector<double> A(c, c + (size_t)W * W);
    double scale = 0.0;
    for (double x : A) scale = std::fmax(scale, std::fabs(x));
    if (scale == 0.0) return 0;
    const double tol = 1e-12 * scale;
    int k = 0;
    for (;; ++k) {
        int pi = 0, pj = 0;
        double best = 0.0;
        for (int i = 0; i < W; ++i)
            for (int j = 0; j < W; ++j)
                if (std::fabs(A[i * W + j]) > best) {
                    best = std::fabs(A[i * W + j]);
                    pi = i;
                    pj = j;
                }
        if (best <= tol) return k;
        if (k == max_k) return k + 1;  // more terms than asked for
        const double piv = A[pi * W + pj];
        double *uk = u + (size_t)k * W, *vk = v + (size_t)k * W;
        for (int i = 0; i < W; ++i) uk[i] = A[i * W + pj] / piv;  // column, 1 at the pivot row
        for (int j = 0; j < W; ++j) vk[j] = A[pi * W + j];        // row
        for (int i = 0; i < W; ++i)
            for (int j = 0; j < W; ++j) A[i * W + j] -= uk[i] * vk[j];
    }
}

// The counterpart form of c^(m) this plan runs, by m (cached).  k = 0 means
// the direct form: the rank is above 2, there is no kernel for the radius,
// the option says never, or (automatic choice) the two 1D folds per point,
// 2K(2R+1) multiply-adds plus a shared-memory round trip, would not undercut
// the nonzeros of c^(m), or the sweep is a plain radius-1 or -2 one.
stencil_status_t plan_counterparts(stencil_plan_s *p, int m, const CpFactor **out)
{
    auto it = p->cp.find(m);
    if (it == p->cp.end()) {
        CpFactor f;
        if (p->ndim == 2 && p->counterparts != 2) {
            const std::vector<double> *cm = nullptr;
            stencil_status_t st = plan_folded(p, m, &cm);
            if (st != STENCIL_OK) return st;
            const int R = m * p->r, W = 2 * R + 1;
            std::vector<double> u(2 * W), v(2 * W);
            const int rank = cp_factor(cm->data(), W, 2, u.data(), v.data());
            int nnz = 0;
            for (double x : *cm) nnz += x != 0.0;
            const bool have = rank >= 1 && rank <= 2 && sweep2d_supported(1, R, PAT_CP1 + rank - 1);
            // plain radius-1..2 sweeps are memory-bound: the split pays from
            // a fold or a wide base on
            const bool cheaper = (m >= 2 || R >= 3) && 2 * rank * W + 4 < nnz;
            if (have && (p->counterparts == 1 || cheaper)) {
                f.k = rank;
                f.u.assign(u.begin(), u.begin() + rank * W);
                f.v.assign(v.begin(), v.begin() + rank * W);
            } else if (p->counterparts == 1) {
                set_error("counterpart form: c^(%d) has rank %d (at most 2 supported) or no "
                          "kernel for radius %d",
                          m, rank, R);
                return STENCIL_ERR_UNSUPPORTED;
            }
        }
        it = p->cp.emplace(m, f).first;
    }
    *out = &it->second;
    return STENCIL_OK;
}

}  // namespace sg

extern "C" stencil_status_t stencil_fold_counterparts(int W, const double *folded, int max_k,
                                                      int *k_out, double *u_out, double *v_out)
{
    if (W < 1 || W > 2 * sg::kMaxR2D + 1 || !folded || max_k < 1 || max_k > W || !k_out ||
        !u_out || !v_out) {
        sg::set_error("stencil_fold_counterparts: bad argument");
        return STENCIL_ERR_INVALID_ARG;
    }
    *k_out = sg::cp_factor(folded, W, max_k, u_out, v_out);
    return STENCIL_OK;
}
