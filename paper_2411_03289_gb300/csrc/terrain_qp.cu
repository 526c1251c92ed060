// Terrain-weight estimation, Eq. 4 (Alg. 1 Step 3), host code.
//
//   w* = argmin_w |Y_v - F_v w|^2 + |Y_w - F_w w|^2 + gamma |w - w_prev|_1
//        s.t. 0 <= w_i <= 1, sum_i w_i = 1
//
// The objective is convex and piecewise quadratic.  At the minimiser every
// weight is either 0, equal to its previous value (a kink of the L1 term),
// or strictly above / below it; on the face that this pattern fixes, the
// free weights minimise a quadratic with a linear term gamma s_i and the one
// equality constraint, i.e. they solve a small KKT system.  With M <= 8
// terrains all 4^M patterns are solved (each a system of at most M + 1
// unknowns); the feasible candidate of least objective is the minimiser.
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace {

// A x = b for n <= 9 by Gaussian elimination with partial pivoting; false
// when a pivot is negligible against the matrix scale.
bool solve_small(double* A, double* b, int n, double scale) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (std::fabs(A[piv * n + c]) <= 1e-13 * scale) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r * n + c] / A[c * n + c];
            if (f == 0.0) continue;
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double v = b[r];
        for (int k = r + 1; k < n; ++k) v -= A[r * n + k] * b[k];
        b[r] = v / A[r * n + r];
    }
    return true;
}

}  // namespace

extern "C" int terrain_weights(const double* Yv, const double* Yw, const double* Fv, const double* Fw,
                               int32_t H, int32_t M, const double* w_prev, double gamma, double* w_out) {
    using gpm::fail;
    if (!Yv || !Yw || !Fv || !Fw || !w_prev || !w_out)
        return fail(GPMPPI_ERR_INVALID_ARG, "terrain_weights: NULL argument");
    if (H < 1 || M < 1 || M > gpm::kMaxTerrains)
        return fail(GPMPPI_ERR_INVALID_ARG, "terrain_weights: H >= 1 and 1 <= M <= 8 required");
    if (!(gamma >= 0.0) || !std::isfinite(gamma))
        return fail(GPMPPI_ERR_INVALID_ARG, "terrain_weights: gamma must be finite and >= 0");
    for (int h = 0; h < H; ++h) {
        if (!std::isfinite(Yv[h]) || !std::isfinite(Yw[h]))
            return fail(GPMPPI_ERR_NONFINITE, "terrain_weights: non-finite observation");
        for (int i = 0; i < M; ++i)
            if (!std::isfinite(Fv[h * M + i]) || !std::isfinite(Fw[h * M + i]))
                return fail(GPMPPI_ERR_NONFINITE, "terrain_weights: non-finite prediction");
    }
    for (int i = 0; i < M; ++i)
        if (!std::isfinite(w_prev[i])) return fail(GPMPPI_ERR_NONFINITE, "terrain_weights: non-finite w_prev");
    // Q = Fv^T Fv + Fw^T Fw, c = Fv^T Yv + Fw^T Yw, y2 = |Yv|^2 + |Yw|^2
    double Q[64] = {0}, c[8] = {0}, y2 = 0.0;
    for (int h = 0; h < H; ++h) {
        y2 += Yv[h] * Yv[h] + Yw[h] * Yw[h];
        for (int i = 0; i < M; ++i) {
            c[i] += Fv[h * M + i] * Yv[h] + Fw[h * M + i] * Yw[h];
            for (int j = 0; j < M; ++j) Q[i * M + j] += Fv[h * M + i] * Fv[h * M + j] + Fw[h * M + i] * Fw[h * M + j];
        }
    }
    double qscale = 1.0;
    for (int i = 0; i < M; ++i) qscale = std::fmax(qscale, std::fabs(Q[i * M + i]));
    auto objective = [&](const double* w) {
        double v = y2;
        for (int i = 0; i < M; ++i) {
            v -= 2.0 * c[i] * w[i];
            for (int j = 0; j < M; ++j) v += w[i] * Q[i * M + j] * w[j];
            v += gamma * std::fabs(w[i] - w_prev[i]);
        }
        return v;
    };
    const double tol = 1e-10;
    double best = INFINITY, wbest[8] = {0};
    int npat = 1;
    for (int i = 0; i < M; ++i) npat *= 4;
    for (int pat = 0; pat < npat; ++pat) {
        int st[8], free_idx[8], nf = 0;
        double w[8], fixed_sum = 0.0;
        bool ok = true;
        for (int i = 0, p = pat; i < M; ++i, p /= 4) {
            st[i] = p % 4;              // 0: zero, 1: at w_prev, 2: above, 3: below
            if (st[i] == 0) w[i] = 0.0;
            if (st[i] == 1) {
                if (w_prev[i] < 0.0 || w_prev[i] > 1.0) ok = false;
                w[i] = w_prev[i];
            }
            if (st[i] >= 2) free_idx[nf++] = i;
            else fixed_sum += w[i];
        }
        if (!ok) continue;
        if (nf == 0) {
            if (std::fabs(fixed_sum - 1.0) > tol) continue;
        } else {
            // [2 Q_RR  1] [w_R   ]   [2 c_R - gamma s_R - 2 Q_RF w_F]
            // [1^T     0] [lambda] = [1 - sum w_F                   ]
            const int n = nf + 1;
            double A[81], b[9];
            for (int r = 0; r < nf; ++r) {
                const int i = free_idx[r];
                for (int q = 0; q < nf; ++q) A[r * n + q] = 2.0 * Q[i * M + free_idx[q]];
                A[r * n + nf] = 1.0;
                double rhs = 2.0 * c[i] - gamma * (st[i] == 2 ? 1.0 : -1.0);
                for (int j = 0; j < M; ++j)
                    if (st[j] < 2) rhs -= 2.0 * Q[i * M + j] * w[j];
                b[r] = rhs;
                A[nf * n + r] = 1.0;
            }
            A[nf * n + nf] = 0.0;
            b[nf] = 1.0 - fixed_sum;
            double A0[81], b0[9];
            std::memcpy(A0, A, sizeof(A));
            std::memcpy(b0, b, sizeof(b));
            if (!solve_small(A, b, n, qscale)) {
                // a flat direction: minimise the slightly regularised quadratic instead
                for (int r = 0; r < nf; ++r) A0[r * n + r] += 1e-12 * qscale;
                if (!solve_small(A0, b0, n, qscale)) continue;
                std::memcpy(b, b0, sizeof(b0));
            }
            for (int r = 0; r < nf; ++r) {
                const int i = free_idx[r];
                w[i] = b[r];
                const double sgn = (st[i] == 2) ? 1.0 : -1.0;
                if (w[i] < -tol || w[i] > 1.0 + tol || sgn * (w[i] - w_prev[i]) < -tol) ok = false;
            }
            if (!ok) continue;
        }
        for (int i = 0; i < M; ++i) w[i] = std::fmin(1.0, std::fmax(0.0, w[i]));
        const double v = objective(w);
        if (v < best) {
            best = v;
            std::memcpy(wbest, w, sizeof(double) * M);
        }
    }
    if (!std::isfinite(best)) return fail(GPMPPI_ERR_CUDA, "terrain_weights: no feasible candidate (internal)");
    double sum = 0.0;
    for (int i = 0; i < M; ++i) sum += wbest[i];
    for (int i = 0; i < M; ++i) w_out[i] = wbest[i] / sum;
    return GPMPPI_OK;
}
