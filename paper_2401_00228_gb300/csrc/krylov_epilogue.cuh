// Device-side least squares and Arnoldi bookkeeping shared by the Krylov kernels.
#pragma once

#include "kernels.h"

namespace mk {

// ---------------------------------------------------------------------------------------
// Givens least squares helpers (one thread).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void givens_solve(double *R, int ld, int n, double beta, double *gg, double *y,
                             double *res) {
    // least squares min || beta e1 - H y ||, H (n+1) x n (column-major, leading dim ld),
    // rotated in place into R; gg receives the rotated right-hand side (n+1 entries)
    for (int r = 0; r <= n; ++r) gg[r] = 0.0;
    gg[0] = beta;
    for (int c = 0; c < n; ++c) {
        double a = R[c + c * ld], b = R[c + 1 + c * ld];
        double rr = sqrt(a * a + b * b);
        double cs = rr > 0.0 ? a / rr : 1.0, sn = rr > 0.0 ? b / rr : 0.0;
        for (int k = c; k < n; ++k) {
            double t1 = R[c + k * ld], t2 = R[c + 1 + k * ld];
            R[c + k * ld] = cs * t1 + sn * t2;
            R[c + 1 + k * ld] = -sn * t1 + cs * t2;
        }
        double t1 = gg[c], t2 = gg[c + 1];
        gg[c] = cs * t1 + sn * t2;
        gg[c + 1] = -sn * t1 + cs * t2;
    }
    for (int c = n - 1; c >= 0; --c) {
        double s = gg[c];
        for (int k = c + 1; k < n; ++k) s -= R[c + k * ld] * y[k];
        double d = R[c + c * ld];
        y[c] = (fabs(d) > 0.0) ? s / d : 0.0;
    }
    if (res) *res = fabs(gg[n]);
}

// ---------------------------------------------------------------------------------------
// update: V_{j+1} = src - sum_i c_i V_i, c_i = tmp_i sigma_i ; ||.||^2 ; epilogue.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void update_epilogue(double nrm2, KState ks, int j, int mode, int second) {
    double nrm = sqrt(nrm2);
    double *misc = ks.misc();
    const int m = ks.m;
    if (!isfinite(nrm)) {
        ks.flags[3] = 1;
        ks.flags[0] = 1;
        ks.flags[1] = 0;
        return;
    }
    if (!second && ((mode & UPD_REORTH_ALWAYS) ||
                    ((mode & UPD_REORTH) && nrm < 0.70710678118654752 * sqrt(misc[2])))) {
        ks.flags[2] = 1;  // a second Gram-Schmidt pass follows
        return;
    }
    ks.flags[2] = 0;
    double *H = ks.H() + (int64_t)j * (m + 1);
    H[j + 1] = nrm;
    ks.sigma()[j + 1] = nrm > 0.0 ? 1.0 / nrm : 0.0;
    if (mode & UPD_GIVENS) {
        double *cs = ks.cs(), *sn = ks.sn(), *g = ks.g();
        for (int i = 0; i < j; ++i) {
            double t = cs[i] * H[i] + sn[i] * H[i + 1];
            H[i + 1] = -sn[i] * H[i] + cs[i] * H[i + 1];
            H[i] = t;
        }
        double a = H[j], b = H[j + 1];
        double r = sqrt(a * a + b * b);
        double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
        H[j] = r;
        H[j + 1] = 0.0;
        cs[j] = c;
        sn[j] = s;
        g[j + 1] = -s * g[j];
        g[j] = c * g[j];
        double est = fabs(g[j + 1]);
        misc[6] = est;
        ks.flags[4] += 1;
        bool conv = (est <= misc[1]) || (nrm == 0.0);
        if (conv || j == m - 1) {
            int jf = j + 1;
            ks.flags[1] = jf;
            double *y = ks.y();
            for (int c2 = jf - 1; c2 >= 0; --c2) {
                double sacc = g[c2];
                for (int k = c2 + 1; k < jf; ++k) sacc -= ks.H()[c2 + (int64_t)k * (m + 1)] * y[k];
                double d = ks.H()[c2 + (int64_t)c2 * (m + 1)];
                y[c2] = (fabs(d) > 0.0) ? sacc / d : 0.0;
            }
            if (conv) ks.flags[0] = 1;
        }
    } else if (mode & UPD_INNER_LSQ) {
        if (j == m - 1) givens_solve(ks.H(), m + 1, m, misc[0], ks.g(), ks.y(), nullptr);
    }
}

}  // namespace mk
