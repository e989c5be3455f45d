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
//
// Run by every thread of the last block of the reduction (nrm2 valid in thread 0).  What
// the sequential part needs (H's column j, the previous rotations, g, or the whole small H
// of an inner level) is first staged in shared memory by parallel loads, one thread then
// works on the staged copy, and the block writes the results back in parallel, so the
// epilogue costs a few memory round trips instead of one per Hessenberg entry.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void update_epilogue_block(double nrm2, KState ks, int j, int mode,
                                                      int second) {
    __shared__ double sh[MK_MAX_RESTART + 2];
    __shared__ double scs[MK_MAX_RESTART], ssn[MK_MAX_RESTART];
    __shared__ double sg[MK_MAX_RESTART + 1];
    __shared__ double sy[MK_MAX_RESTART];
    __shared__ double sR[(MK_MAX_INNER + 1) * MK_MAX_INNER];
    __shared__ double sval[4];
    __shared__ int sact;
    const int tid = threadIdx.x;
    const int nth = blockDim.x;
    const int m = ks.m;
    double *misc = ks.misc();
    double *Hj = ks.H() + (int64_t)j * (m + 1);
    const bool givens = (mode & UPD_GIVENS) != 0;
    const bool lsq = !givens && (mode & UPD_INNER_LSQ) && j == m - 1;
    if (tid == 0) {
        sval[0] = nrm2;
        sval[1] = misc[2];
        sval[2] = misc[0];
        sval[3] = misc[1];
    }
    if (givens) {
        for (int i = tid; i <= j; i += nth) {
            sh[i] = Hj[i];
            sg[i] = ks.g()[i];
        }
        for (int i = tid; i < j; i += nth) {
            scs[i] = ks.cs()[i];
            ssn[i] = ks.sn()[i];
        }
    } else if (lsq) {
        for (int i = tid; i < (m + 1) * m; i += nth) sR[i] = ks.H()[i];
    }
    __syncthreads();
    if (tid == 0) {
        const double nrm = sqrt(sval[0]);
        int act = 0;   // 0 nothing to write back, 1 Givens column, 2 column + solution, 3 inner LSQ
        if (!isfinite(nrm)) {
            ks.flags[3] = 1;
            ks.flags[0] = 1;
            ks.flags[1] = 0;
        } else if (!second && ((mode & UPD_REORTH_ALWAYS) ||
                               ((mode & UPD_REORTH) && nrm < 0.70710678118654752 * sqrt(sval[1])))) {
            ks.flags[2] = 1;  // a second Gram-Schmidt pass follows
        } else {
            ks.flags[2] = 0;
            Hj[j + 1] = nrm;
            ks.sigma()[j + 1] = nrm > 0.0 ? 1.0 / nrm : 0.0;
            if (givens) {
                sh[j + 1] = nrm;
                for (int i = 0; i < j; ++i) {
                    const double t = scs[i] * sh[i] + ssn[i] * sh[i + 1];
                    sh[i + 1] = -ssn[i] * sh[i] + scs[i] * sh[i + 1];
                    sh[i] = t;
                }
                const double a = sh[j], b = sh[j + 1];
                const double r = sqrt(a * a + b * b);
                const double c = r > 0.0 ? a / r : 1.0, sn = r > 0.0 ? b / r : 0.0;
                sh[j] = r;
                sh[j + 1] = 0.0;
                scs[j] = c;
                ssn[j] = sn;
                sg[j + 1] = -sn * sg[j];
                sg[j] = c * sg[j];
                const double est = fabs(sg[j + 1]);
                misc[6] = est;
                ks.flags[4] += 1;
                const bool conv = (est <= sval[3]) || (nrm == 0.0);
                act = 1;
                if (conv || j == m - 1) {
                    // y = R^{-1} g over the jf = j + 1 columns; column j is the staged one
                    const int jf = j + 1;
                    ks.flags[1] = jf;
                    for (int c2 = jf - 1; c2 >= 0; --c2) {
                        double sacc = sg[c2];
                        for (int k = c2 + 1; k < jf; ++k) {
                            const double rk = (k == j) ? sh[c2] : ks.H()[c2 + (int64_t)k * (m + 1)];
                            sacc -= rk * sy[k];
                        }
                        const double d = (c2 == j) ? sh[c2] : ks.H()[c2 + (int64_t)c2 * (m + 1)];
                        sy[c2] = (fabs(d) > 0.0) ? sacc / d : 0.0;
                    }
                    if (conv) ks.flags[0] = 1;
                    act = 2;
                }
            } else if (lsq) {
                sR[j * (m + 1) + j + 1] = nrm;
                givens_solve(sR, m + 1, m, sval[2], sg, sy, nullptr);
                act = 3;
            }
        }
        sact = act;
    }
    __syncthreads();
    const int act = sact;
    if (act == 1 || act == 2) {
        for (int i = tid; i <= j + 1; i += nth) Hj[i] = sh[i];
        if (tid == 0) {
            ks.cs()[j] = scs[j];
            ks.sn()[j] = ssn[j];
            ks.g()[j] = sg[j];
            ks.g()[j + 1] = sg[j + 1];
        }
        if (act == 2)
            for (int i = tid; i <= j; i += nth) ks.y()[i] = sy[i];
    } else if (act == 3) {
        for (int i = tid; i < m; i += nth) ks.y()[i] = sy[i];
        for (int i = tid; i <= m; i += nth) ks.g()[i] = sg[i];
    }
}

}  // namespace mk
