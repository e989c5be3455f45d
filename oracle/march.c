/*
 * CPU oracle, plain C, FP64: sequential theta-march.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file; only the tests, the smoke check and the bench's CPU-baseline leg do.
 *
 * It solves the all-at-once system of Sec. 2, Eq. (finesys), by block forward
 * substitution, which is the sequential recurrence of Eq. (thetascheme) /
 * Eq. (timemarch):
 *
 *     u_0 = f_0,
 *     (I - a L) u_k = (I + b L) u_{k-1} + f_k,   k = 1..nt,
 *
 * with a = theta*dt and b = (1-theta)*dt on the fine grid (psi = I - aL,
 * phi = I + bL) and f_k = dt*((1-theta) g_{k-1} + theta g_k).  The same
 * routine marches any level of the hierarchy (other a, b, L).
 *
 * The spatial operator is a sum of one tridiagonal operator per direction,
 *     (Lx v)_i = lo[i] v_{i-1} + di[i] v_i + up[i] v_{i+1},  v_{-1} = v_n = 0,
 * which covers the second-order FD Laplacian of Sec. 3.3 (lo = up = tau/h^2,
 * di = -2 tau/h^2) and its agglomerated Galerkin versions.
 *
 * 1D: Thomas algorithm on I - aL, factored once.
 * 2D: banded LU (no pivoting; I - aL is strictly diagonally dominant), band
 *     half-width nx, factored once.  Unknown (j,i) has index j*nx + i.
 *
 * Compiled with -ffp-contract=off: every product and sum is rounded as written.
 */
#include <stdlib.h>
#include <string.h>

/* y = (I + b L) x for one time row, 1D. */
static void explicit_1d(int n, double b, const double *lo, const double *di,
                        const double *up, const double *x, double *y)
{
    for (int i = 0; i < n; ++i) {
        double lx = di[i] * x[i];
        if (i > 0) lx += lo[i] * x[i - 1];
        if (i < n - 1) lx += up[i] * x[i + 1];
        y[i] = x[i] + b * lx;
    }
}

int oracle_march_1d(int n, int nt, double a, double b,
                    const double *lo, const double *di, const double *up,
                    const double *f, double *u)
{
    if (n < 1 || nt < 0) return 1;
    double *cp = (double *)malloc(sizeof(double) * n);   /* modified super-diagonal */
    double *dinv = (double *)malloc(sizeof(double) * n); /* 1 / pivot */
    double *rhs = (double *)malloc(sizeof(double) * n);
    if (!cp || !dinv || !rhs) { free(cp); free(dinv); free(rhs); return 2; }

    /* Thomas factorisation of M = I - aL:  sub_i = -a lo_i, diag_i = 1 - a di_i, sup_i = -a up_i */
    for (int i = 0; i < n; ++i) {
        double sub = (i > 0) ? -a * lo[i] : 0.0;
        double diag = 1.0 - a * di[i];
        double sup = (i < n - 1) ? -a * up[i] : 0.0;
        double piv = (i > 0) ? diag - sub * cp[i - 1] : diag;
        dinv[i] = 1.0 / piv;
        cp[i] = sup * dinv[i];
    }

    memcpy(u, f, sizeof(double) * n); /* u_0 = f_0 */
    for (int k = 1; k <= nt; ++k) {
        const double *prev = u + (size_t)(k - 1) * n;
        double *cur = u + (size_t)k * n;
        const double *fk = f + (size_t)k * n;
        explicit_1d(n, b, lo, di, up, prev, rhs);
        for (int i = 0; i < n; ++i) rhs[i] += fk[i];
        /* forward elimination */
        for (int i = 0; i < n; ++i) {
            double sub = (i > 0) ? -a * lo[i] : 0.0;
            double r = rhs[i];
            if (i > 0) r -= sub * rhs[i - 1];
            rhs[i] = r * dinv[i];
        }
        /* back substitution */
        cur[n - 1] = rhs[n - 1];
        for (int i = n - 2; i >= 0; --i) cur[i] = rhs[i] - cp[i] * cur[i + 1];
    }
    free(cp); free(dinv); free(rhs);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* 2D                                                                         */
/* ------------------------------------------------------------------------- */

static void apply_L_2d(int nx, int ny, const double *xlo, const double *xdi, const double *xup,
                       const double *ylo, const double *ydi, const double *yup,
                       const double *v, double *out)
{
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            size_t p = (size_t)j * nx + i;
            double s = (xdi[i] + ydi[j]) * v[p];
            if (i > 0) s += xlo[i] * v[p - 1];
            if (i < nx - 1) s += xup[i] * v[p + 1];
            if (j > 0) s += ylo[j] * v[p - nx];
            if (j < ny - 1) s += yup[j] * v[p + nx];
            out[p] = s;
        }
    }
}

int oracle_march_2d(int nx, int ny, int nt, double a, double b,
                    const double *xlo, const double *xdi, const double *xup,
                    const double *ylo, const double *ydi, const double *yup,
                    const double *f, double *u)
{
    if (nx < 1 || ny < 1 || nt < 0) return 1;
    const int N = nx * ny;
    const int w = nx;              /* band half-width */
    const int W = 2 * w + 1;       /* band storage width: column q stored at [p][w + q - p] */
    double *band = (double *)calloc((size_t)N * W, sizeof(double));
    double *rhs = (double *)malloc(sizeof(double) * N);
    double *lv = (double *)malloc(sizeof(double) * N);
    if (!band || !rhs || !lv) { free(band); free(rhs); free(lv); return 2; }
#define B(p, q) band[(size_t)(p) * W + (w + (q) - (p))]

    /* assemble M = I - aL */
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            int p = j * nx + i;
            B(p, p) = 1.0 - a * (xdi[i] + ydi[j]);
            if (i > 0) B(p, p - 1) = -a * xlo[i];
            if (i < nx - 1) B(p, p + 1) = -a * xup[i];
            if (j > 0) B(p, p - nx) = -a * ylo[j];
            if (j < ny - 1) B(p, p + nx) = -a * yup[j];
        }
    }
    /* in-place banded LU without pivoting: L unit lower (multipliers), U upper */
    for (int k = 0; k < N; ++k) {
        double piv = B(k, k);
        int last = (k + w < N - 1) ? k + w : N - 1;
        for (int p = k + 1; p <= last; ++p) {
            double mult = B(p, k) / piv;
            B(p, k) = mult;
            if (mult != 0.0)
                for (int q = k + 1; q <= last; ++q) B(p, q) -= mult * B(k, q);
        }
    }

    memcpy(u, f, sizeof(double) * N);
    for (int k = 1; k <= nt; ++k) {
        const double *prev = u + (size_t)(k - 1) * N;
        double *cur = u + (size_t)k * N;
        const double *fk = f + (size_t)k * N;
        apply_L_2d(nx, ny, xlo, xdi, xup, ylo, ydi, yup, prev, lv);
        for (int p = 0; p < N; ++p) rhs[p] = prev[p] + b * lv[p] + fk[p];
        /* forward: L y = rhs */
        for (int p = 0; p < N; ++p) {
            int first = (p - w > 0) ? p - w : 0;
            double s = rhs[p];
            for (int q = first; q < p; ++q) s -= B(p, q) * rhs[q];
            rhs[p] = s;
        }
        /* backward: U x = y */
        for (int p = N - 1; p >= 0; --p) {
            int last = (p + w < N - 1) ? p + w : N - 1;
            double s = rhs[p];
            for (int q = p + 1; q <= last; ++q) s -= B(p, q) * cur[q];
            cur[p] = s / B(p, p);
        }
    }
#undef B
    free(band); free(rhs); free(lv);
    return 0;
}
