// Host-side numerics of the level hierarchy (FP64, run once per hierarchy).
//
//  * fd_laplacian: A_n / tau scaled by tau, second-order FD, zero Dirichlet (Sec. 3.3).
//  * agglomerate:  L' = Y^T L Z with the agglomeration matrices of Eqs. (constructZ) and
//                  (constructY): aggregates {2j, 2j+1}, a trailing singleton for odd n.
//  * tri_lambda_max_neg: largest eigenvalue of -L, for the shift mu = lambda_max(A_l)
//                  (Sec. 3.1); A_l is block triangular, so lambda_max(A_l) = 1 + a lambda_max(-L).
//  * pcr_tables:   coefficient tables of parallel cyclic reduction on I - aL.
//  * tri_eigen:    L = S diag(lam) S^{-1} for the fast-diagonalisation slab solver.
#include <algorithm>
#include <array>
#include <cmath>

#include "mk_internal.h"

namespace mk {

Geom make_geom(int dim, int nx, int ny, int nt) {
    Geom g;
    g.dim = dim;
    g.nx = nx;
    g.ny = dim == 1 ? 1 : ny;
    g.nt = nt;
    g.ldx = ((nx + 1 + 7) / 8) * 8;
    g.plane = dim == 1 ? (int64_t)g.ldx : (int64_t)(g.ny + 1) * g.ldx;
    g.guard = g.ldx;
    int64_t len = g.guard + (int64_t)(nt + 1) * g.plane + g.ldx;
    // a whole number of 4096-element tiles: the Krylov kernels then sweep tiles without
    // bounds checks (the extra elements are zero like the rest of the padding)
    g.len = ((len + 4095) / 4096) * 4096;
    return g;
}

Tri fd_laplacian(int n, double tau) {
    Tri t;
    double h = 1.0 / (n + 1);
    double c = tau / (h * h);
    t.lo.assign(n, c);
    t.up.assign(n, c);
    t.di.assign(n, -2.0 * c);
    t.lo[0] = 0.0;
    t.up[n - 1] = 0.0;
    return t;
}

static double Lentry(const Tri &L, int p, int q) {
    if (p == q) return L.di[p];
    if (q == p - 1) return L.lo[p];
    if (q == p + 1) return L.up[p];
    return 0.0;
}

Tri agglomerate(const Tri &L) {
    const int n = L.n();
    const int m = (n + 1) / 2;
    Tri c;
    c.lo.assign(m, 0.0);
    c.di.assign(m, 0.0);
    c.up.assign(m, 0.0);
    auto members = [&](int j, int &p0, int &p1) {
        p0 = 2 * j;
        p1 = std::min(2 * j + 1, n - 1);
    };
    for (int j = 0; j < m; ++j) {
        int a0, a1;
        members(j, a0, a1);
        double inv = 1.0 / (a1 - a0 + 1);
        for (int jj = std::max(0, j - 1); jj <= std::min(m - 1, j + 1); ++jj) {
            int b0, b1;
            members(jj, b0, b1);
            double s = 0.0;
            for (int p = a0; p <= a1; ++p)
                for (int q = b0; q <= b1; ++q) s += Lentry(L, p, q);
            s *= inv;
            if (jj == j) c.di[j] = s;
            else if (jj == j - 1) c.lo[j] = s;
            else c.up[j] = s;
        }
    }
    return c;
}

// Symmetrised off-diagonal of a tridiagonal matrix whose off-diagonal products are >= 0.
static double sym_off(const Tri &L, int i) {   // between i and i+1
    double p = L.lo[i + 1] * L.up[i];
    return p > 0.0 ? std::sqrt(p) : 0.0;
}

double tri_lambda_max_neg(const Tri &L) {
    // eigenvalues of -L = eigenvalues of the symmetric tridiagonal T (diag -di, off -e)
    const int n = L.n();
    std::vector<double> d(n), e2(std::max(0, n - 1));
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
        d[i] = -L.di[i];
        double r = 0.0;
        if (i > 0) r += sym_off(L, i - 1);
        if (i < n - 1) r += sym_off(L, i);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    for (int i = 0; i + 1 < n; ++i) {
        double e = sym_off(L, i);
        e2[i] = e * e;
    }
    // count of eigenvalues < x (Sturm sequence / LDL^T inertia)
    auto count_below = [&](double x) {
        int c = 0;
        double q = 1.0;
        for (int i = 0; i < n; ++i) {
            q = (d[i] - x) - (i > 0 ? e2[i - 1] / q : 0.0);
            if (q == 0.0) q = -1e-300;
            if (q < 0.0) ++c;
        }
        return c;
    };
    double a = lo - 1.0, b = hi + 1.0;   // count(a) = 0, count(b) = n
    for (int it = 0; it < 200 && b - a > 1e-15 * std::max(1.0, std::fabs(b)); ++it) {
        double mid = 0.5 * (a + b);
        if (count_below(mid) >= n) b = mid;
        else a = mid;
    }
    return 0.5 * (a + b);
}

int pcr_levels(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

void pcr_tables(const Tri &L, double a, int npad, std::vector<double> &alpha,
                std::vector<double> &gamma, std::vector<double> &binv) {
    const int n = L.n();
    const int nlev = pcr_levels(n);
    std::vector<double> A(npad, 0.0), B(npad, 1.0), C(npad, 0.0);
    for (int i = 0; i < n; ++i) {
        A[i] = -a * L.lo[i];
        B[i] = 1.0 - a * L.di[i];
        C[i] = -a * L.up[i];
    }
    alpha.assign((size_t)nlev * npad, 0.0);
    gamma.assign((size_t)nlev * npad, 0.0);
    std::vector<double> A2(npad), B2(npad), C2(npad);
    for (int l = 0; l < nlev; ++l) {
        const int s = 1 << l;
        for (int i = 0; i < npad; ++i) {
            double al = (i - s >= 0) ? -A[i] / B[i - s] : 0.0;
            double ga = (i + s < npad) ? -C[i] / B[i + s] : 0.0;
            alpha[(size_t)l * npad + i] = al;
            gamma[(size_t)l * npad + i] = ga;
            A2[i] = (i - s >= 0) ? al * A[i - s] : 0.0;
            C2[i] = (i + s < npad) ? ga * C[i + s] : 0.0;
            B2[i] = B[i] + ((i - s >= 0) ? al * C[i - s] : 0.0) + ((i + s < npad) ? ga * A[i + s] : 0.0);
        }
        A.swap(A2);
        B.swap(B2);
        C.swap(C2);
    }
    binv.assign(npad, 0.0);
    for (int i = 0; i < npad; ++i) binv[i] = 1.0 / B[i];
}

// Tables of the partitioned (spike) slab solver for M = I - aL (see slab.cu,
// k_slab_1d_spike).  The system is padded to P*U rows (identity beyond n) and split into P
// blocks of U rows, one per thread (P = 32 * warps).  Per thread p (rows pU .. pU+U-1),
// stored item-major (item * P + p):
//   m[U]     Thomas multipliers (m[0] unused)      uinv[U]  1 / pivots
//   sup[U]   super-diagonal of the block            v[U], w[U]  spikes M_p^{-1} e_0, e_{U-1}
//   lo, di, up [U each]  the rows of L (for the explicit part (I + bL) x_{k-1})
//   A, C     couplings M[pU, pU-1], M[pU+U-1, pU+U]
//   alpha[nl][4], gamma[nl][4]  2x2 block-PCR multipliers on the interface unknowns
//                               (F_p, G_p) = (x[pU], x[pU+U-1]), strides 1, 2, .., P/2
//   dinv[4]  inverse of the final 2x2 diagonal block
// with nl = log2(P).
int spike_levels(int P) {
    int l = 0;
    while ((1 << l) < P) ++l;
    return l;
}

int spike_items(int U, int P) { return 8 * U + 2 + 8 * spike_levels(P) + 4; }

void spike_tables(const Tri &L, double a, int U, int P, std::vector<double> &tab) {
    const int n = L.n();
    const int N = P * U;
    const int nl = spike_levels(P);
    std::vector<double> sub(N, 0.0), dia(N, 1.0), sup(N, 0.0);
    for (int i = 0; i < n; ++i) {
        sub[i] = (i > 0) ? -a * L.lo[i] : 0.0;
        dia[i] = 1.0 - a * L.di[i];
        sup[i] = (i < n - 1) ? -a * L.up[i] : 0.0;
    }
    const int items = spike_items(U, P);
    tab.assign((size_t)items * P, 0.0);
    auto T = [&](int item, int p) -> double & { return tab[(size_t)item * P + p]; };
    typedef std::array<double, 4> M2;   // row-major 2x2
    std::vector<M2> D(P), E(P), Hm(P);
    for (int p = 0; p < P; ++p) {
        const int r0 = p * U;
        std::vector<double> m(U, 0.0), u(U), c(U, 0.0);
        u[0] = dia[r0];
        for (int q = 0; q < U; ++q) c[q] = (q < U - 1) ? sup[r0 + q] : 0.0;
        for (int q = 1; q < U; ++q) {
            m[q] = sub[r0 + q] / u[q - 1];
            u[q] = dia[r0 + q] - m[q] * c[q - 1];
        }
        auto solve = [&](std::vector<double> d) {
            for (int q = 1; q < U; ++q) d[q] -= m[q] * d[q - 1];
            std::vector<double> y(U);
            y[U - 1] = d[U - 1] / u[U - 1];
            for (int q = U - 2; q >= 0; --q) y[q] = (d[q] - c[q] * y[q + 1]) / u[q];
            return y;
        };
        std::vector<double> e0(U, 0.0), e1(U, 0.0);
        e0[0] = 1.0;
        e1[U - 1] = 1.0;
        std::vector<double> v = solve(e0), w = solve(e1);
        for (int q = 0; q < U; ++q) {
            T(q, p) = m[q];
            T(U + q, p) = 1.0 / u[q];
            T(2 * U + q, p) = c[q];
            T(3 * U + q, p) = v[q];
            T(4 * U + q, p) = w[q];
            const int i = r0 + q;
            T(5 * U + q, p) = (i < n) ? L.lo[i] : 0.0;
            T(6 * U + q, p) = (i < n) ? L.di[i] : 0.0;
            T(7 * U + q, p) = (i < n) ? L.up[i] : 0.0;
        }
        const double A = (p > 0) ? sub[r0] : 0.0;
        const double C = (p < P - 1) ? sup[r0 + U - 1] : 0.0;
        T(8 * U, p) = A;
        T(8 * U + 1, p) = C;
        // interface equations: z_p + E_p z_{p-1} + H_p z_{p+1} = (y_p[0], y_p[U-1])
        D[p] = {1.0, 0.0, 0.0, 1.0};
        E[p] = {0.0, A * v[0], 0.0, A * v[U - 1]};
        Hm[p] = {C * w[0], 0.0, C * w[U - 1], 0.0};
    }
    auto mul = [](const M2 &x, const M2 &y) {
        return M2{x[0] * y[0] + x[1] * y[2], x[0] * y[1] + x[1] * y[3],
                  x[2] * y[0] + x[3] * y[2], x[2] * y[1] + x[3] * y[3]};
    };
    auto inv = [](const M2 &x) {
        double det = x[0] * x[3] - x[1] * x[2];
        return M2{x[3] / det, -x[1] / det, -x[2] / det, x[0] / det};
    };
    auto add = [](const M2 &x, const M2 &y) {
        return M2{x[0] + y[0], x[1] + y[1], x[2] + y[2], x[3] + y[3]};
    };
    auto neg = [](const M2 &x) { return M2{-x[0], -x[1], -x[2], -x[3]}; };
    const M2 Z = {0.0, 0.0, 0.0, 0.0};
    for (int l = 0; l < nl; ++l) {
        const int s = 1 << l;
        std::vector<M2> D2(P), E2(P), H2(P);
        for (int p = 0; p < P; ++p) {
            M2 al = (p - s >= 0) ? neg(mul(E[p], inv(D[p - s]))) : Z;
            M2 ga = (p + s < P) ? neg(mul(Hm[p], inv(D[p + s]))) : Z;
            for (int e = 0; e < 4; ++e) {
                T(8 * U + 2 + l * 4 + e, p) = al[e];
                T(8 * U + 2 + 4 * nl + l * 4 + e, p) = ga[e];
            }
            D2[p] = D[p];
            if (p - s >= 0) D2[p] = add(D2[p], mul(al, Hm[p - s]));
            if (p + s < P) D2[p] = add(D2[p], mul(ga, E[p + s]));
            E2[p] = (p - s >= 0) ? mul(al, E[p - s]) : Z;
            H2[p] = (p + s < P) ? mul(ga, Hm[p + s]) : Z;
        }
        D.swap(D2);
        E.swap(E2);
        Hm.swap(H2);
    }
    for (int p = 0; p < P; ++p) {
        M2 di = inv(D[p]);
        for (int e = 0; e < 4; ++e) T(8 * U + 2 + 8 * nl + e, p) = di[e];
    }
}

// Cyclic Jacobi eigenvalue iteration for a dense symmetric matrix (row-major n x n).
static void jacobi_eigen(int n, std::vector<double> &Am, std::vector<double> &lam,
                         std::vector<double> &U) {
    U.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) U[(size_t)i * n + i] = 1.0;
    auto a = [&](int r, int c) -> double & { return Am[(size_t)r * n + c]; };
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < n; ++c) {
                double v = a(r, c) * a(r, c);
                tot += v;
                if (r != c) off += v;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = a(p, q);
                if (apq == 0.0) continue;
                double app = a(p, p), aqq = a(q, q);
                double th = (aqq - app) / (2.0 * apq);
                double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = a(k, p), akq = a(k, q);
                    a(k, p) = c * akp - s * akq;
                    a(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = a(p, k), aqk = a(q, k);
                    a(p, k) = c * apk - s * aqk;
                    a(q, k) = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double ukp = U[(size_t)k * n + p], ukq = U[(size_t)k * n + q];
                    U[(size_t)k * n + p] = c * ukp - s * ukq;
                    U[(size_t)k * n + q] = s * ukp + c * ukq;
                }
            }
    }
    lam.resize(n);
    for (int i = 0; i < n; ++i) lam[i] = a(i, i);
}

void tri_eigen(const Tri &L, std::vector<double> &lam, std::vector<double> &S,
               std::vector<double> &Sinv) {
    const int n = L.n();
    // L = D T D^{-1} with T symmetric: T_{i,i+1} = sqrt(lo_{i+1} up_i), d_{i+1} = d_i sqrt(lo_{i+1}/up_i)
    std::vector<double> dsc(n, 1.0);
    for (int i = 0; i + 1 < n; ++i) {
        double r = (L.lo[i + 1] > 0.0 && L.up[i] > 0.0) ? std::sqrt(L.lo[i + 1] / L.up[i]) : 1.0;
        dsc[i + 1] = dsc[i] * r;
    }
    std::vector<double> T((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        T[(size_t)i * n + i] = L.di[i];
        if (i + 1 < n) {
            double e = sym_off(L, i);
            T[(size_t)i * n + i + 1] = e;
            T[(size_t)(i + 1) * n + i] = e;
        }
    }
    std::vector<double> U;
    jacobi_eigen(n, T, lam, U);
    S.assign((size_t)n * n, 0.0);
    Sinv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            S[(size_t)i * n + j] = dsc[i] * U[(size_t)i * n + j];
            Sinv[(size_t)i * n + j] = U[(size_t)j * n + i] / dsc[j];
        }
}

// L = c tridiag(1, -2, 1) with zero ends (to a relative 1e-13): the operator the sine
// transform diagonalises.
bool tri_uniform(const Tri &L, double &c) {
    const int n = L.n();
    if (n < 1) return false;
    c = -0.5 * L.di[0];
    if (!(c > 0.0)) return false;
    const double tol = 1e-13 * c;
    for (int i = 0; i < n; ++i) {
        if (std::fabs(L.di[i] + 2.0 * c) > tol) return false;
        if (std::fabs(L.lo[i] - (i > 0 ? c : 0.0)) > tol) return false;
        if (std::fabs(L.up[i] - (i + 1 < n ? c : 0.0)) > tol) return false;
    }
    return true;
}

// Sine-transform slab tables for I - aL, I + bL with L = c tridiag(1, -2, 1):
//   tab = [alpha_j (n) | beta_j (n)], lam_j = -4c sin^2(pi (j+1) / (2(n+1))),
//   beta_j = 1 / (1 - a lam_j), alpha_j = (1 + b lam_j) beta_j.
void dst_tables(int n, double c, double a, double b, std::vector<double> &tab,
                std::vector<double> &tw) {
    const double pi = 3.14159265358979323846;
    const int N = n + 1;
    tab.assign(2 * (size_t)n, 0.0);
    for (int j = 0; j < n; ++j) {
        const double sj = std::sin(pi * (j + 1) / (2.0 * N));
        const double lam = -4.0 * c * sj * sj;
        const double beta = 1.0 / (1.0 - a * lam);
        tab[j] = (1.0 + b * lam) * beta;
        tab[n + j] = beta;
    }
    // twiddles exp(-2 pi i k r / (Ns R)) of the FFT passes over N2 = 2(n+1) points (radix 8,
    // then one radix-4 or radix-2 pass), interleaved (re, im), pass after pass
    tw.clear();
    const int N2 = 2 * N;
    int p = 0;
    while ((1 << p) < N2) ++p;
    int Ns = 1;
    while (p > 0) {
        const int R = p >= 3 ? 8 : (p == 2 ? 4 : 2);
        for (int k = 0; k < Ns; ++k)   // Ns (R - 1) entries per pass, also for Ns = 1
            for (int r = 1; r < R; ++r) {
                const double ang = -2.0 * pi * (double)k * r / ((double)Ns * R);
                tw.push_back(std::cos(ang));
                tw.push_back(std::sin(ang));
            }
        Ns *= R;
        p -= (R == 8 ? 3 : (R == 4 ? 2 : 1));
    }
    if (tw.empty()) tw.assign(2, 0.0);
}

}  // namespace mk
