// Command-line harness for the host-side setup numerics of libmk (csrc/setup.cpp), built and
// run by tests/test_host_setup.py on the CPU (no GPU, no CUDA kernels).  Prints numbers as
// whitespace-separated text:
//   agg  n tau k       -> m, then lo, di, up of fd_laplacian(n, tau) agglomerated k times
//   lmax n tau k       -> largest eigenvalue of -L for that operator
//   eig  n tau k       -> m, lam (m), S (m x m row-major), S^{-1} (m x m)
//   uni  n tau k       -> 1 c  if the operator is c tridiag(1, -2, 1), else 0 0
//   dst  n c a b       -> alpha (n), beta (n) of the sine-transform slab tables
//   geom dim nx ny nt  -> ldx plane guard len of the padded layout
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "mk_internal.h"

using namespace mk;

static Tri op(int argc, char **argv) {
    if (argc < 5) std::exit(2);
    Tri t = fd_laplacian(std::atoi(argv[2]), std::atof(argv[3]));
    for (int k = std::atoi(argv[4]); k > 0; --k) t = agglomerate(t);
    return t;
}

static void put(const std::vector<double> &v) {
    for (double x : v) std::printf("%.17g\n", x);
}

int main(int argc, char **argv) {
    if (argc < 2) return 2;
    const char *cmd = argv[1];
    if (!std::strcmp(cmd, "agg")) {
        Tri t = op(argc, argv);
        std::printf("%d\n", t.n());
        put(t.lo);
        put(t.di);
        put(t.up);
    } else if (!std::strcmp(cmd, "lmax")) {
        std::printf("%.17g\n", tri_lambda_max_neg(op(argc, argv)));
    } else if (!std::strcmp(cmd, "eig")) {
        Tri t = op(argc, argv);
        std::vector<double> lam, S, Si;
        tri_eigen(t, lam, S, Si);
        std::printf("%d\n", t.n());
        put(lam);
        put(S);
        put(Si);
    } else if (!std::strcmp(cmd, "uni")) {
        double c = 0.0;
        const bool u = tri_uniform(op(argc, argv), c);
        std::printf("%d %.17g\n", u ? 1 : 0, u ? c : 0.0);
    } else if (!std::strcmp(cmd, "dst")) {
        if (argc < 6) return 2;
        std::vector<double> tab, tw;
        dst_tables(std::atoi(argv[2]), std::atof(argv[3]), std::atof(argv[4]), std::atof(argv[5]),
                   tab, tw);
        put(tab);
    } else if (!std::strcmp(cmd, "geom")) {
        if (argc < 6) return 2;
        Geom g = make_geom(std::atoi(argv[2]), std::atoi(argv[3]), std::atoi(argv[4]),
                           std::atoi(argv[5]));
        std::printf("%d %lld %lld %lld\n", g.ldx, (long long)g.plane, (long long)g.guard,
                    (long long)g.len);
    } else {
        return 2;
    }
    return 0;
}
