// Internal declarations of libmk (not part of the ABI).
//
// Device layout of a space-time vector on one level (the "padded layout"):
//   element (k, j, i) lives at  guard + k*plane + j*ldx + i,
//   1D: plane = ldx,  2D: plane = (ny+1)*ldx  (row j = ny of every plane is a zero row),
//   ldx = round_up(nx+1, 8) (columns nx..ldx-1 are zero),  guard = ldx zeros in front,
//   and one more zero row after the last plane.
// With the zero padding every stencil neighbour (i-1, i+1, j-1, j+1) is a valid address
// that reads 0, which is exactly the zero Dirichlet boundary (Sec. 3.3), so the kernels
// carry no boundary branches.  Kernels write interior points only, and element-wise
// kernels map zeros to zeros, so the padding stays zero once allocated zeroed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mk.h"

namespace mk {

constexpr int MK_MAX_RESTART = 128;   // outer FGMRES(m) restart length limit
constexpr int MK_MAX_INNER = 8;       // fixed inner FGMRES iterations limit

// ---------------------------------------------------------------------------------------
// Geometry of one level.
// ---------------------------------------------------------------------------------------
struct Geom {
    int dim, nx, ny, ldx, nt;
    int64_t plane, guard, len;

    __host__ __device__ inline int64_t at(int k, int j, int i) const {
        return guard + (int64_t)k * plane + (int64_t)j * ldx + i;
    }
    __host__ __device__ inline int64_t npts() const { return (int64_t)nx * ny; }
    __host__ __device__ inline int64_t interior() const { return (int64_t)(nt + 1) * nx * ny; }
};

Geom make_geom(int dim, int nx, int ny, int nt);

// Spatial operator L = Lx (+) Ly on the device: per direction three coefficient rows
// (lo, di, up) stored contiguously: c[0..n) = lo, c[n..2n) = di, c[2n..3n) = up,
// (Lx v)_i = lo[i] v_{i-1} + di[i] v_i + up[i] v_{i+1}.
template <typename T>
struct SpaceOp {
    const T *x;
    const T *y;   // nullptr in 1D
};

// Time weights of a level: (A x)_0 = x_0, (A x)_k = (x_k - a L x_k) - (x_{k-1} + b L x_{k-1}).
struct Weights {
    double a, b, mu;
};

// ---------------------------------------------------------------------------------------
// Host-side numerics (setup.cpp).
// ---------------------------------------------------------------------------------------
struct Tri {               // host tridiagonal operator, lo/di/up of length n
    std::vector<double> lo, di, up;
    int n() const { return (int)di.size(); }
};

Tri fd_laplacian(int n, double tau);
Tri agglomerate(const Tri &L);                 // Y^T L Z for pair agglomeration (Sec. 3.2)
double tri_lambda_max_neg(const Tri &L);       // largest eigenvalue of -L
// Parallel cyclic reduction tables for M = I - a L:
//   nlev = ceil(log2 n); stride of level l is 2^l; alpha/gamma[l*npad + i]; binv[i].
int pcr_levels(int n);
void pcr_tables(const Tri &L, double a, int npad, std::vector<double> &alpha,
                std::vector<double> &gamma, std::vector<double> &binv);
// Tables of the partitioned (spike) slab solver for I - aL with P blocks of U rows.
int spike_levels(int P);
int spike_items(int U, int P);
void spike_tables(const Tri &L, double a, int U, int P, std::vector<double> &tab);
// Uniform operator test and tables of the sine-transform slab solver (slab_dst.cu).
bool tri_uniform(const Tri &L, double &c);
// tab = [alpha (n) | beta (n)], tw = FFT twiddles pass after pass (interleaved re, im)
void dst_tables(int n, double c, double a, double b, std::vector<double> &tab,
                std::vector<double> &tw);
// Diagonalisation L = S diag(lam) S^{-1} (real: L is similar to a symmetric matrix).
// S, Sinv row-major n x n.
void tri_eigen(const Tri &L, std::vector<double> &lam, std::vector<double> &S,
               std::vector<double> &Sinv);

// ---------------------------------------------------------------------------------------
// Launch bookkeeping and kernel-class timing.
//   count_launch(): one library kernel launched (or captured into a graph: captured
//   launches are counted once per replay of the graph).
//   prof_begin()/prof_end(): when profiling is on, a pair of CUDA events brackets the
//   launch on its stream (inside a captured graph the events become graph nodes); the
//   pair carries the kernel class, the level, the Arnoldi index j of the enclosing outer
//   iteration (-1 outside iterations) and the launch's algorithmic bytes.
// ---------------------------------------------------------------------------------------
extern int g_num_sms;
void count_launch(int n = 1);
void add_launches(int64_t n);   // n kernels of a replayed graph
void set_cuda_error(cudaError_t e);

enum ProfClass {
    PROF_RESTRICT = 0, PROF_INTERP, PROF_MULTIDOT, PROF_UPDATE, PROF_SLAB, PROF_RESIDUAL,
    PROF_COMBINE, PROF_MARCH, PROF_OTHER, PROF_INNER, PROF_NCLASS
};
struct ProfPair {
    cudaEvent_t a, b;
    int cls, level, j;
    double bytes;
};
bool prof_enabled();
void prof_begin(cudaStream_t s);
void prof_end(cudaStream_t s, int cls, double bytes);
void prof_set_context(int level, int j, double alg_n = 0.0);
double prof_alg_n();   // interior element count of the current level (0 = unknown)
// destination of the pairs recorded by this thread (nullptr: the transient list)
void prof_set_sink(std::vector<ProfPair> *sink);
// accumulate pairs whose outer iteration index j < j_limit (j = -1 always counts)
void prof_accumulate(const std::vector<ProfPair> &pairs, int j_limit);
void prof_accumulate_transient();
// while capturing, launches are counted into *c instead of the global counter
void set_capture_counter(int64_t *c);

// Two-stage deterministic reduction scratch: per-block partials + arrival counter.
struct ReduceScratch {
    double *partials;   // [slots][max_blocks]
    unsigned *counter;  // one counter per concurrent reduction site
    int max_blocks;
};

}  // namespace mk
