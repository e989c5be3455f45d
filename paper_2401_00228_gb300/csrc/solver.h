// Solver core of libmk (internal): the level hierarchy, the MK cycle and FGMRES.
#pragma once

#include <memory>
#include <vector>

#include "kernels.h"

namespace mk {

// Owning device allocation.
struct DevMem {
    void *p = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem &) = delete;
    DevMem &operator=(const DevMem &) = delete;
    ~DevMem() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t n) {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = n;
        cudaError_t e = cudaMalloc(&p, n > 0 ? n : 16);
        if (e == cudaSuccess) e = cudaMemset(p, 0, n > 0 ? n : 16);
        return e;
    }
    template <typename T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

struct OptsKey {
    int levels, n_cgs, mu_mode, precision, restart, orth, autotune, transfer, inner_kernel, augment;
    int nu[MK_MAX_LEVELS], space[MK_MAX_LEVELS], m_inner[MK_MAX_LEVELS];
    double mu_value;
    bool operator==(const OptsKey &o) const;
};

struct Level {
    Geom g;
    Weights w;
    Tri Lx, Ly;
    int nu = 1;        // coarsening factor to the next level
    bool space = false;
    int m = 0;         // restart (level 1) or fixed iterations (intermediate levels)
    bool coarsest = false;
    DevMem c64, c32;   // [3nx | 3ny] coefficients
    DevMem cdf;        // mixed level 1: double-float a*L then b*L, each [3nx | 3ny]
    DevMem cuni;       // mixed level 1 with uniform L: double-float (a cx, b cx, a cy, b cy)
    bool cuni_square = false;   // ... and cx == cy
    SpaceOp<double> op64{nullptr, nullptr};
    SpaceOp<float> op32{nullptr, nullptr};
    // vectors (level 1: V, W in FP64, X in the cycle precision; others in cycle precision)
    DevMem V, X, W;
    int64_t stride = 0;
    // FGMRES state
    DevMem ksd, ksf;
    KState ks{nullptr, nullptr, 0};
    // coarsest-level direct solver tables (cycle precision)
    DevMem R;          // coarsest right-hand side
    DevMem alpha, gamma, binv;
    int npad = 0, nlev = 0;
    DevMem spike;      // one-warp partitioned solver tables (1D), spikeU = rows per lane
    int spikeU = 0;
    DevMem dst, dsttw, dstbuf;   // sine-transform slab solver (1D uniform L, FP32 cycle)
    int dstN2 = 0, dstld = 0;
    // autotuned choices (0 = heuristic): tile depth of the restriction from / interpolation
    // on this level, and the coarsest solver (1 sine transform, 2 partitioned, 3 PCR)
    int kc_r = 0, kc_i = 0, coarse_kind = 0, coarse_kind_best = 0;
    int kr_bpsm = 0;   // blocks per SM of this level's small-basis Gram-Schmidt (0: default)
    DevMem Sx, Sxi, lamx, Sy, Syi, lamy;
    DevMem fdmbuf;     // 2D coarsest: transformed rows, (nt+1) nx ny in the cycle precision
};

struct Hierarchy {
    OptsKey key;
    int precision = 0;  // 0 FP64, 1 mixed
    std::vector<std::unique_ptr<Level>> lv;
    // MGRIT transfers (transfer = MK_TRANSFER_MGRIT): the fine-step march between coarse
    // points as decoupled slabs (fine a, b and L; n_T slabs of nu - 1 steps; R = phi xt_K on
    // each slab's first row, X = the marched points) and zt = Z xt on the fine geometry
    std::unique_ptr<Level> fprop;
    DevMem zt;
    // the inner levels in one cooperative kernel (inner_coop.cu): parameters in device
    // memory, grid size, and whether the cycle uses it
    bool coop_ok = false, use_coop = false;
    int coop_grid = 0, coop_bpsm = 2;
    DevMem coopP;
    DevMem f, u;        // level-1 right-hand side and iterate (FP64)
    DevMem partials, counters;
    ReduceScratch rs{nullptr, nullptr, 0};
    cudaGraphExec_t graph = nullptr;
    bool graph_profiled = false;        // captured with kernel-class timing events
    int64_t graph_kernels = 0;          // kernels in one replay of the graph
    std::vector<ProfPair> graph_pairs;  // timing events inside the graph
    // recycled corrections (mk_solve_opts.augment = aug_k > 0): ring of aug_k level-1 vectors
    // in the X precision, and the restart cycle whose last aug_k slots use them
    int aug_k = 0;
    DevMem aug;
    cudaGraphExec_t graph_aug = nullptr;
    bool graph_aug_profiled = false;
    int64_t graph_aug_kernels = 0;
    std::vector<ProfPair> graph_aug_pairs;
    int cycle_host = 0;                 // source of the cycle index's host-to-device copy
    double tol_host = 0.0;              // source of the tolerance's host-to-device copy
    ~Hierarchy();
};

struct Problem {
    int dim, nx, ny, nt;
    double theta, dt, tau;
    Geom g;                       // fine-level geometry
    DevMem fsrc;                  // padded FP64 source blocks f_k (k >= 1), block 0 zero
    bool has_source = false;
    std::unique_ptr<Hierarchy> H; // cached for the last options
    // march tables (fine level, FP64)
    bool march_ready = false;
    DevMem m_c64, m_alpha, m_gamma, m_binv;
    // 2D march: eigenvalues of L_x, L_y and, where n + 1 is not a power of two, the dense
    // sine matrices
    DevMem m_lamx, m_lamy, m_Sx, m_Sy;
    int m_npad = 0, m_nlev = 0;
    DevMem m_spike;
    int m_spikeU = 0;
    // 2D march by a sine-transform solve per step (FFT twiddles, scratch)
    double m_cx = 0.0, m_cy = 0.0;
    DevMem m_twx, m_twy, m_t1;
};

template <typename T>
inline SpaceOp<T> op_of(const Level &L);
template <>
inline SpaceOp<double> op_of<double>(const Level &L) { return L.op64; }
template <>
inline SpaceOp<float> op_of<float>(const Level &L) { return L.op32; }

mk_status build_hierarchy(Problem &P, const mk_solve_opts &o, Hierarchy *&out);
// A hierarchy owned by the caller (not cached in P).
mk_status build_hierarchy_new(Problem &P, const mk_solve_opts &o, std::unique_ptr<Hierarchy> &out);
// Time the tile depths of the 1D transfers on every level and the coarsest solver variants
// on this hierarchy's own buffers, and keep the fastest (a few ms; state is reset by a solve).
mk_status autotune_hierarchy(Hierarchy &H, cudaStream_t s);
// Sine-transform slab tables for coarsest level C when they apply (1D, L uniform, 2(n + 1) a
// power of two up to 4096; any slab length, n_cgs = 0 included); C.dstN2 stays 0 otherwise.
mk_status build_dst_tables(Level &C, int n_cgs);
mk_status validate_opts(const Problem &P, const mk_solve_opts &o);

// FGMRES + MK on f (padded FP64, level 1) -> H.u.  f is copied into H.f.
mk_status run_solve(Problem &P, Hierarchy &H, const mk_solve_opts &o, const double *f_padded,
                    mk_solve_info *info, cudaStream_t s);
// The part of run_solve before its restart loop: u = 0, flags, tolerance, r_0 = f.
mk_status solve_prepare(Hierarchy &H, const mk_solve_opts &o, cudaStream_t s);
// One CUDA graph whose replay runs one restart cycle of every hierarchy, each on its own
// branch (captured on streams[i]); kernels counts the graph's kernels.
mk_status capture_batch(std::vector<Problem *> &P, std::vector<Hierarchy *> &H,
                        std::vector<cudaStream_t> &streams, cudaGraphExec_t &graph,
                        int64_t &kernels);

// x_j = Q_l v_j, w = A_l x_j for basis slot j of level l (enqueue only).
void enqueue_cycle_step(Hierarchy &H, int l, int j, const int *done, cudaStream_t s);
void enqueue_coarsest(Hierarchy &H, const int *done, cudaStream_t s);

mk_status prepare_march(Problem &P);

// Allocation-free fine-level residual with a static-memory reduction scratch (noalloc.cu).
int64_t noalloc_partials_needed(const Problem &P);
mk_status residual_noalloc(const Problem &P, const double *f, const double *u, double *r,
                           double *rnorm, double *rnorm_steps, cudaStream_t s);

}  // namespace mk
