// Solver core: the level hierarchy (Sec. 3.2 Galerkin levels, Sec. 4 recursion), the MK
// cycle of substeps 4.1-4.5, inner fixed-iteration FGMRES on intermediate levels
// (Sec. 4.1/4.2), the decoupled coarsest level (Sec. 3.3.2) and the outer FGMRES of
// Algorithm 2 with restarts.  Everything between host synchronisations is a fixed
// sequence of kernel launches on one stream, captured once per hierarchy into a CUDA
// graph that runs one restart cycle; convergence is decided on the device and the
// remaining kernels of a converged cycle return immediately.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "df64.cuh"
#include <type_traits>

#include "solver.h"

namespace mk {

int64_t launches_total();

bool OptsKey::operator==(const OptsKey &o) const {
    if (levels != o.levels || n_cgs != o.n_cgs || mu_mode != o.mu_mode ||
        precision != o.precision || restart != o.restart || mu_value != o.mu_value || orth != o.orth ||
        autotune != o.autotune || transfer != o.transfer || inner_kernel != o.inner_kernel ||
        augment != o.augment)
        return false;
    for (int i = 0; i < MK_MAX_LEVELS; ++i)
        if (nu[i] != o.nu[i] || space[i] != o.space[i] || m_inner[i] != o.m_inner[i]) return false;
    return true;
}

static OptsKey make_key(const mk_solve_opts &o) {
    OptsKey k;
    std::memset(&k, 0, sizeof(k));
    k.levels = o.levels;
    k.n_cgs = o.n_cgs;
    k.mu_mode = o.mu_mode;
    k.precision = o.precision;
    k.restart = o.restart;
    k.orth = o.orth;
    k.autotune = o.autotune ? 1 : 0;
    k.transfer = o.transfer;
    k.inner_kernel = o.inner_kernel;
    k.augment = o.augment;
    k.mu_value = o.mu_mode == 2 ? o.mu_value : 0.0;
    for (int i = 0; i < o.levels - 1 && i < MK_MAX_LEVELS; ++i) {
        k.nu[i] = o.nu[i];
        k.space[i] = o.space[i] ? 1 : 0;
    }
    for (int i = 0; i < o.levels - 2 && i < MK_MAX_LEVELS; ++i) k.m_inner[i] = o.m_inner[i];
    return k;
}

mk_status validate_opts(const Problem &P, const mk_solve_opts &o) {
    if (!(o.tol > 0.0) || o.restart < 1 || o.restart > MK_MAX_RESTART || o.max_iters < 1)
        return MK_ERR_INVALID;
    if (o.levels < 2 || o.levels > MK_MAX_LEVELS) return MK_ERR_INVALID;
    if (o.precision < 0 || o.precision > 2) return MK_ERR_INVALID;
    if (o.mu_mode < 0 || o.mu_mode > 2) return MK_ERR_INVALID;
    if (o.orth < 0 || o.orth > 2) return MK_ERR_INVALID;
    if (o.n_cgs < 0) return MK_ERR_INVALID;
    if (o.transfer != MK_TRANSFER_MK && o.transfer != MK_TRANSFER_MGRIT) return MK_ERR_INVALID;
    if (o.inner_kernel < MK_INNER_AUTO || o.inner_kernel > MK_INNER_COOP) return MK_ERR_INVALID;
    if (o.augment < 0 || o.augment > MK_MAX_AUGMENT || o.augment >= o.restart) return MK_ERR_INVALID;
    if (o.transfer == MK_TRANSFER_MGRIT &&
        (P.dim != 1 || o.levels != 2 || o.space[0] != 0 || o.nu[0] < 2 ||
         P.nt % o.nu[0] != 0 || P.nt / o.nu[0] > 65535))
        return MK_ERR_INVALID;
    int nt = P.nt, nx = P.nx, ny = P.dim == 2 ? P.ny : 1;
    for (int l = 0; l < o.levels - 1; ++l) {
        if (o.nu[l] < 1) return MK_ERR_INVALID;
        if (nt % o.nu[l]) return MK_ERR_INVALID;
        nt /= o.nu[l];
        if (o.space[l]) {
            if (nx < 2 || (P.dim == 2 && ny < 2)) return MK_ERR_INVALID;
            nx = (nx + 1) / 2;
            if (P.dim == 2) ny = (ny + 1) / 2;
        }
    }
    for (int l = 0; l < o.levels - 2; ++l)
        if (o.m_inner[l] < 1 || o.m_inner[l] > MK_MAX_INNER) return MK_ERR_INVALID;
    if (o.n_cgs > 0 && nt % o.n_cgs) return MK_ERR_INVALID;
    if (nt < 1) return MK_ERR_INVALID;
    if (P.dim == 1 && nx > 4096) return MK_ERR_INVALID;
    // 2D coarsest: fast diagonalisation in one CTA's shared memory
    const int lim2d = o.precision == 0 ? 48 : 64;
    if (P.dim == 2 && (nx > lim2d || ny > lim2d)) return MK_ERR_INVALID;
    return MK_OK;
}

#define MKCK(call)                                         \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) {                           \
            set_cuda_error(e_);                            \
            return e_ == cudaErrorMemoryAllocation ? MK_ERR_NOMEM : MK_ERR_CUDA; \
        }                                                  \
    } while (0)

template <typename T>
static cudaError_t upload(DevMem &m, const std::vector<double> &h) {
    std::vector<T> t(h.begin(), h.end());
    cudaError_t e = m.alloc(sizeof(T) * (t.empty() ? 1 : t.size()));
    if (e != cudaSuccess) return e;
    if (!t.empty()) e = cudaMemcpy(m.p, t.data(), sizeof(T) * t.size(), cudaMemcpyHostToDevice);
    return e;
}

static std::vector<double> coef_concat(const Tri &Lx, const Tri *Ly) {
    std::vector<double> c;
    c.insert(c.end(), Lx.lo.begin(), Lx.lo.end());
    c.insert(c.end(), Lx.di.begin(), Lx.di.end());
    c.insert(c.end(), Lx.up.begin(), Lx.up.end());
    if (Ly) {
        c.insert(c.end(), Ly->lo.begin(), Ly->lo.end());
        c.insert(c.end(), Ly->di.begin(), Ly->di.end());
        c.insert(c.end(), Ly->up.begin(), Ly->up.end());
    }
    return c;
}

static mk_status upload_coefs(Level &L, int dim) {
    std::vector<double> c = coef_concat(L.Lx, dim == 2 ? &L.Ly : nullptr);
    MKCK(upload<double>(L.c64, c));
    MKCK(upload<float>(L.c32, c));
    L.op64.x = L.c64.as<double>();
    L.op64.y = dim == 2 ? L.c64.as<double>() + 3 * L.Lx.n() : nullptr;
    L.op32.x = L.c32.as<float>();
    L.op32.y = dim == 2 ? L.c32.as<float>() + 3 * L.Lx.n() : nullptr;
    return MK_OK;
}

static mk_status alloc_kstate(Level &L, int m) {
    MKCK(L.ksd.alloc(sizeof(double) * KState::ndoubles(m)));
    MKCK(L.ksf.alloc(sizeof(int) * 8));
    L.ks.d = L.ksd.as<double>();
    L.ks.flags = L.ksf.as<int>();
    L.ks.m = m;
    return MK_OK;
}

mk_status build_dst_tables(Level &C, int n_cgs) {
    C.dstN2 = 0;
    if (C.g.dim != 1 || n_cgs < 0 || (n_cgs > 0 && C.g.nt % n_cgs != 0)) return MK_OK;
    const int n = C.g.nx;
    const int N2 = dst_transform_size(n);
    double c = 0.0;
    if (N2 == 0 || !tri_uniform(C.Lx, c)) return MK_OK;
    std::vector<double> tab, tw;
    dst_tables(n, c, C.w.a, C.w.b, tab, tw);
    MKCK(upload<float>(C.dst, tab));
    MKCK(upload<float>(C.dsttw, tw));
    C.dstld = ((n + 31) / 32) * 32;
    MKCK(C.dstbuf.alloc(sizeof(float) * (size_t)(C.g.nt + 1) * C.dstld));
    C.dstN2 = N2;
    return MK_OK;
}

// Coarsest-level direct solver tables.
static mk_status build_coarsest_tables(Level &C, int dim, bool fp64, int n_cgs) {
    if (dim == 1) {
        int n = C.Lx.n();
        int np = 32;
        while (np < n) np *= 2;
        C.npad = np;
        C.nlev = pcr_levels(n);
        std::vector<double> al, ga, bi;
        pcr_tables(C.Lx, C.w.a, np, al, ga, bi);
        if (al.empty()) {
            al.assign(np, 0.0);
            ga.assign(np, 0.0);
        }
        if (fp64) {
            MKCK(upload<double>(C.alpha, al));
            MKCK(upload<double>(C.gamma, ga));
            MKCK(upload<double>(C.binv, bi));
        } else {
            MKCK(upload<float>(C.alpha, al));
            MKCK(upload<float>(C.gamma, ga));
            MKCK(upload<float>(C.binv, bi));
        }
        // one-warp partitioned solver where the block per lane fits in registers
        if (fp64 ? slab_warp_supported<double>(n) : slab_warp_supported<float>(n)) {
            C.spikeU = spike_block_size(n);
            std::vector<double> tab;
            spike_tables(C.Lx, C.w.a, C.spikeU, spike_threads(n), tab);
            if (fp64) MKCK(upload<double>(C.spike, tab));
            else MKCK(upload<float>(C.spike, tab));
        }
        if (!fp64) {
            mk_status st = build_dst_tables(C, n_cgs);
            if (st != MK_OK) return st;
        }
    } else {
        std::vector<double> lx, Sx, Sxi, ly, Sy, Syi;
        tri_eigen(C.Lx, lx, Sx, Sxi);
        tri_eigen(C.Ly, ly, Sy, Syi);
        MKCK(C.fdmbuf.alloc((fp64 ? sizeof(double) : sizeof(float)) * (size_t)(C.g.nt + 1) *
                            C.g.nx * C.g.ny));
        if (fp64) {
            MKCK(upload<double>(C.Sx, Sx));
            MKCK(upload<double>(C.Sxi, Sxi));
            MKCK(upload<double>(C.lamx, lx));
            MKCK(upload<double>(C.Sy, Sy));
            MKCK(upload<double>(C.Syi, Syi));
            MKCK(upload<double>(C.lamy, ly));
        } else {
            MKCK(upload<float>(C.Sx, Sx));
            MKCK(upload<float>(C.Sxi, Sxi));
            MKCK(upload<float>(C.lamx, lx));
            MKCK(upload<float>(C.Sy, Sy));
            MKCK(upload<float>(C.Syi, Syi));
            MKCK(upload<float>(C.lamy, ly));
        }
    }
    return MK_OK;
}

// Whether the inner levels can run as one cooperative kernel (1D, mixed, time coarsening by
// 2 without space below level 2, sine-transform coarsest solver, co-residency possible).
static bool coop_eligible(const Hierarchy &H, const mk_solve_opts &o) {
    const int L = (int)H.lv.size();
    if (H.precision != 1 || o.transfer != MK_TRANSFER_MK || L < 3) return false;
    if (H.lv[0]->g.dim != 1) return false;
    for (int l = 1; l + 1 < L; ++l)
        if (H.lv[l]->nu != 2 || H.lv[l]->space) return false;
    const Level &C = *H.lv.back();
    return C.dstN2 > 0 && coop_grid_size(C.dstN2) > 0;
}

// Parameters of the cooperative kernel for a grid of bpsm blocks per SM (device copy).
mk_status coop_configure(Hierarchy &H, int bpsm) {
    const Level &C = *H.lv.back();
    const int cap = coop_grid_size(C.dstN2);
    int grid = g_num_sms * bpsm;
    if (grid > cap) grid = cap;
    if (grid < 1) return MK_ERR_INVALID;
    CoopParams cp;
    std::memset(&cp, 0, sizeof(cp));
    const int L = (int)H.lv.size();
    cp.nl = L - 2;
    for (int l = 1; l + 1 < L; ++l) {
        const Level &Lv = *H.lv[l];
        CoopLevel &c = cp.lv[l - 1];
        c.g = Lv.g;
        c.a = (float)Lv.w.a;
        c.b = (float)Lv.w.b;
        c.mu = (float)Lv.w.mu;
        c.L = Lv.c32.as<float>();
        c.V = Lv.V.as<float>();
        c.X = Lv.X.as<float>();
        c.W = Lv.W.as<float>();
        c.stride = Lv.stride;
        c.m = Lv.m;
        c.ks = Lv.ks;
    }
    int logN2 = 0;
    while ((1 << logN2) < C.dstN2) ++logN2;
    cp.c.g = C.g;
    cp.c.tab = C.dst.as<float>();
    cp.c.tw = C.dsttw.as<float2>();
    cp.c.N2 = C.dstN2;
    cp.c.logN2 = logN2;
    cp.c.ldd = C.dstld;
    cp.c.n_cgs = H.key.n_cgs;
    cp.c.rh = C.dstbuf.as<float>();
    cp.c.R = C.R.as<float>();
    cp.c.X = C.X.as<float>();
    cp.partials = H.partials.as<double>();
    cp.max_blocks = grid;
    if (!H.coopP.p) MKCK(H.coopP.alloc(sizeof(CoopParams)));
    MKCK(cudaMemcpy(H.coopP.p, &cp, sizeof(cp), cudaMemcpyHostToDevice));
    H.coop_grid = grid;
    H.coop_bpsm = bpsm;
    return MK_OK;
}

mk_status build_hierarchy(Problem &P, const mk_solve_opts &o, Hierarchy *&out) {
    OptsKey key = make_key(o);
    if (P.H && P.H->key == key) {
        out = P.H.get();
        return MK_OK;
    }
    P.H.reset();
    std::unique_ptr<Hierarchy> H;
    mk_status st = build_hierarchy_new(P, o, H);
    if (st != MK_OK) return st;
    if (o.autotune) {
        st = autotune_hierarchy(*H, nullptr);
        if (st != MK_OK) return st;
        MKCK(cudaStreamSynchronize(nullptr));
    }
    P.H = std::move(H);
    out = P.H.get();
    return MK_OK;
}

mk_status build_hierarchy_new(Problem &P, const mk_solve_opts &o, std::unique_ptr<Hierarchy> &out) {
    OptsKey key = make_key(o);
    std::unique_ptr<Hierarchy> H(new Hierarchy());
    H->key = key;
    H->precision = o.precision;
    const bool fp64 = o.precision == 0;
    const size_t cs = fp64 ? sizeof(double) : sizeof(float);
    const int L = o.levels;
    for (int l = 0; l < L; ++l) {
        std::unique_ptr<Level> lv(new Level());
        if (l == 0) {
            lv->Lx = fd_laplacian(P.nx, P.tau);
            if (P.dim == 2) lv->Ly = fd_laplacian(P.ny, P.tau);
            lv->w.a = P.theta * P.dt;
            lv->w.b = (1.0 - P.theta) * P.dt;
            lv->g = P.g;
        } else {
            Level &pv = *H->lv[l - 1];
            int nu = o.nu[l - 1];
            bool sp = o.space[l - 1] != 0;
            lv->Lx = sp ? agglomerate(pv.Lx) : pv.Lx;
            if (P.dim == 2) lv->Ly = sp ? agglomerate(pv.Ly) : pv.Ly;
            if (o.transfer == MK_TRANSFER_MGRIT) {
                // non-Galerkin coarse matrix of Eq. (coarsemat): the theta-scheme with the same
                // theta and step nu dt (Psi_n, Phi_n of Eq. (timemarchdT))
                lv->w.a = P.theta * nu * P.dt;
                lv->w.b = (1.0 - P.theta) * nu * P.dt;
            } else {
                // Galerkin coarse operator as a theta-scheme with a larger step (Eqs.
                // (timecoarse1)-(timecoarse3), literal product nu psi - (nu-1) phi)
                lv->w.a = nu * pv.w.a + (nu - 1) * pv.w.b;
                lv->w.b = pv.w.b;
            }
            lv->g = make_geom(P.dim, lv->Lx.n(), P.dim == 2 ? lv->Ly.n() : 1, pv.g.nt / nu);
        }
        if (l < L - 1) {
            lv->nu = o.nu[l];
            lv->space = o.space[l] != 0;
        }
        lv->coarsest = (l == L - 1);
        // shift mu_l = lambda_max(A_l) (Sec. 3.1), or 1, or a given value
        double lam = tri_lambda_max_neg(lv->Lx);
        if (P.dim == 2) lam += tri_lambda_max_neg(lv->Ly);
        if (o.mu_mode == 0) lv->w.mu = std::max(1.0, 1.0 + lv->w.a * lam);
        else if (o.mu_mode == 1) lv->w.mu = 1.0;
        else lv->w.mu = o.mu_value;
        mk_status st = upload_coefs(*lv, P.dim);
        if (st == MK_OK && l == 0 && o.precision == 1) {
            // double-float a*L and b*L rows for the level-1 matvec of the mixed solve
            std::vector<double> c = coef_concat(lv->Lx, P.dim == 2 ? &lv->Ly : nullptr);
            std::vector<float2> t;
            for (double v : c) t.push_back(df_pack_host(lv->w.a * v));
            for (double v : c) t.push_back(df_pack_host(lv->w.b * v));
            MKCK(lv->cdf.alloc(sizeof(float2) * t.size()));
            MKCK(cudaMemcpy(lv->cdf.p, t.data(), sizeof(float2) * t.size(), cudaMemcpyHostToDevice));
            // uniform operator: (a cx, b cx, a cy, b cy) for the exact-stencil kernels
            double cx = 0.0, cy = 0.0;
            if (tri_uniform(lv->Lx, cx) && (P.dim == 1 || tri_uniform(lv->Ly, cy))) {
                const float2 u[4] = {df_pack_host(lv->w.a * cx), df_pack_host(lv->w.b * cx),
                                     df_pack_host(lv->w.a * cy), df_pack_host(lv->w.b * cy)};
                MKCK(lv->cuni.alloc(sizeof(u)));
                MKCK(cudaMemcpy(lv->cuni.p, u, sizeof(u), cudaMemcpyHostToDevice));
                lv->cuni_square = P.dim == 2 && cx == cy;
            }
        }
        if (st != MK_OK) return st;
        lv->stride = lv->g.len;
        const size_t len = (size_t)lv->g.len;
        if (l == 0) {
            lv->m = o.restart;
            // level-1 basis: FP64 or double-float pairs (8 bytes), FP32 with precision 2
            const size_t vs = o.precision == 2 ? sizeof(float) : sizeof(double);
            MKCK(lv->V.alloc(vs * len * (lv->m + 1)));
            MKCK(lv->X.alloc(cs * len * lv->m));
            if (o.augment > 0) {
                MKCK(H->aug.alloc(cs * len * o.augment));
                H->aug_k = o.augment;
            }
            MKCK(lv->W.alloc(vs * len));
            st = alloc_kstate(*lv, lv->m);
            if (st != MK_OK) return st;
        } else if (l < L - 1) {
            lv->m = o.m_inner[l - 1];
            MKCK(lv->V.alloc(cs * len * (lv->m + 1)));
            MKCK(lv->X.alloc(cs * len * lv->m));
            MKCK(lv->W.alloc(cs * len));
            st = alloc_kstate(*lv, lv->m);
            if (st != MK_OK) return st;
        } else {
            lv->m = 1;
            MKCK(lv->R.alloc(cs * len));
            MKCK(lv->X.alloc(cs * len));
            st = build_coarsest_tables(*lv, P.dim, fp64, o.n_cgs);
            if (st != MK_OK) return st;
        }
        H->lv.push_back(std::move(lv));
    }
    if (o.transfer == MK_TRANSFER_MGRIT) {
        // ideal interpolation: the fine steps of every coarse interval as one decoupled slab
        const Level &F0 = *H->lv[0];
        const int nu = o.nu[0], nT = P.nt / nu;
        std::unique_ptr<Level> fp(new Level());
        fp->Lx = F0.Lx;
        fp->w = F0.w;
        fp->g = make_geom(1, P.nx, 1, nT * (nu - 1));
        fp->coarsest = true;
        mk_status st = upload_coefs(*fp, 1);
        if (st != MK_OK) return st;
        MKCK(fp->R.alloc(cs * (size_t)fp->g.len));
        MKCK(fp->X.alloc(cs * (size_t)fp->g.len));
        st = build_coarsest_tables(*fp, 1, fp64, nT);
        if (st != MK_OK) return st;
        H->fprop = std::move(fp);
        MKCK(H->zt.alloc(cs * (size_t)F0.g.len));
    }
    const size_t len0 = (size_t)P.g.len;
    MKCK(H->f.alloc(sizeof(double) * len0));
    MKCK(H->u.alloc(sizeof(double) * len0));
    H->rs.max_blocks = 65536;
    MKCK(H->partials.alloc(sizeof(double) * (size_t)H->rs.max_blocks *
                           (std::max(o.restart, MK_MAX_INNER) + 4)));
    MKCK(H->counters.alloc(sizeof(unsigned) * 16));
    H->rs.partials = H->partials.as<double>();
    H->rs.counter = H->counters.as<unsigned>();
    H->coop_ok = coop_eligible(*H, o);
    if (o.inner_kernel == MK_INNER_COOP && !H->coop_ok) return MK_ERR_INVALID;
    // MK_INNER_COOP: the cooperative kernel; MK_INNER_AUTO: separate launches (measured faster)
    if (H->coop_ok && o.inner_kernel == MK_INNER_COOP) {
        mk_status st = coop_configure(*H, 3);
        if (st != MK_OK) return st;
        H->use_coop = true;
    }
    out = std::move(H);
    return MK_OK;
}

// ---------------------------------------------------------------------------------------
// MK cycle (enqueue only)
// ---------------------------------------------------------------------------------------
// Decoupled slab solve on level C (n_cgs slabs; 0 = one coupled march).
template <typename Tc>
static void enqueue_slabs_t(Level &C, int n_cgs, const int *done, cudaStream_t s) {
    const int kind = C.coarse_kind;   // 0: sine transform, else partitioned, else PCR
    if constexpr (std::is_same<Tc, float>::value) {
        if (C.dstN2 > 0 && (kind == 0 || kind == 1)) {
            launch_slab_1d_dst(C.g, C.dst.as<float>(), C.dsttw.as<float2>(), C.dstN2, n_cgs,
                               C.dstbuf.as<float>(), C.dstld, C.R.as<float>(), C.X.as<float>(),
                               done, s);
            return;
        }
    }
    if (C.g.dim == 1 && C.spikeU > 0 && kind != 3)
        launch_slab_1d_warp<Tc>(C.g, C.w.b, C.spike.as<Tc>(), C.spikeU, n_cgs, C.R.as<Tc>(),
                                C.X.as<Tc>(), done, s, PROF_SLAB);
    else if (C.g.dim == 1)
        launch_slab_1d<Tc>(C.g, C.w.b, op_of<Tc>(C), C.alpha.as<Tc>(), C.gamma.as<Tc>(),
                           C.binv.as<Tc>(), C.npad, C.nlev, n_cgs, C.R.as<Tc>(), C.X.as<Tc>(),
                           done, s);
    else
        launch_slab_2d_fdm<Tc>(C.g, C.w.a, C.w.b, C.Sx.as<Tc>(), C.Sxi.as<Tc>(), C.lamx.as<Tc>(),
                               C.Sy.as<Tc>(), C.Syi.as<Tc>(), C.lamy.as<Tc>(), n_cgs,
                               C.fdmbuf.as<Tc>(), C.R.as<Tc>(), C.X.as<Tc>(), done, s);
}

template <typename Tc>
void enqueue_coarsest_t(Hierarchy &H, const int *done, cudaStream_t s) {
    enqueue_slabs_t<Tc>(*H.lv.back(), H.key.n_cgs, done, s);
}

void enqueue_coarsest(Hierarchy &H, const int *done, cudaStream_t s) {
    if (H.precision == 0) enqueue_coarsest_t<double>(H, done, s);
    else enqueue_coarsest_t<float>(H, done, s);
}

template <typename Tc>
static void enqueue_inner_solve(Hierarchy &H, int l, const int *done, cudaStream_t s);

// x_j = Q_l v_j and w = A_l x_j; Tv = type of level l's basis, Tx = type of its X,
// Tw/Tcw = type and arithmetic of w.
// Index of the outer FGMRES iteration being enqueued (-1 outside iterations); every kernel
// launched for it, on any level, is attributed to it by the kernel-class timing.
static thread_local int t_outer_j = -1;

static void set_ctx(const Level &L, int level) {
    prof_set_context(level + 1, t_outer_j, (double)L.g.interior());
    set_tile_hint(L.kc_r, L.kc_i);
    set_krylov_hint(L.kr_bpsm);
}

// x_j = sigma_j V_j - Z vt and w = A x_j (K4).  Level 1 of the mixed solve keeps V and w as
// double-float pairs and evaluates w in double-float arithmetic.
// gc, nu, space, cstride: geometry, coarsening and stride of the vectors Xc that Z acts on
// (the next level's, or the fine geometry with nu = 1 when Z has been applied already).
template <typename Tv, typename Tc, typename Tx, typename Tw, typename Tcw>
struct InterpStep {
    static void run(Level &L, const Geom &gc, int nu, bool space, int64_t cstride, const Tv *vj,
                    const double *sig, const Tc *Xc, int mc, const double *yc, int j,
                    const int *done, cudaStream_t s) {
        launch_interp<Tv, Tc, Tx, Tw, Tcw>(L.g, gc, nu, space, L.w, op_of<Tcw>(L), vj, sig, Xc,
                                           mc, cstride, yc, L.X.as<Tx>() + (int64_t)j * L.stride,
                                           L.W.as<Tw>(), done, s);
    }
};
template <>
struct InterpStep<float2, float, float, float2, double> {
    static void run(Level &L, const Geom &gc, int nu, bool space, int64_t cstride,
                    const float2 *vj, const double *sig, const float *Xc, int mc,
                    const double *yc, int j, const int *done, cudaStream_t s) {
        const int64_t nc = 3 * (int64_t)L.g.nx + (L.g.dim == 2 ? 3 * (int64_t)L.g.ny : 0);
        const float2 *ca = L.cdf.as<float2>();
        launch_interp_df(L.g, gc, nu, space, ca, ca + nc, L.w.b != 0.0, vj, sig, Xc, mc,
                         cstride, yc, L.X.as<float>() + (int64_t)j * L.stride, L.W.as<float2>(),
                         done, s, L.cuni.p ? L.cuni.as<float2>() : nullptr, L.cuni_square);
    }
};
template <typename Tv, typename Tc, typename Tx, typename Tw, typename Tcw>
static void interp_step(Level &L, Level &C, const Tv *vj, const double *sig, const Tc *Xc, int mc,
                        const double *yc, int j, const int *done, cudaStream_t s) {
    InterpStep<Tv, Tc, Tx, Tw, Tcw>::run(L, C.g, L.nu, L.space, C.stride, vj, sig, Xc, mc, yc, j,
                                         done, s);
}

// Substeps 4.1-4.5 with the MGRIT transfers (two levels, 1D): injection of the shifted
// residual at the coarse points, the coarse theta-scheme solve, the ideal interpolation
// (phi xt_K on the first fine step of every interval, the decoupled march of the interval's
// nu - 1 fine steps, gather), then x = sigma v - Z xt and w = A x by the interpolation kernel
// with nu = 1 on the gathered vector.
template <typename Tc, typename Tv, typename Tx, typename Tw, typename Tcw>
static void mgrit_step_t(Hierarchy &H, int j, const Tv *vj, const double *sig, const int *done,
                         cudaStream_t s) {
    Level &L = *H.lv[0];
    Level &C = *H.lv[1];
    Level &F = *H.fprop;
    set_ctx(L, 0);
    launch_inject_restrict_1d<Tv, Tc>(L.g, C.g, L.nu, L.w, op_of<Tc>(L), vj, sig, C.R.as<Tc>(),
                                      done, s);                          // 4.1-4.2, Eq. (mgritY)
    set_ctx(C, 1);
    enqueue_coarsest_t<Tc>(H, done, s);                                  // 4.3, Eq. (coarsemat)
    set_ctx(L, 0);
    launch_ideal_interp_rhs_1d<Tc>(C.g, F.g, L.nu, L.w.b, op_of<Tc>(L), C.X.as<Tc>(),
                                   F.R.as<Tc>(), done, s);               // 4.4, Eq. (mgritZ)
    enqueue_slabs_t<Tc>(F, C.g.nt, done, s);
    launch_ideal_interp_gather_1d<Tc>(L.g, C.g, F.g, L.nu, C.X.as<Tc>(), F.X.as<Tc>(),
                                      H.zt.as<Tc>(), done, s);
    InterpStep<Tv, Tc, Tx, Tw, Tcw>::run(L, L.g, 1, false, L.stride, vj, sig, H.zt.as<Tc>(), 1,
                                         nullptr, j, done, s);           // 4.5 and step 5
}

template <typename Tc, typename Tv, typename Tx, typename Tw, typename Tcw>
static void cycle_step_t(Hierarchy &H, int l, int j, const int *done, cudaStream_t s) {
    Level &L = *H.lv[l];
    Level &C = *H.lv[l + 1];
    const Tv *vj = L.V.as<Tv>() + (int64_t)j * L.stride;
    const double *sig = L.ks.sigma() + j;
    if (H.fprop && l == 0) {   // MGRIT transfers: two levels only
        mgrit_step_t<Tc, Tv, Tx, Tw, Tcw>(H, j, vj, sig, done, s);
        return;
    }
    // 4.1-4.2: restriction of the shifted residual of the basis vector
    set_ctx(L, l);
    if (C.coarsest) {
        launch_restrict<Tv, Tc, Tc>(L.g, C.g, L.nu, L.space, L.w, op_of<Tc>(L), vj, sig,
                                    C.R.as<Tc>(), H.rs, 0, KState{nullptr, nullptr, 0}, done, s);
        set_ctx(C, l + 1);
        enqueue_coarsest_t<Tc>(H, done, s);                          // 4.3 (decoupled slabs)
    } else {
        launch_restrict<Tv, Tc, Tc>(L.g, C.g, L.nu, L.space, L.w, op_of<Tc>(L), vj, sig,
                                    C.V.as<Tc>(), H.rs, 0, C.ks, done, s);
        if (l == 0 && H.use_coop) {                                  // 4.3, one cooperative kernel
            set_ctx(C, l + 1);
            launch_inner_coop(H.coopP.as<CoopParams>(), H.lv.back()->dstN2, H.coop_grid, done, s);
        } else {
            enqueue_inner_solve<Tc>(H, l + 1, done, s);              // 4.3 (recursion)
        }
    }
    // 4.4-4.5 and step 5: x = v - Z vt, w = A x
    set_ctx(L, l);
    const Tc *Xc = C.X.as<Tc>();
    const double *yc = C.coarsest ? nullptr : C.ks.y();
    int mc = C.coarsest ? 1 : C.m;
    interp_step<Tv, Tc, Tx, Tw, Tcw>(L, C, vj, sig, Xc, mc, yc, j, done, s);
}

template <typename Tc>
static void enqueue_inner_solve(Hierarchy &H, int l, const int *done, cudaStream_t s) {
    Level &L = *H.lv[l];
    const int64_t len = L.g.len;
    for (int j = 0; j < L.m; ++j) {
        cycle_step_t<Tc, Tc, Tc, Tc, Tc>(H, l, j, done, s);
        set_ctx(L, l);
        if (j < L.m - 1) {
            launch_multidot<Tc, Tc>(len, L.W.as<Tc>(), L.V.as<Tc>(), L.stride, j, H.rs, L.ks, false,
                                    done, s);
            launch_update<Tc, Tc>(len, L.W.as<Tc>(), L.V.as<Tc>(), L.stride, j, true, H.rs, L.ks,
                                  UPD_INNER, false, done, s);
        } else {
            // last iteration: V_m is not needed; its norm by Pythagoras, least squares in the
            // same kernel
            launch_multidot<Tc, Tc>(len, L.W.as<Tc>(), L.V.as<Tc>(), L.stride, j, H.rs, L.ks, false,
                                    done, s, UPD_INNER);
        }
    }
}

void enqueue_cycle_step(Hierarchy &H, int l, int j, const int *done, cudaStream_t s) {
    if (H.precision == 0) {
        cycle_step_t<double, double, double, double, double>(H, l, j, done, s);
    } else if (l == 0 && H.precision == 1) {
        cycle_step_t<float, float2, float, float2, double>(H, l, j, done, s);
    } else {
        cycle_step_t<float, float, float, float, float>(H, l, j, done, s);
    }
}

// One restart cycle of the outer FGMRES (Algorithm 2), ending with the true residual of
// the updated iterate, which also starts the next cycle.
// With aug (recycled corrections in use): the last H.aug_k slots take x_j = the stored
// correction of an earlier cycle and w = A x_j (FP64, then double-float pairs in the mixed
// solve) instead of x_j = Q_1 v_j; the Gram-Schmidt and least squares are the same.
static void enqueue_outer_cycle(Problem &P, Hierarchy &H, cudaStream_t s, bool aug = false) {
    Level &L = *H.lv[0];
    const int *done = L.ks.flags;
    const int64_t len = L.g.len;
    const bool fp64 = H.precision == 0;
    const bool sp = H.precision == 2;   // FP32 level-1 basis
    const size_t xs = fp64 ? sizeof(double) : sizeof(float);
    double *V = L.V.as<double>();
    double *W = L.W.as<double>();
    float2 *Vd = L.V.as<float2>();
    float2 *Wd = L.W.as<float2>();
    float *Vf = L.V.as<float>();
    float *Wf = L.W.as<float>();
    for (int j = 0; j < L.m; ++j) {
        t_outer_j = j;
        const int q = j - (L.m - H.aug_k);
        if (aug && q >= 0) {
            set_ctx(L, 0);
            char *xj = L.X.as<char>() + (size_t)j * L.stride * xs;
            const char *dq = H.aug.as<char>() + (size_t)q * L.stride * xs;
            cudaMemcpyAsync(xj, dq, (size_t)len * xs, cudaMemcpyDeviceToDevice, s);
            if (fp64) {
                launch_apply<double, double, double>(L.g, L.w, L.op64, reinterpret_cast<double *>(xj), W, s);
            } else if (sp) {
                launch_apply<float, float, float>(L.g, L.w, L.op32, reinterpret_cast<float *>(xj), Wf, s);
            } else {
                launch_apply<float, double, double>(L.g, L.w, L.op64, reinterpret_cast<float *>(xj), W, s);
                launch_f64_to_df(len, W, done, s);
            }
        } else {
            enqueue_cycle_step(H, 0, j, done, s);
        }
        set_ctx(L, 0);
        const int orth = H.key.orth;
        const int mode = orth == 0 ? UPD_GIVENS : (orth == 2 ? UPD_GIVENS | UPD_REORTH_ALWAYS : UPD_OUTER);
        if (fp64) {
            launch_multidot<double, double>(len, W, V, L.stride, j, H.rs, L.ks, false, done, s);
            launch_update<double, double>(len, W, V, L.stride, j, true, H.rs, L.ks, mode, false, done,
                                          s);
        } else if (sp) {
            launch_multidot<float, float>(len, Wf, Vf, L.stride, j, H.rs, L.ks, false, done, s);
            launch_update<float, float>(len, Wf, Vf, L.stride, j, true, H.rs, L.ks, mode, false, done,
                                        s);
        } else {
            launch_multidot_df(len, Wd, Vd, L.stride, j, H.rs, L.ks, false, done, s);
            launch_update_df(len, Wd, Vd, L.stride, j, H.rs, L.ks, mode, false, done, s);
        }
        if (orth != 0) {
            if (fp64) {
                launch_multidot<double, double>(len, W, V, L.stride, j, H.rs, L.ks, true, done, s);
                launch_update<double, double>(len, W, V, L.stride, j, true, H.rs, L.ks, UPD_GIVENS,
                                              true, done, s);
            } else if (sp) {
                launch_multidot<float, float>(len, Wf, Vf, L.stride, j, H.rs, L.ks, true, done, s);
                launch_update<float, float>(len, Wf, Vf, L.stride, j, true, H.rs, L.ks, UPD_GIVENS,
                                            true, done, s);
            } else {
                launch_multidot_df(len, Wd, Vd, L.stride, j, H.rs, L.ks, true, done, s);
                launch_update_df(len, Wd, Vd, L.stride, j, H.rs, L.ks, UPD_GIVENS, true, done, s);
            }
        }
    }
    t_outer_j = -1;
    set_ctx(L, 0);
    if (fp64) {
        launch_combine<double>(len, H.u.as<double>(), L.X.as<double>(), L.stride, L.ks, s,
                               H.aug_k ? H.aug.as<double>() : nullptr, H.aug_k);
        launch_residual(L.g, L.w, L.op64, H.f.as<double>(), H.u.as<double>(), V, H.rs, 0, L.ks,
                        EPI_OUTER_START, s);
    } else {
        launch_combine_df(len, H.u.as<double>(), L.X.as<float>(), L.stride, L.ks, s,
                          H.aug_k ? H.aug.as<float>() : nullptr, H.aug_k);
        if (sp)
            launch_residual_f32(L.g, L.w, L.op64, H.f.as<double>(), H.u.as<double>(), Vf, H.rs, 0,
                                L.ks, EPI_OUTER_START, s);
        else
            launch_residual_df(L.g, L.w, L.op64, H.f.as<double>(), H.u.as<double>(), Vd, H.rs, 0,
                               L.ks, EPI_OUTER_START, s);
    }
}

void release_pairs(std::vector<ProfPair> &pairs);

Hierarchy::~Hierarchy() {
    if (graph) cudaGraphExecDestroy(graph);
    if (graph_aug) cudaGraphExecDestroy(graph_aug);
    release_pairs(graph_pairs);
    release_pairs(graph_aug_pairs);
}

// One restart cycle captured into a graph: the plain cycle, or (aug) the cycle whose last
// aug_k slots use the recycled corrections.
static mk_status capture_cycle(Problem &P, Hierarchy &H, bool aug = false) {
    cudaGraphExec_t &exec = aug ? H.graph_aug : H.graph;
    std::vector<ProfPair> &pairs = aug ? H.graph_aug_pairs : H.graph_pairs;
    int64_t &kernels = aug ? H.graph_aug_kernels : H.graph_kernels;
    if (exec) {
        cudaGraphExecDestroy(exec);
        exec = nullptr;
    }
    release_pairs(pairs);
    kernels = 0;
    (aug ? H.graph_aug_profiled : H.graph_profiled) = prof_enabled();
    cudaStream_t cs;
    MKCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    MKCK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    set_capture_counter(&kernels);
    prof_set_sink(&pairs);
    enqueue_outer_cycle(P, H, cs, aug);
    prof_set_sink(nullptr);
    set_capture_counter(nullptr);
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (ce != cudaSuccess) {
        cudaStreamDestroy(cs);
        set_cuda_error(ce);
        return MK_ERR_CUDA;
    }
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (ce != cudaSuccess) {
        set_cuda_error(ce);
        exec = nullptr;
        return MK_ERR_CUDA;
    }
    return MK_OK;
}

mk_status solve_prepare(Hierarchy &H, const mk_solve_opts &o, cudaStream_t s) {
    Level &L = *H.lv[0];
    const int64_t len = L.g.len;
    MKCK(cudaMemsetAsync(H.u.p, 0, sizeof(double) * len, s));
    MKCK(cudaMemsetAsync(L.ks.flags, 0, sizeof(int) * 8, s));
    // the tolerance goes through a device-side copy of H's own (the source buffer of an
    // asynchronous copy must outlive it)
    H.tol_host = o.tol;
    MKCK(cudaMemcpyAsync(L.ks.misc() + 7, &H.tol_host, sizeof(double), cudaMemcpyHostToDevice, s));
    // r_0 = f (u^0 = 0): ||f||, tol * ||f||, v_1
    t_outer_j = -1;
    set_ctx(L, 0);
    if (H.precision == 0)
        launch_residual(L.g, L.w, L.op64, H.f.as<double>(), H.u.as<double>(), L.V.as<double>(),
                        H.rs, 0, L.ks, EPI_OUTER_INIT, s);
    else if (H.precision == 2)
        launch_residual_f32(L.g, L.w, L.op64, H.f.as<double>(), H.u.as<double>(), L.V.as<float>(),
                            H.rs, 0, L.ks, EPI_OUTER_INIT, s);
    else
        launch_residual_df(L.g, L.w, L.op64, H.f.as<double>(), H.u.as<double>(), L.V.as<float2>(),
                           H.rs, 0, L.ks, EPI_OUTER_INIT, s);
    return MK_OK;
}

mk_status run_solve(Problem &P, Hierarchy &H, const mk_solve_opts &o, const double *f_padded,
                    mk_solve_info *info, cudaStream_t s) {
    Level &L = *H.lv[0];
    const int64_t len = L.g.len;
    const int64_t launches_start = launches_total();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MKCK(cudaEventCreate(&e0));
    MKCK(cudaEventCreate(&e1));
    MKCK(cudaEventRecord(e0, s));
    if (f_padded && f_padded != H.f.as<double>())
        MKCK(cudaMemcpyAsync(H.f.p, f_padded, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    {
        mk_status st = solve_prepare(H, o, s);
        if (st != MK_OK) return st;
    }
    // one restart cycle as a CUDA graph (captured once per hierarchy and profiling mode)
    if (o.use_graph && (!H.graph || H.graph_profiled != prof_enabled())) {
        mk_status st = capture_cycle(P, H);
        if (st != MK_OK) return st;
    }
    int hflags[8] = {0};
    double hmisc[8] = {0};
    mk_status status = MK_OK;
    int cycles = 0;
    int iters_before = 0;
    std::vector<ProfPair> cycle_pairs;
    for (;;) {
        // recycled corrections: the cycle index selects the ring slot its correction goes to;
        // once aug_k cycles have completed, the cycle uses them
        const bool aug = H.aug_k > 0 && cycles >= H.aug_k;
        if (H.aug_k > 0) {
            H.cycle_host = cycles;
            MKCK(cudaMemcpyAsync(L.ks.flags + 5, &H.cycle_host, sizeof(int), cudaMemcpyHostToDevice, s));
        }
        if (o.use_graph && aug && (!H.graph_aug || H.graph_aug_profiled != prof_enabled())) {
            mk_status st = capture_cycle(P, H, true);
            if (st != MK_OK) return st;
        }
        if (o.use_graph) {
            MKCK(cudaGraphLaunch(aug ? H.graph_aug : H.graph, s));
            add_launches(aug ? H.graph_aug_kernels : H.graph_kernels);
        } else {
            prof_set_sink(&cycle_pairs);
            enqueue_outer_cycle(P, H, s, aug);
            prof_set_sink(nullptr);
        }
        ++cycles;
        MKCK(cudaMemcpyAsync(hflags, L.ks.flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
        MKCK(cudaMemcpyAsync(hmisc, L.ks.misc(), sizeof(hmisc), cudaMemcpyDeviceToHost, s));
        MKCK(cudaStreamSynchronize(s));
        // kernel-class timing: only the iterations of this cycle that did work
        const int worked = hflags[4] - iters_before;
        iters_before = hflags[4];
        if (prof_enabled()) {
            if (o.use_graph) prof_accumulate(aug ? H.graph_aug_pairs : H.graph_pairs, worked);
            else {
                prof_accumulate(cycle_pairs, worked);
                release_pairs(cycle_pairs);
            }
        }
        if (hflags[3]) {
            status = MK_ERR_NONFINITE;
            break;
        }
        if (hflags[0]) break;                 // true residual below tol * ||f||
        if (hflags[4] >= o.max_iters) {
            status = MK_ERR_NOT_CONVERGED;
            break;
        }
    }
    MKCK(cudaEventRecord(e1, s));
    MKCK(cudaEventSynchronize(e1));
    if (prof_enabled()) prof_accumulate_transient();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) {
        info->iterations = hflags[4];
        info->restarts = cycles;
        info->f_norm = hmisc[3];
        info->rel_residual = hmisc[3] > 0.0 ? hmisc[4] / hmisc[3] : 0.0;
        info->solve_ms = ms;
        info->levels = (int)H.lv.size();
        info->kernel_launches = (int32_t)(launches_total() - launches_start);
    }
    return status;
}

mk_status capture_batch(std::vector<Problem *> &P, std::vector<Hierarchy *> &H,
                        std::vector<cudaStream_t> &streams, cudaGraphExec_t &graph,
                        int64_t &kernels) {
    const size_t n = P.size();
    if (n == 0 || H.size() != n || streams.size() < n + 1) return MK_ERR_INVALID;
    kernels = 0;
    cudaStream_t cs = streams[n];   // the capture origin
    std::vector<cudaEvent_t> ev(n + 1, nullptr);
    for (auto &e : ev) MKCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    set_capture_counter(&kernels);
    prof_set_sink(nullptr);
    if (ce == cudaSuccess) ce = cudaEventRecord(ev[n], cs);
    // fork: every problem's restart cycle on its own branch, then join on the origin
    for (size_t i = 0; i < n && ce == cudaSuccess; ++i) {
        ce = cudaStreamWaitEvent(streams[i], ev[n], 0);
        if (ce != cudaSuccess) break;
        enqueue_outer_cycle(*P[i], *H[i], streams[i]);
        ce = cudaEventRecord(ev[i], streams[i]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cs, ev[i], 0);
    }
    set_capture_counter(nullptr);
    cudaError_t ce2 = cudaStreamEndCapture(cs, &g);
    if (ce == cudaSuccess) ce = ce2;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&graph, g, 0);
    if (g) cudaGraphDestroy(g);
    for (auto &e : ev) cudaEventDestroy(e);
    if (ce != cudaSuccess) {
        set_cuda_error(ce);
        graph = nullptr;
        return MK_ERR_CUDA;
    }
    return MK_OK;
}

// ---------------------------------------------------------------------------------------
// Autotuner: tile depths of the 1D transfers per level, coarsest solver variant.
// ---------------------------------------------------------------------------------------
template <typename F>
static float time_launch(F launch, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    launch();   // warm-up
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    return best;
}

template <typename Tc, typename Tv>
static void tune_level(Hierarchy &H, int l, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    Level &L = *H.lv[l];
    Level &C = *H.lv[l + 1];
    if (L.g.dim != 1 || L.nu != 2) return;
    const Tv *v = L.V.as<Tv>();
    // restriction into the next level's first basis slot (or the coarsest right-hand side)
    Tc *dst = C.coarsest ? C.R.as<Tc>() : C.V.as<Tc>();
    const KState ksc = C.coarsest ? KState{nullptr, nullptr, 0} : C.ks;
    float best = 1e30f;
    for (int kc : {1, 2, 4, 8}) {
        set_tile_hint(kc, 0);
        const float t = time_launch([&] {
            launch_restrict<Tv, Tc, Tc>(L.g, C.g, L.nu, L.space, L.w, op_of<Tc>(L), v, nullptr, dst,
                                        H.rs, 0, ksc, nullptr, s);
        }, s, e0, e1);
        if (t < best) {
            best = t;
            L.kc_r = kc;
        }
    }
    set_tile_hint(0, 0);
}

template <typename Tc>
static void tune_interp(Hierarchy &H, int l, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    Level &L = *H.lv[l];
    Level &C = *H.lv[l + 1];
    if (L.g.dim != 1 || L.nu != 2) return;
    const int mc = C.coarsest ? 1 : C.m;
    const double *yc = C.coarsest ? nullptr : C.ks.y();
    float best = 1e30f;
    for (int kc : {2, 4}) {
        set_tile_hint(0, kc);
        const float t = time_launch([&] {
            if (l == 0 && H.precision == 1)
                interp_step<float2, float, float, float2, double>(L, C, L.V.as<float2>(), nullptr,
                                                                  C.X.as<float>(), mc, yc, 0,
                                                                  nullptr, s);
            else
                interp_step<Tc, Tc, Tc, Tc, Tc>(L, C, L.V.as<Tc>(), nullptr, C.X.as<Tc>(), mc, yc,
                                                0, nullptr, s);
        }, s, e0, e1);
        if (t < best) {
            best = t;
            L.kc_i = kc;
        }
    }
    set_tile_hint(0, 0);
}

// Blocks per SM of an inner level's small-basis Gram-Schmidt (dot products and update of
// the second basis vector, the common case), on the level's own buffers.
template <typename Tc>
static void tune_krylov(Hierarchy &H, int l, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    Level &L = *H.lv[l];
    const int j = L.m >= 2 ? 1 : 0;
    float best = 1e30f;
    for (int b : {1, 2, 4}) {
        set_krylov_hint(b);
        const float t = time_launch([&] {
            launch_multidot<Tc, Tc>(L.g.len, L.W.as<Tc>(), L.V.as<Tc>(), L.stride, j, H.rs, L.ks,
                                    false, nullptr, s);
            if (j + 1 < L.m)
                launch_update<Tc, Tc>(L.g.len, L.W.as<Tc>(), L.V.as<Tc>(), L.stride, j, true,
                                      H.rs, L.ks, UPD_INNER, false, nullptr, s);
        }, s, e0, e1);
        if (t < best) {
            best = t;
            L.kr_bpsm = b;
        }
    }
    set_krylov_hint(0);
}

mk_status autotune_hierarchy(Hierarchy &H, cudaStream_t s) {
    cudaEvent_t e0, e1;
    MKCK(cudaEventCreate(&e0));
    MKCK(cudaEventCreate(&e1));
    const int L = (int)H.lv.size();
    const bool fp64 = H.precision == 0;
    for (int l = 1; l + 1 < L; ++l) {
        if (fp64) tune_krylov<double>(H, l, s, e0, e1);
        else tune_krylov<float>(H, l, s, e0, e1);
    }
    for (int l = 0; l + 1 < L; ++l) {
        if (fp64) {
            tune_level<double, double>(H, l, s, e0, e1);
            tune_interp<double>(H, l, s, e0, e1);
        } else {
            if (l == 0 && H.precision == 1) tune_level<float, float2>(H, l, s, e0, e1);
            else tune_level<float, float>(H, l, s, e0, e1);
            tune_interp<float>(H, l, s, e0, e1);
        }
    }
    // coarsest: every applicable variant of the decoupled slab solve
    Level &C = *H.lv.back();
    // inner levels in the cooperative kernel (MK_INNER_COOP only): its grid, 2 or 3 blocks
    // per SM.  (Timing one cycle step outside a graph would favour it over the separate
    // launches, whose per-launch host cost a captured graph does not pay; whole solves measure
    // it slower, so MK_INNER_AUTO keeps the separate launches.)
    if (H.use_coop && !fp64) {
        float best = 1e30f;
        int best_b = 0;
        for (int b : {2, 3}) {
            if (coop_configure(H, b) != MK_OK) continue;
            const float t = time_launch([&] { enqueue_cycle_step(H, 0, 0, nullptr, s); }, s, e0, e1);
            if (t < best) {
                best = t;
                best_b = b;
            }
        }
        if (best_b > 0) {
            mk_status st = coop_configure(H, best_b);
            if (st != MK_OK) return st;
        }
    }
    if (C.g.dim == 1) {
        float best = 1e30f;
        for (int kind : {1, 2, 3}) {
            if (kind == 1 && (fp64 || C.dstN2 == 0)) continue;
            if (kind == 2 && C.spikeU == 0) continue;
            C.coarse_kind = kind;
            const float t = time_launch([&] { enqueue_coarsest(H, nullptr, s); }, s, e0, e1);
            if (t < best) {
                best = t;
                C.coarse_kind_best = kind;
            }
        }
        C.coarse_kind = C.coarse_kind_best;
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return MK_ERR_CUDA;
    }
    return MK_OK;
}

// ---------------------------------------------------------------------------------------
// theta-march tables (fine level, FP64)
// ---------------------------------------------------------------------------------------
mk_status prepare_march(Problem &P) {
    if (P.march_ready) return MK_OK;
    Tri Lx = fd_laplacian(P.nx, P.tau);
    Tri Ly;
    if (P.dim == 2) Ly = fd_laplacian(P.ny, P.tau);
    std::vector<double> c = coef_concat(Lx, P.dim == 2 ? &Ly : nullptr);
    MKCK(upload<double>(P.m_c64, c));
    const double a = P.theta * P.dt;
    if (P.dim == 1) {
        if (P.nx > 4096) return MK_ERR_INVALID;
        int np = 32;
        while (np < P.nx) np *= 2;
        P.m_npad = np;
        P.m_nlev = pcr_levels(P.nx);
        std::vector<double> al, ga, bi;
        pcr_tables(Lx, a, np, al, ga, bi);
        if (al.empty()) {
            al.assign(np, 0.0);
            ga.assign(np, 0.0);
        }
        MKCK(upload<double>(P.m_alpha, al));
        MKCK(upload<double>(P.m_gamma, ga));
        MKCK(upload<double>(P.m_binv, bi));
        if (slab_warp_supported<double>(P.nx)) {
            P.m_spikeU = spike_block_size(P.nx);
            std::vector<double> tab;
            spike_tables(Lx, a, P.m_spikeU, spike_threads(P.nx), tab);
            MKCK(upload<double>(P.m_spike, tab));
        }
    } else if ((march2d_transform_size(P.nx) || P.nx <= MARCH2D_DENSE_MAX) &&
               (march2d_transform_size(P.ny) || P.ny <= MARCH2D_DENSE_MAX)) {
        // uniform fine-level operator: analytic eigenvalues, sine transform per step
        const double pi = 3.14159265358979323846;
        double cx = 0.0, cy = 0.0;
        if (!tri_uniform(Lx, cx) || !tri_uniform(Ly, cy)) return MK_ERR_INVALID;
        std::vector<double> lx(P.nx), ly(P.ny), tab, twx, twy;
        for (int i = 0; i < P.nx; ++i) {
            const double sn = std::sin(pi * (i + 1) / (2.0 * (P.nx + 1)));
            lx[i] = -4.0 * cx * sn * sn;
        }
        for (int j = 0; j < P.ny; ++j) {
            const double sn = std::sin(pi * (j + 1) / (2.0 * (P.ny + 1)));
            ly[j] = -4.0 * cy * sn * sn;
        }
        dst_tables(P.nx, cx, 0.0, 0.0, tab, twx);
        dst_tables(P.ny, cy, 0.0, 0.0, tab, twy);
        MKCK(upload<double>(P.m_lamx, lx));
        MKCK(upload<double>(P.m_lamy, ly));
        MKCK(upload<double>(P.m_twx, twx));
        MKCK(upload<double>(P.m_twy, twy));
        // dense sine matrices for directions whose n + 1 is not a power of two
        // (the angle reduced modulo 2 pi exactly, in integers, before the sine)
        auto sine_matrix = [&](int n, DevMem &m) -> cudaError_t {
            if (march2d_transform_size(n)) return cudaSuccess;
            std::vector<double> S((size_t)n * n);
            const int64_t period = 2 * (int64_t)(n + 1);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j)
                    S[(size_t)i * n + j] =
                        std::sin(pi * (double)(((int64_t)(i + 1) * (j + 1)) % period) / (n + 1));
            return upload<double>(m, S);
        };
        MKCK(sine_matrix(P.nx, P.m_Sx));
        MKCK(sine_matrix(P.ny, P.m_Sy));
        MKCK(P.m_t1.alloc(sizeof(double) * (size_t)P.nx * P.ny));
        P.m_cx = cx;
        P.m_cy = cy;
    } else {
        return MK_ERR_INVALID;
    }
    P.march_ready = true;
    return MK_OK;
}

}  // namespace mk
