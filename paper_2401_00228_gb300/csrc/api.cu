// C ABI of libmk (see include/mk.h): argument checks, host/device pointer staging, and
// the operator-level entry points used to check each step of the path on its own.
#include <atomic>
#include <cmath>
#include <type_traits>
#include <cstring>
#include <memory>

#include "solver.h"

namespace mk {

int g_num_sms = 0;
static thread_local std::string g_last_err;

void set_cuda_error(cudaError_t e) { g_last_err = cudaGetErrorString(e); }

int64_t launches_total();
void prof_set_enabled(bool on);
void prof_reset();
bool prof_read(int cls, int level, double &ms, double &bytes, int64_t &n);

cudaError_t slab_set_attributes();
cudaError_t interp2d_set_attributes();

// adjoint helpers (stencil.cu)
void launch_reverse_pack(const Geom &g, const double *dense, double *padded, cudaStream_t s);
void launch_adjoint_grads(const Geom &g, double theta, double dt, double tau, SpaceOp<double> L,
                          const double *y, const double *b, const double *upad, double *lam,
                          double *grad_u0, double *grad_g, const ReduceScratch &rs, KState ks,
                          cudaStream_t s);

}  // namespace mk

using namespace mk;

struct mk_problem {
    Problem P;
};

// A batch: its own hierarchy per problem and one CUDA graph whose replay runs one restart
// cycle of every problem, each on its own branch.
struct mk_batch {
    std::vector<mk_problem *> probs;
    std::vector<mk_solve_opts> opts;
    std::vector<std::unique_ptr<Hierarchy>> H;
    std::vector<cudaStream_t> streams;   // one per problem + the capture origin
    cudaGraphExec_t graph = nullptr;
    int64_t graph_kernels = 0;
    DevMem flagptrs, miscptrs, gflags, gmisc;   // status gather
    std::vector<int> one;                       // source of the "stop" flag copies
    ~mk_batch() {
        cudaDeviceSynchronize();
        if (graph) cudaGraphExecDestroy(graph);
        for (cudaStream_t s : streams)
            if (s) cudaStreamDestroy(s);
    }
};

namespace mk {
// flags[0..7] and misc[0..7] of every problem's level-1 FGMRES state into two arrays
__global__ void k_gather_status(const int *const *flags, const double *const *misc, int n,
                                int *of, double *om) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int q = 0; q < 8; ++q) {
        of[8 * i + q] = flags[i][q];
        om[8 * i + q] = misc[i][q];
    }
}
}  // namespace mk

#define CK(call)                                                                 \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            set_cuda_error(e_);                                                  \
            return e_ == cudaErrorMemoryAllocation ? MK_ERR_NOMEM : MK_ERR_CUDA; \
        }                                                                        \
    } while (0)

#define CKS(expr)                       \
    do {                                \
        mk_status s_ = (expr);          \
        if (s_ != MK_OK) return s_;     \
    } while (0)

static mk_status ensure_device() {
    if (g_num_sms > 0) return MK_OK;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(slab_set_attributes());
    CK(interp2d_set_attributes());
    CK(dst_set_attributes());
    CK(coop_set_attributes());
    CK(march2d_set_attributes());
    g_num_sms = sms > 0 ? sms : 1;
    return MK_OK;
}

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Input array: device pointer as is, host array copied into tmp.
static mk_status stage_in(const double *p, size_t n, DevMem &tmp, const double *&dp, cudaStream_t s) {
    if (is_device_ptr(p)) {
        dp = p;
        return MK_OK;
    }
    CK(tmp.alloc(sizeof(double) * (n ? n : 1)));
    CK(cudaMemcpyAsync(tmp.p, p, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    dp = tmp.as<double>();
    return MK_OK;
}

// Output array: device pointer as is, host array gets a device staging buffer.
struct OutStage {
    double *user = nullptr;
    double *dev = nullptr;
    size_t n = 0;
    bool host = false;
    DevMem tmp;
};
static mk_status stage_out(double *p, size_t n, OutStage &o) {
    o.user = p;
    o.n = n;
    if (is_device_ptr(p)) {
        o.dev = p;
        return MK_OK;
    }
    o.host = true;
    CK(o.tmp.alloc(sizeof(double) * (n ? n : 1)));
    o.dev = o.tmp.as<double>();
    return MK_OK;
}
static mk_status finish_out(OutStage &o, cudaStream_t s) {
    if (!o.host) return MK_OK;
    CK(cudaMemcpyAsync(o.user, o.dev, sizeof(double) * o.n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return MK_OK;
}

static size_t space_n(const Problem &P) { return (size_t)P.nx * (P.dim == 2 ? P.ny : 1); }
static size_t st_n(const Problem &P) { return space_n(P) * (size_t)(P.nt + 1); }

static mk_solve_opts resolve_opts(const mk_solve_opts *o) {
    mk_solve_opts r;
    if (o) r = *o;
    else mk_default_opts(&r);
    return r;
}

extern "C" {

void mk_default_opts(mk_solve_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-12;
    o->restart = 40;
    o->max_iters = 2000;
    o->levels = 3;
    for (int i = 0; i < MK_MAX_LEVELS; ++i) {
        o->nu[i] = 2;
        o->space[i] = 0;
        o->m_inner[i] = 2;
    }
    o->m_inner[0] = 1;   // with 3 levels the only intermediate level sits above the coarsest
    o->n_cgs = 16;
    o->mu_mode = 0;
    o->mu_value = 1.0;
    o->precision = 0;
    o->use_graph = 1;
    o->orth = 1;
}

mk_status mk_schedule_alternate(int32_t dim, int32_t nx, int32_t ny, int32_t nt, double tau,
                                double dt, int32_t levels, int32_t n_cgs, double c_max,
                                mk_solve_opts *opts) {
    if (!opts || (dim != 1 && dim != 2) || levels < 2 || levels > MK_MAX_LEVELS) return MK_ERR_INVALID;
    if (dim == 1) ny = 1;
    if (nx < 1 || ny < 1 || nt < 1 || n_cgs < 1) return MK_ERR_INVALID;
    if (!(tau > 0.0) || !(dt > 0.0) || !(c_max > 0.0)) return MK_ERR_INVALID;
    const double cd = dim == 1 ? 2.0 : 3.0;
    const double h = 1.0 / (nx + 1);
    mk_solve_opts o = *opts;
    double dT = dt, dx2 = h * h;
    int n_t = nt, mx = nx, my = ny;
    bool alternating = false, next_space = true;
    for (int l = 0; l + 1 < levels; ++l) {
        if (!alternating && cd * tau * dT / dx2 > c_max) alternating = true;
        const bool space = alternating && next_space;
        if (alternating) next_space = !next_space;
        if (space) {
            if (mx < 2 || (dim == 2 && my < 2)) return MK_ERR_INVALID;
            mx = (mx + 1) / 2;
            if (dim == 2) my = (my + 1) / 2;
            dx2 *= 2.0;
            o.nu[l] = 1;
            o.space[l] = 1;
        } else {
            if (n_t % 2) return MK_ERR_INVALID;
            n_t /= 2;
            dT *= 2.0;
            o.nu[l] = 2;
            o.space[l] = 0;
        }
    }
    if (n_t % n_cgs) return MK_ERR_INVALID;
    for (int l = 0; l + 2 < levels; ++l) o.m_inner[l] = (l + 3 == levels) ? 1 : 2;
    o.levels = levels;
    o.n_cgs = n_cgs;
    *opts = o;
    return MK_OK;
}

const char *mk_status_string(mk_status s) {
    switch (s) {
        case MK_OK: return "MK_OK";
        case MK_ERR_INVALID: return "MK_ERR_INVALID";
        case MK_ERR_NOMEM: return "MK_ERR_NOMEM";
        case MK_ERR_CUDA: return "MK_ERR_CUDA";
        case MK_ERR_NONFINITE: return "MK_ERR_NONFINITE";
        case MK_ERR_NOT_CONVERGED: return "MK_ERR_NOT_CONVERGED";
        case MK_ERR_TIMEOUT: return "MK_ERR_TIMEOUT";
        case MK_ERR_TOO_LARGE: return "MK_ERR_TOO_LARGE";
    }
    return "MK_ERR_UNKNOWN";
}

const char *mk_last_cuda_error(void) { return g_last_err.c_str(); }

int64_t mk_kernel_launch_count(void) { return launches_total(); }

void mk_set_profiling(int32_t on) { prof_set_enabled(on != 0); }

void mk_profile_reset(void) { prof_reset(); }

mk_status mk_profile_read(int32_t cls, int32_t level, double *ms, double *bytes, int64_t *launches) {
    double a = 0.0, b = 0.0;
    int64_t n = 0;
    if (!prof_read(cls, level, a, b, n)) return MK_ERR_INVALID;
    if (ms) *ms = a;
    if (bytes) *bytes = b;
    if (launches) *launches = n;
    return MK_OK;
}

const char *mk_profile_class_name(int32_t cls) {
    static const char *names[] = {"restrict", "interp_correct", "multidot", "update", "slab",
                                  "residual", "combine", "march", "other", "inner_coop"};
    if (cls < 0 || cls >= PROF_NCLASS) return "";
    return names[cls];
}

mk_status mk_problem_shape(const mk_problem *p, int32_t *dim, int32_t *nx, int32_t *ny,
                           int32_t *nt, double *theta, double *dt, double *tau) {
    if (!p) return MK_ERR_INVALID;
    if (dim) *dim = p->P.dim;
    if (nx) *nx = p->P.nx;
    if (ny) *ny = p->P.ny;
    if (nt) *nt = p->P.nt;
    if (theta) *theta = p->P.theta;
    if (dt) *dt = p->P.dt;
    if (tau) *tau = p->P.tau;
    return MK_OK;
}

mk_status mk_set_source(mk_problem *p, const double *g, void *stream) {
    if (!p) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Problem &P = p->P;
    CK(cudaMemsetAsync(P.fsrc.p, 0, sizeof(double) * P.g.len, s));
    P.has_source = g != nullptr;
    if (!g) return MK_OK;
    DevMem tmp;
    const double *dg = nullptr;
    CKS(stage_in(g, st_n(P), tmp, dg, s));
    launch_rhs_source(P.g, P.theta, P.dt, dg, P.fsrc.as<double>(), s);
    CK(cudaGetLastError());
    if (tmp.p) CK(cudaStreamSynchronize(s));
    return MK_OK;
}

mk_status mk_create_problem(const mk_stencil *A, double theta, double dt, int32_t nt,
                            const double *g, mk_problem **out) {
    if (!A || !out) return MK_ERR_INVALID;
    *out = nullptr;
    if (A->dim != 1 && A->dim != 2) return MK_ERR_INVALID;
    if (A->nx < 1 || (A->dim == 2 && A->ny < 1)) return MK_ERR_INVALID;
    if (!(theta >= 0.0 && theta <= 1.0) || !(dt > 0.0) || nt < 1 || !(A->tau > 0.0))
        return MK_ERR_INVALID;
    if (!std::isfinite(dt) || !std::isfinite(A->tau)) return MK_ERR_INVALID;
    CKS(ensure_device());
    std::unique_ptr<mk_problem> p(new mk_problem());
    Problem &P = p->P;
    P.dim = A->dim;
    P.nx = A->nx;
    P.ny = A->dim == 2 ? A->ny : 1;
    P.nt = nt;
    P.theta = theta;
    P.dt = dt;
    P.tau = A->tau;
    P.g = make_geom(P.dim, P.nx, P.ny, nt);
    CK(P.fsrc.alloc(sizeof(double) * P.g.len));
    CKS(mk_set_source(p.get(), g, nullptr));
    CK(cudaStreamSynchronize(nullptr));
    *out = p.release();
    return MK_OK;
}

void mk_destroy(mk_problem *p) {
    if (!p) return;
    cudaDeviceSynchronize();
    delete p;
}

mk_status mk_trim(mk_problem *p) {
    if (!p) return MK_ERR_INVALID;
    CK(cudaDeviceSynchronize());
    p->P.H.reset();
    return MK_OK;
}

// pack a dense (nt+1) x n array into the padded fine-level layout
static void pack_fine(const Problem &P, const double *dense, double *padded, cudaStream_t s) {
    launch_pack<double, double>(P.g, dense, padded, s);
}

static mk_status solve_common(mk_problem *p, const mk_solve_opts &o, mk_solve_info *info,
                              cudaStream_t s, Hierarchy *H, double *u_out_dev) {
    Problem &P = p->P;
    int64_t before = mk_kernel_launch_count();
    mk_status st = run_solve(P, *H, o, nullptr, info, s);
    if (st != MK_OK && st != MK_ERR_NOT_CONVERGED) return st;
    launch_unpack<double, double>(P.g, H->u.as<double>(), u_out_dev, s);
    CK(cudaGetLastError());
    if (info) info->kernel_launches = (int32_t)(mk_kernel_launch_count() - before);
    return st;
}

mk_status mk_solve(mk_problem *p, const double *u0, const mk_solve_opts *opts, double *u_out,
                   mk_solve_info *info, void *stream) {
    if (!p || !u0 || !u_out) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    mk_solve_opts o = resolve_opts(opts);
    Problem &P = p->P;
    CKS(validate_opts(P, o));
    Hierarchy *H = nullptr;
    CKS(build_hierarchy(P, o, H));
    DevMem tin;
    const double *du0 = nullptr;
    CKS(stage_in(u0, space_n(P), tin, du0, s));
    OutStage os;
    CKS(stage_out(u_out, st_n(P), os));
    // f = source blocks, f_0 = u0
    CK(cudaMemcpyAsync(H->f.p, P.fsrc.p, sizeof(double) * P.g.len, cudaMemcpyDeviceToDevice, s));
    Geom g0 = P.g;
    g0.nt = 0;
    launch_pack<double, double>(g0, du0, H->f.as<double>(), s);
    mk_status st = solve_common(p, o, info, s, H, os.dev);
    if (st != MK_OK && st != MK_ERR_NOT_CONVERGED) return st;
    CKS(finish_out(os, s));
    return st;
}

mk_status mk_solve_rhs(mk_problem *p, const double *f, const mk_solve_opts *opts, double *u_out,
                       mk_solve_info *info, void *stream) {
    if (!p || !f || !u_out) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    mk_solve_opts o = resolve_opts(opts);
    Problem &P = p->P;
    CKS(validate_opts(P, o));
    Hierarchy *H = nullptr;
    CKS(build_hierarchy(P, o, H));
    DevMem tin;
    const double *df = nullptr;
    CKS(stage_in(f, st_n(P), tin, df, s));
    OutStage os;
    CKS(stage_out(u_out, st_n(P), os));
    pack_fine(P, df, H->f.as<double>(), s);
    mk_status st = solve_common(p, o, info, s, H, os.dev);
    if (st != MK_OK && st != MK_ERR_NOT_CONVERGED) return st;
    CKS(finish_out(os, s));
    return st;
}

mk_status mk_march(mk_problem *p, const double *u0, double *u_out, void *stream) {
    if (!p || !u0 || !u_out) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Problem &P = p->P;
    CKS(prepare_march(P));
    DevMem tin, fbuf, ubuf;
    const double *du0 = nullptr;
    CKS(stage_in(u0, space_n(P), tin, du0, s));
    OutStage os;
    CKS(stage_out(u_out, st_n(P), os));
    CK(fbuf.alloc(sizeof(double) * P.g.len));
    CK(ubuf.alloc(sizeof(double) * P.g.len));
    CK(cudaMemcpyAsync(fbuf.p, P.fsrc.p, sizeof(double) * P.g.len, cudaMemcpyDeviceToDevice, s));
    Geom g0 = P.g;
    g0.nt = 0;
    launch_pack<double, double>(g0, du0, fbuf.as<double>(), s);
    SpaceOp<double> op{P.m_c64.as<double>(), P.dim == 2 ? P.m_c64.as<double>() + 3 * P.nx : nullptr};
    const double a = P.theta * P.dt, b = (1.0 - P.theta) * P.dt;
    if (P.dim == 1 && P.m_spikeU > 0)
        launch_slab_1d_warp<double>(P.g, b, P.m_spike.as<double>(), P.m_spikeU, 0, fbuf.as<double>(),
                                    ubuf.as<double>(), nullptr, s, PROF_MARCH);
    else if (P.dim == 1)
        launch_march_1d(P.g, b, op, P.m_alpha.as<double>(), P.m_gamma.as<double>(),
                        P.m_binv.as<double>(), P.m_npad, P.m_nlev, fbuf.as<double>(),
                        ubuf.as<double>(), s);
    else {
        // 2D: u_0 = f_0 (guard and plane 0), then the steps
        CK(cudaMemcpyAsync(ubuf.p, fbuf.p, sizeof(double) * (size_t)(P.g.guard + P.g.plane),
                           cudaMemcpyDeviceToDevice, s));
        launch_march_2d_dst(P.g, a, b, P.m_cx, P.m_cy, P.m_lamx.as<double>(), P.m_lamy.as<double>(),
                            P.m_twx.as<double2>(), P.m_twy.as<double2>(), P.m_Sx.as<double>(),
                            P.m_Sy.as<double>(), fbuf.as<double>(), ubuf.as<double>(),
                            P.m_t1.as<double>(), s);
    }
    launch_unpack<double, double>(P.g, ubuf.as<double>(), os.dev, s);
    CK(cudaGetLastError());
    CKS(finish_out(os, s));
    // keep the staging buffers alive until the work that uses them is done
    CK(cudaStreamSynchronize(s));
    return MK_OK;
}

mk_status mk_adjoint(mk_problem *p, const double *u, const double *dJdu, const mk_solve_opts *opts,
                     double *grad_u0, double *grad_g, double *grad_tau, double *lam_out,
                     mk_solve_info *info, void *stream) {
    if (!p || !dJdu) return MK_ERR_INVALID;
    if (grad_tau && !u) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    mk_solve_opts o = resolve_opts(opts);
    Problem &P = p->P;
    CKS(validate_opts(P, o));
    Hierarchy *H = nullptr;
    CKS(build_hierarchy(P, o, H));
    DevMem tb, tu, upad;
    const double *db = nullptr, *du = nullptr;
    CKS(stage_in(dJdu, st_n(P), tb, db, s));
    if (u) {
        CKS(stage_in(u, st_n(P), tu, du, s));
        CK(upad.alloc(sizeof(double) * P.g.len));
        pack_fine(P, du, upad.as<double>(), s);
    }
    // time-reversed transposed system: f_rev[0] = 0, f_rev[j] = b[nt+1-j]
    launch_reverse_pack(P.g, db, H->f.as<double>(), s);
    mk_status st = run_solve(P, *H, o, nullptr, info, s);
    if (st != MK_OK && st != MK_ERR_NOT_CONVERGED) return st;
    OutStage o_lam, o_gu0, o_gg;
    DevMem d_lam, d_gu0, d_gg;
    if (lam_out) CKS(stage_out(lam_out, st_n(P), o_lam));
    if (grad_u0) CKS(stage_out(grad_u0, space_n(P), o_gu0));
    if (grad_g) CKS(stage_out(grad_g, st_n(P), o_gg));
    Level &L0 = *H->lv[0];
    launch_adjoint_grads(P.g, P.theta, P.dt, P.tau, L0.op64, H->u.as<double>(), db,
                         u ? upad.as<double>() : nullptr, lam_out ? o_lam.dev : nullptr,
                         grad_u0 ? o_gu0.dev : nullptr, grad_g ? o_gg.dev : nullptr, H->rs, L0.ks,
                         s);
    CK(cudaGetLastError());
    if (grad_tau) {
        double hmisc[8];
        CK(cudaMemcpyAsync(hmisc, L0.ks.misc(), sizeof(hmisc), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        double v = hmisc[5];
        if (is_device_ptr(grad_tau)) CK(cudaMemcpy(grad_tau, &v, sizeof(double), cudaMemcpyHostToDevice));
        else *grad_tau = v;
    }
    if (lam_out) CKS(finish_out(o_lam, s));
    if (grad_u0) CKS(finish_out(o_gu0, s));
    if (grad_g) CKS(finish_out(o_gg, s));
    CK(cudaStreamSynchronize(s));
    return st;
}

// ------------------------------------------------------------------------------------
// operator-level entry points
// ------------------------------------------------------------------------------------
static mk_status get_level(mk_problem *p, const mk_solve_opts *opts, int level, Hierarchy *&H,
                           mk_solve_opts &o) {
    if (!p) return MK_ERR_INVALID;
    o = resolve_opts(opts);
    CKS(validate_opts(p->P, o));
    CKS(build_hierarchy(p->P, o, H));
    if (level < 1 || level > (int)H->lv.size()) return MK_ERR_INVALID;
    return MK_OK;
}

mk_status mk_level_info(mk_problem *p, const mk_solve_opts *opts, int32_t level,
                        mk_level_desc *d, double *xcoef, double *ycoef) {
    Hierarchy *H = nullptr;
    mk_solve_opts o;
    CKS(get_level(p, opts, level, H, o));
    Level &L = *H->lv[level - 1];
    if (d) {
        d->dim = L.g.dim;
        d->nx = L.g.nx;
        d->ny = L.g.ny;
        d->nt = L.g.nt;
        d->a = L.w.a;
        d->b = L.w.b;
        d->mu = L.w.mu;
    }
    auto put = [](const Tri &t, double *c) {
        int n = t.n();
        for (int i = 0; i < n; ++i) {
            c[i] = t.lo[i];
            c[n + i] = t.di[i];
            c[2 * n + i] = t.up[i];
        }
    };
    if (xcoef) put(L.Lx, xcoef);
    if (ycoef && L.g.dim == 2) put(L.Ly, ycoef);
    return MK_OK;
}

mk_status mk_op_rhs(mk_problem *p, const double *u0, double *f, void *stream) {
    if (!p || !u0 || !f) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Problem &P = p->P;
    DevMem tin, fp;
    const double *du0 = nullptr;
    CKS(stage_in(u0, space_n(P), tin, du0, s));
    OutStage os;
    CKS(stage_out(f, st_n(P), os));
    CK(fp.alloc(sizeof(double) * P.g.len));
    CK(cudaMemcpyAsync(fp.p, P.fsrc.p, sizeof(double) * P.g.len, cudaMemcpyDeviceToDevice, s));
    Geom g0 = P.g;
    g0.nt = 0;
    launch_pack<double, double>(g0, du0, fp.as<double>(), s);
    launch_unpack<double, double>(P.g, fp.as<double>(), os.dev, s);
    CK(cudaGetLastError());
    CKS(finish_out(os, s));
    CK(cudaStreamSynchronize(s));
    return MK_OK;
}

}  // extern "C"

template <typename T>
static mk_status op_apply_t(Level &L, const double *dx, double *dw, cudaStream_t s) {
    DevMem xp, wp;
    CK(xp.alloc(sizeof(T) * L.g.len));
    CK(wp.alloc(sizeof(T) * L.g.len));
    launch_pack<double, T>(L.g, dx, xp.as<T>(), s);
    launch_apply<T, T, T>(L.g, L.w, op_of<T>(L),
                          xp.as<T>(), wp.as<T>(), s);
    launch_unpack<T, double>(L.g, wp.as<T>(), dw, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return MK_OK;
}

static size_t level_n(const Level &L) { return (size_t)L.g.nx * L.g.ny * (size_t)(L.g.nt + 1); }

extern "C" {

mk_status mk_op_apply(mk_problem *p, const mk_solve_opts *opts, int32_t level, int32_t precision,
                      const double *x, double *w, void *stream) {
    if (!x || !w || (precision != 0 && precision != 1)) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Hierarchy *H = nullptr;
    mk_solve_opts o;
    CKS(get_level(p, opts, level, H, o));
    Level &L = *H->lv[level - 1];
    DevMem tin;
    const double *dx = nullptr;
    CKS(stage_in(x, level_n(L), tin, dx, s));
    OutStage os;
    CKS(stage_out(w, level_n(L), os));
    CKS(precision == 0 ? op_apply_t<double>(L, dx, os.dev, s) : op_apply_t<float>(L, dx, os.dev, s));
    return finish_out(os, s);
}

mk_status mk_op_residual(mk_problem *p, const double *f, const double *u, double *r, double *rnorm,
                         void *stream) {
    if (!p || !f || !u || !r) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Problem &P = p->P;
    // a standalone fine level (no hierarchy needed): coefficients, state, reduction scratch
    Level L;
    L.g = P.g;
    L.w.a = P.theta * P.dt;
    L.w.b = (1.0 - P.theta) * P.dt;
    {
        Tri Lx = fd_laplacian(P.nx, P.tau), Ly;
        if (P.dim == 2) Ly = fd_laplacian(P.ny, P.tau);
        std::vector<double> c(Lx.lo);
        c.insert(c.end(), Lx.di.begin(), Lx.di.end());
        c.insert(c.end(), Lx.up.begin(), Lx.up.end());
        if (P.dim == 2) {
            c.insert(c.end(), Ly.lo.begin(), Ly.lo.end());
            c.insert(c.end(), Ly.di.begin(), Ly.di.end());
            c.insert(c.end(), Ly.up.begin(), Ly.up.end());
        }
        CK(L.c64.alloc(sizeof(double) * c.size()));
        CK(cudaMemcpy(L.c64.p, c.data(), sizeof(double) * c.size(), cudaMemcpyHostToDevice));
        L.op64.x = L.c64.as<double>();
        L.op64.y = P.dim == 2 ? L.c64.as<double>() + 3 * P.nx : nullptr;
    }
    CK(L.ksd.alloc(sizeof(double) * KState::ndoubles(1)));
    CK(L.ksf.alloc(sizeof(int) * 8));
    L.ks = KState{L.ksd.as<double>(), L.ksf.as<int>(), 1};
    DevMem part, cnt;
    ReduceScratch rs;
    rs.max_blocks = 65536;
    CK(part.alloc(sizeof(double) * rs.max_blocks));
    CK(cnt.alloc(sizeof(unsigned) * 4));
    rs.partials = part.as<double>();
    rs.counter = cnt.as<unsigned>();
    size_t n = st_n(P);
    DevMem tf, tu, fp, up, rp;
    const double *df = nullptr, *du = nullptr;
    CKS(stage_in(f, n, tf, df, s));
    CKS(stage_in(u, n, tu, du, s));
    OutStage os;
    CKS(stage_out(r, n, os));
    CK(fp.alloc(sizeof(double) * L.g.len));
    CK(up.alloc(sizeof(double) * L.g.len));
    CK(rp.alloc(sizeof(double) * L.g.len));
    launch_pack<double, double>(L.g, df, fp.as<double>(), s);
    launch_pack<double, double>(L.g, du, up.as<double>(), s);
    launch_residual(L.g, L.w, L.op64, fp.as<double>(), up.as<double>(), rp.as<double>(), rs, 0,
                    L.ks, EPI_NONE, s);
    launch_unpack<double, double>(L.g, rp.as<double>(), os.dev, s);
    CK(cudaGetLastError());
    double hm[8];
    CK(cudaMemcpyAsync(hm, L.ks.misc(), sizeof(hm), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (rnorm) *rnorm = std::sqrt(hm[5]);
    return finish_out(os, s);
}

}  // extern "C"

template <typename T>
static mk_status op_restrict_t(Hierarchy &H, int l, const double *dv, double *dvh, cudaStream_t s) {
    Level &L = *H.lv[l];
    Level &C = *H.lv[l + 1];
    DevMem vp, cp;
    CK(vp.alloc(sizeof(T) * L.g.len));
    CK(cp.alloc(sizeof(T) * C.g.len));
    launch_pack<double, T>(L.g, dv, vp.as<T>(), s);
    SpaceOp<T> op = op_of<T>(L);
    launch_restrict<T, T, T>(L.g, C.g, L.nu, L.space, L.w, op, vp.as<T>(), nullptr, cp.as<T>(),
                             H.rs, 0, KState{nullptr, nullptr, 0}, nullptr, s);
    launch_unpack<T, double>(C.g, cp.as<T>(), dvh, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return MK_OK;
}

extern "C" {

mk_status mk_op_restrict(mk_problem *p, const mk_solve_opts *opts, int32_t level, int32_t precision,
                         const double *v, double *vhat, void *stream) {
    if (!v || !vhat || (precision != 0 && precision != 1)) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Hierarchy *H = nullptr;
    mk_solve_opts o;
    CKS(get_level(p, opts, level, H, o));
    if (o.transfer != MK_TRANSFER_MK) return MK_ERR_INVALID;
    if (level >= (int)H->lv.size()) return MK_ERR_INVALID;
    Level &L = *H->lv[level - 1];
    Level &C = *H->lv[level];
    DevMem tin;
    const double *dv = nullptr;
    CKS(stage_in(v, level_n(L), tin, dv, s));
    OutStage os;
    CKS(stage_out(vhat, level_n(C), os));
    CKS(precision == 0 ? op_restrict_t<double>(*H, level - 1, dv, os.dev, s)
                       : op_restrict_t<float>(*H, level - 1, dv, os.dev, s));
    return finish_out(os, s);
}

}  // extern "C"

template <typename T>
static mk_status op_interp_t(Hierarchy &H, int l, const double *dv, const double *dvt, double *dx,
                             double *dw, cudaStream_t s) {
    Level &L = *H.lv[l];
    Level &C = *H.lv[l + 1];
    DevMem vp, cp, xp, wp;
    CK(vp.alloc(sizeof(T) * L.g.len));
    CK(cp.alloc(sizeof(T) * C.g.len));
    CK(xp.alloc(sizeof(T) * L.g.len));
    CK(wp.alloc(sizeof(T) * L.g.len));
    launch_pack<double, T>(L.g, dv, vp.as<T>(), s);
    launch_pack<double, T>(C.g, dvt, cp.as<T>(), s);
    SpaceOp<T> op = op_of<T>(L);
    launch_interp<T, T, T, T, T>(L.g, C.g, L.nu, L.space, L.w, op, vp.as<T>(), nullptr, cp.as<T>(),
                                 1, C.stride, nullptr, xp.as<T>(), wp.as<T>(), nullptr, s);
    launch_unpack<T, double>(L.g, xp.as<T>(), dx, s);
    launch_unpack<T, double>(L.g, wp.as<T>(), dw, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return MK_OK;
}

extern "C" {

mk_status mk_op_interp_correct(mk_problem *p, const mk_solve_opts *opts, int32_t level,
                               int32_t precision, const double *v, const double *vt, double *x,
                               double *w, void *stream) {
    if (!v || !vt || !x || !w || (precision != 0 && precision != 1)) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Hierarchy *H = nullptr;
    mk_solve_opts o;
    CKS(get_level(p, opts, level, H, o));
    if (o.transfer != MK_TRANSFER_MK) return MK_ERR_INVALID;
    if (level >= (int)H->lv.size()) return MK_ERR_INVALID;
    Level &L = *H->lv[level - 1];
    Level &C = *H->lv[level];
    DevMem t1, t2;
    const double *dv = nullptr, *dvt = nullptr;
    CKS(stage_in(v, level_n(L), t1, dv, s));
    CKS(stage_in(vt, level_n(C), t2, dvt, s));
    OutStage ox, ow;
    CKS(stage_out(x, level_n(L), ox));
    CKS(stage_out(w, level_n(L), ow));
    CKS(precision == 0 ? op_interp_t<double>(*H, level - 1, dv, dvt, ox.dev, ow.dev, s)
                       : op_interp_t<float>(*H, level - 1, dv, dvt, ox.dev, ow.dev, s));
    CKS(finish_out(ox, s));
    return finish_out(ow, s);
}

}  // extern "C"

// x = sigma v - Z sum_m y_m vt_m and w = A x with the types of the solve: T throughout, or
// (DF) level 1 of the mixed solve (v and w double-float pairs, x and vt FP32)
template <typename T, bool DF>
static mk_status op_interp_comb_t(Hierarchy &H, int l, const double *dv, double sigma,
                                  const double *dvt, int nvt, const double *y, double *dx,
                                  double *dw, cudaStream_t s) {
    using Tv = typename std::conditional<DF, float2, T>::type;
    Level &L = *H.lv[l];
    Level &C = *H.lv[l + 1];
    DevMem vp, cp, xp, wp, sg, yd;
    CK(vp.alloc(sizeof(Tv) * L.g.len));
    CK(cp.alloc(sizeof(T) * C.g.len * nvt));
    CK(xp.alloc(sizeof(T) * L.g.len));
    CK(wp.alloc(sizeof(Tv) * L.g.len));
    CK(sg.alloc(sizeof(double)));
    CK(cudaMemcpyAsync(sg.p, &sigma, sizeof(double), cudaMemcpyHostToDevice, s));
    if (y) {
        CK(yd.alloc(sizeof(double) * nvt));
        CK(cudaMemcpyAsync(yd.p, y, sizeof(double) * nvt, cudaMemcpyHostToDevice, s));
    }
    const double *ydev = y ? yd.as<double>() : nullptr;
    launch_pack<double, Tv>(L.g, dv, vp.as<Tv>(), s);
    for (int m = 0; m < nvt; ++m)
        launch_pack<double, T>(C.g, dvt + (size_t)m * level_n(C), cp.as<T>() + (int64_t)m * C.g.len, s);
    if constexpr (DF) {
        const int64_t nc = 3 * (int64_t)L.g.nx + (L.g.dim == 2 ? 3 * (int64_t)L.g.ny : 0);
        const float2 *ca = L.cdf.as<float2>();
        launch_interp_df(L.g, C.g, L.nu, L.space, ca, ca + nc, L.w.b != 0.0, vp.as<float2>(),
                         sg.as<double>(), cp.as<float>(), nvt, C.g.len, ydev, xp.as<float>(),
                         wp.as<float2>(), nullptr, s, L.cuni.p ? L.cuni.as<float2>() : nullptr,
                         L.cuni_square);
    } else {
        launch_interp<T, T, T, T, T>(L.g, C.g, L.nu, L.space, L.w, op_of<T>(L), vp.as<T>(),
                                     sg.as<double>(), cp.as<T>(), nvt, C.g.len, ydev, xp.as<T>(),
                                     wp.as<T>(), nullptr, s);
    }
    launch_unpack<T, double>(L.g, xp.as<T>(), dx, s);
    launch_unpack<Tv, double>(L.g, wp.as<Tv>(), dw, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return MK_OK;
}

extern "C" {

mk_status mk_op_interp_combine(mk_problem *p, const mk_solve_opts *opts, int32_t level,
                               int32_t precision, const double *v, double sigma,
                               const double *vt, int32_t nvt, const double *y, double *x,
                               double *w, void *stream) {
    if (!v || !vt || !x || !w || precision < 0 || precision > 2) return MK_ERR_INVALID;
    if (nvt < 1 || nvt > MK_MAX_INNER || (!y && nvt != 1)) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Hierarchy *H = nullptr;
    mk_solve_opts o;
    CKS(get_level(p, opts, level, H, o));
    if (o.transfer != MK_TRANSFER_MK) return MK_ERR_INVALID;
    if (level >= (int)H->lv.size()) return MK_ERR_INVALID;
    if (precision == 2 && (level != 1 || o.precision != 1)) return MK_ERR_INVALID;
    Level &L = *H->lv[level - 1];
    Level &C = *H->lv[level];
    DevMem t1, t2;
    const double *dv = nullptr, *dvt = nullptr;
    CKS(stage_in(v, level_n(L), t1, dv, s));
    CKS(stage_in(vt, level_n(C) * (size_t)nvt, t2, dvt, s));
    OutStage ox, ow;
    CKS(stage_out(x, level_n(L), ox));
    CKS(stage_out(w, level_n(L), ow));
    if (precision == 0)
        CKS((op_interp_comb_t<double, false>(*H, level - 1, dv, sigma, dvt, nvt, y, ox.dev, ow.dev, s)));
    else if (precision == 1)
        CKS((op_interp_comb_t<float, false>(*H, level - 1, dv, sigma, dvt, nvt, y, ox.dev, ow.dev, s)));
    else
        CKS((op_interp_comb_t<float, true>(*H, level - 1, dv, sigma, dvt, nvt, y, ox.dev, ow.dev, s)));
    CKS(finish_out(ox, s));
    return finish_out(ow, s);
}

}  // extern "C"

template <typename T>
static mk_status op_coarsest_t(Hierarchy &H, const double *dr, double *dx, cudaStream_t s) {
    Level &C = *H.lv.back();
    DevMem rp, xp, al, ga, bi, sx, sxi, lx, sy, syi, ly;
    CK(rp.alloc(sizeof(T) * C.g.len));
    CK(xp.alloc(sizeof(T) * C.g.len));
    launch_pack<double, T>(C.g, dr, rp.as<T>(), s);
    // tables in the requested precision (the hierarchy holds them in its own precision)
    SpaceOp<T> op = op_of<T>(C);
    auto up = [&](DevMem &m, const std::vector<double> &h) -> cudaError_t {
        std::vector<T> t(h.begin(), h.end());
        cudaError_t e = m.alloc(sizeof(T) * t.size());
        if (e == cudaSuccess) e = cudaMemcpy(m.p, t.data(), sizeof(T) * t.size(), cudaMemcpyHostToDevice);
        return e;
    };
    if constexpr (std::is_same<T, float>::value) {
        // the sine-transform slab solver where it applies (as in the solve)
        Level D;
        D.g = C.g;
        D.w = C.w;
        D.Lx = C.Lx;
        mk_status st = build_dst_tables(D, H.key.n_cgs);
        if (st != MK_OK) return st;
        if (D.dstN2 > 0) {
            launch_slab_1d_dst(D.g, D.dst.as<float>(), D.dsttw.as<float2>(), D.dstN2, H.key.n_cgs,
                               D.dstbuf.as<float>(), D.dstld, rp.as<float>(), xp.as<float>(),
                               nullptr, s);
            launch_unpack<float, double>(C.g, xp.as<float>(), dx, s);
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(s));
            return MK_OK;
        }
    }
    if (C.g.dim == 1) {
        std::vector<double> a1, g1, b1;
        pcr_tables(C.Lx, C.w.a, C.npad, a1, g1, b1);
        if (a1.empty()) {
            a1.assign(C.npad, 0.0);
            g1.assign(C.npad, 0.0);
        }
        CK(up(al, a1));
        CK(up(ga, g1));
        CK(up(bi, b1));
        if (slab_warp_supported<T>(C.g.nx)) {
            const int U = spike_block_size(C.g.nx);
            std::vector<double> tab;
            spike_tables(C.Lx, C.w.a, U, spike_threads(C.g.nx), tab);
            DevMem sp;
            CK(up(sp, tab));
            launch_slab_1d_warp<T>(C.g, C.w.b, sp.as<T>(), U, H.key.n_cgs, rp.as<T>(), xp.as<T>(),
                                   nullptr, s, PROF_SLAB);
            launch_unpack<T, double>(C.g, xp.as<T>(), dx, s);
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(s));
            return MK_OK;
        }
        launch_slab_1d<T>(C.g, C.w.b, op, al.as<T>(), ga.as<T>(), bi.as<T>(), C.npad, C.nlev,
                          H.key.n_cgs, rp.as<T>(), xp.as<T>(), nullptr, s);
    } else {
        std::vector<double> lx1, Sx1, Sxi1, ly1, Sy1, Syi1;
        tri_eigen(C.Lx, lx1, Sx1, Sxi1);
        tri_eigen(C.Ly, ly1, Sy1, Syi1);
        CK(up(sx, Sx1));
        CK(up(sxi, Sxi1));
        CK(up(lx, lx1));
        CK(up(sy, Sy1));
        CK(up(syi, Syi1));
        CK(up(ly, ly1));
        DevMem rh;
        CK(rh.alloc(sizeof(T) * (size_t)(C.g.nt + 1) * C.g.nx * C.g.ny));
        launch_slab_2d_fdm<T>(C.g, C.w.a, C.w.b, sx.as<T>(), sxi.as<T>(), lx.as<T>(), sy.as<T>(),
                              syi.as<T>(), ly.as<T>(), H.key.n_cgs, rh.as<T>(), rp.as<T>(),
                              xp.as<T>(), nullptr, s);
        CK(cudaStreamSynchronize(s));   // rh is released at the end of this scope
    }
    launch_unpack<T, double>(C.g, xp.as<T>(), dx, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return MK_OK;
}

extern "C" {

mk_status mk_op_coarsest(mk_problem *p, const mk_solve_opts *opts, int32_t precision,
                         const double *r, double *x, void *stream) {
    if (!r || !x || (precision != 0 && precision != 1)) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Hierarchy *H = nullptr;
    mk_solve_opts o;
    CKS(get_level(p, opts, 1, H, o));
    Level &C = *H->lv.back();
    DevMem t1;
    const double *dr = nullptr;
    CKS(stage_in(r, level_n(C), t1, dr, s));
    OutStage ox;
    CKS(stage_out(x, level_n(C), ox));
    CKS(precision == 0 ? op_coarsest_t<double>(*H, dr, ox.dev, s)
                       : op_coarsest_t<float>(*H, dr, ox.dev, s));
    return finish_out(ox, s);
}

mk_status mk_op_precond(mk_problem *p, const mk_solve_opts *opts, int32_t level, const double *v,
                        double *x, void *stream) {
    if (!v || !x) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Hierarchy *H = nullptr;
    mk_solve_opts o;
    CKS(get_level(p, opts, level, H, o));
    if (level >= (int)H->lv.size()) return MK_ERR_INVALID;
    Level &L = *H->lv[level - 1];
    DevMem t1;
    const double *dv = nullptr;
    CKS(stage_in(v, level_n(L), t1, dv, s));
    OutStage ox;
    CKS(stage_out(x, level_n(L), ox));
    // v -> basis slot 0 of level l with sigma_0 = 1; flags cleared (not done)
    const bool l0 = level == 1;
    if (H->precision == 0) launch_pack<double, double>(L.g, dv, L.V.as<double>(), s);
    else if (l0 && H->precision == 1) launch_pack<double, float2>(L.g, dv, L.V.as<float2>(), s);   // double-float basis
    else launch_pack<double, float>(L.g, dv, L.V.as<float>(), s);
    double one = 1.0;
    CK(cudaMemcpyAsync(L.ks.sigma(), &one, sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(L.ks.flags, 0, sizeof(int) * 8, s));
    enqueue_cycle_step(*H, level - 1, 0, L.ks.flags, s);
    if (H->precision == 0 || l0) {
        if (H->precision == 0) launch_unpack<double, double>(L.g, L.X.as<double>(), ox.dev, s);
        else launch_unpack<float, double>(L.g, L.X.as<float>(), ox.dev, s);
    } else {
        launch_unpack<float, double>(L.g, L.X.as<float>(), ox.dev, s);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return finish_out(ox, s);
}

mk_status mk_op_orthogonalize(mk_problem *p, int32_t j, const double *V, double *w, double *h,
                              void *stream) {
    if (!p || j < 1 || j > MK_MAX_RESTART || !V || !w || !h) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Problem &P = p->P;
    const Geom &g = P.g;
    size_t n = st_n(P);
    DevMem tV, tw, Vp, ksd, ksf;
    const double *dV = nullptr, *dw = nullptr;
    CKS(stage_in(V, n * j, tV, dV, s));
    CKS(stage_in(w, n, tw, dw, s));
    OutStage ow;
    CKS(stage_out(w, n, ow));
    CKS(ensure_device());
    // basis (j vectors) followed by w, all padded
    CK(Vp.alloc(sizeof(double) * g.len * (j + 1)));
    for (int i = 0; i < j; ++i)
        launch_pack<double, double>(g, dV + (size_t)i * n, Vp.as<double>() + (int64_t)i * g.len, s);
    DevMem Wp;
    CK(Wp.alloc(sizeof(double) * g.len));
    launch_pack<double, double>(g, dw, Wp.as<double>(), s);
    KState ks;
    ks.m = j + 1;
    CK(ksd.alloc(sizeof(double) * KState::ndoubles(ks.m)));
    CK(ksf.alloc(sizeof(int) * 8));
    ks.d = ksd.as<double>();
    ks.flags = ksf.as<int>();
    std::vector<double> ones(j + 1, 1.0);
    CK(cudaMemcpyAsync(ks.sigma(), ones.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, s));
    DevMem part, cnt;
    ReduceScratch rs;
    rs.max_blocks = 65536;
    CK(part.alloc(sizeof(double) * rs.max_blocks * (j + 3)));
    CK(cnt.alloc(sizeof(unsigned) * 16));
    rs.partials = part.as<double>();
    rs.counter = cnt.as<unsigned>();
    // first pass; second pass forced (CGS2)
    launch_multidot<double, double>(g.len, Wp.as<double>(), Vp.as<double>(), g.len, j - 1, rs, ks,
                                    false, nullptr, s);
    launch_update<double, double>(g.len, Wp.as<double>(), Vp.as<double>(), g.len, j - 1, true, rs,
                                  ks, UPD_REORTH, false, nullptr, s);
    int one = 1;
    CK(cudaMemcpyAsync(ks.flags + 2, &one, sizeof(int), cudaMemcpyHostToDevice, s));
    launch_multidot<double, double>(g.len, Wp.as<double>(), Vp.as<double>(), g.len, j - 1, rs, ks,
                                    true, nullptr, s);
    launch_update<double, double>(g.len, Wp.as<double>(), Vp.as<double>(), g.len, j - 1, true, rs,
                                  ks, 0, true, nullptr, s);
    // w <- V_j / ||V_j||  (normalised output)
    std::vector<double> hH((size_t)(ks.m + 1) * ks.m);
    std::vector<double> sig(ks.m + 1);
    CK(cudaMemcpyAsync(hH.data(), ks.H(), sizeof(double) * hH.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(sig.data(), ks.sigma(), sizeof(double) * sig.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double *col = hH.data() + (size_t)(j - 1) * (ks.m + 1);
    for (int i = 0; i <= j; ++i) h[i] = col[i];
    // scale V_j on the device by sigma_j via a pack of the unpacked vector
    DevMem tmpd;
    CK(tmpd.alloc(sizeof(double) * n));
    launch_unpack<double, double>(g, Vp.as<double>() + (int64_t)j * g.len, tmpd.as<double>(), s);
    std::vector<double> hv(n);
    CK(cudaMemcpyAsync(hv.data(), tmpd.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (size_t e = 0; e < n; ++e) hv[e] *= sig[j];
    CK(cudaMemcpy(ow.dev, hv.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    return finish_out(ow, s);
}

mk_status mk_op_lsq(int32_t j, const double *H, double beta, double *y, double *res, void *stream) {
    if (j < 1 || j > MK_MAX_RESTART || !H || !y) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    CKS(ensure_device());
    DevMem dH, dg, dy, dr;
    size_t nh = (size_t)(j + 1) * j;
    CK(dH.alloc(sizeof(double) * nh));
    CK(dg.alloc(sizeof(double) * (j + 1)));
    CK(dy.alloc(sizeof(double) * j));
    CK(dr.alloc(sizeof(double)));
    CK(cudaMemcpyAsync(dH.p, H, sizeof(double) * nh, is_device_ptr(H) ? cudaMemcpyDeviceToDevice
                                                                      : cudaMemcpyHostToDevice, s));
    launch_lsq(j, dH.as<double>(), beta, dg.as<double>(), dy.as<double>(), dr.as<double>(), s);
    CK(cudaGetLastError());
    double hr = 0.0;
    std::vector<double> hy(j);
    CK(cudaMemcpyAsync(hy.data(), dy.p, sizeof(double) * j, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&hr, dr.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (is_device_ptr(y)) CK(cudaMemcpy(y, hy.data(), sizeof(double) * j, cudaMemcpyHostToDevice));
    else std::memcpy(y, hy.data(), sizeof(double) * j);
    if (res) *res = hr;
    return MK_OK;
}

mk_status mk_create_batch(mk_problem *const *problems, int32_t count, const mk_solve_opts *opts,
                          int32_t autotune, mk_batch **out) {
    if (!problems || !out || count < 1) return MK_ERR_INVALID;
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        if (!problems[i]) return MK_ERR_INVALID;
        for (int k = 0; k < i; ++k)
            if (problems[k] == problems[i]) return MK_ERR_INVALID;   // one hierarchy each
    }
    CKS(ensure_device());
    std::unique_ptr<mk_batch> b(new mk_batch());
    b->probs.assign(problems, problems + count);
    cudaStream_t s0 = nullptr;
    for (int i = 0; i < count; ++i) {
        mk_solve_opts o = resolve_opts(opts ? &opts[i] : nullptr);
        Problem &P = problems[i]->P;
        CKS(validate_opts(P, o));
        if (o.transfer != MK_TRANSFER_MK) return MK_ERR_INVALID;   // batches: block transfers
        // members run concurrently on graph branches: a cooperative kernel sized to the whole
        // GPU must not overlap other work, so the inner levels take separate launches here
        if (o.inner_kernel == MK_INNER_COOP || o.augment > 0) return MK_ERR_INVALID;
        o.inner_kernel = MK_INNER_SEPARATE;
        std::unique_ptr<Hierarchy> H;
        CKS(build_hierarchy_new(P, o, H));
        if (autotune) CKS(autotune_hierarchy(*H, s0));
        b->opts.push_back(o);
        b->H.push_back(std::move(H));
    }
    CK(cudaStreamSynchronize(s0));
    b->streams.assign(count + 1, nullptr);
    for (auto &st : b->streams) CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    std::vector<Problem *> P;
    std::vector<Hierarchy *> H;
    std::vector<const int *> fp;
    std::vector<const double *> mp;
    for (int i = 0; i < count; ++i) {
        P.push_back(&problems[i]->P);
        H.push_back(b->H[i].get());
        fp.push_back(b->H[i]->lv[0]->ks.flags);
        mp.push_back(b->H[i]->lv[0]->ks.misc());
    }
    CKS(capture_batch(P, H, b->streams, b->graph, b->graph_kernels));
    CK(b->flagptrs.alloc(sizeof(void *) * count));
    CK(b->miscptrs.alloc(sizeof(void *) * count));
    CK(cudaMemcpy(b->flagptrs.p, fp.data(), sizeof(void *) * count, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->miscptrs.p, mp.data(), sizeof(void *) * count, cudaMemcpyHostToDevice));
    CK(b->gflags.alloc(sizeof(int) * 8 * count));
    CK(b->gmisc.alloc(sizeof(double) * 8 * count));
    b->one.assign(count, 1);
    *out = b.release();
    return MK_OK;
}

mk_status mk_solve_batch(mk_batch *b, const double *const *u0, double *const *u_out,
                         mk_solve_info *infos, void *stream) {
    if (!b || !u0 || !u_out) return MK_ERR_INVALID;
    const int n = (int)b->probs.size();
    for (int i = 0; i < n; ++i)
        if (!u0[i] || !u_out[i]) return MK_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t launches_start = mk_kernel_launch_count();
    // right-hand sides (f = source blocks, f_0 = u0) and r_0 = f for every problem
    std::vector<OutStage> os(n);
    {
        std::vector<DevMem> tin(n);
        for (int i = 0; i < n; ++i) {
            Problem &P = b->probs[i]->P;
            Hierarchy &H = *b->H[i];
            const double *du0 = nullptr;
            CKS(stage_in(u0[i], space_n(P), tin[i], du0, s));
            CKS(stage_out(u_out[i], st_n(P), os[i]));
            CK(cudaMemcpyAsync(H.f.p, P.fsrc.p, sizeof(double) * P.g.len, cudaMemcpyDeviceToDevice, s));
            Geom g0 = P.g;
            g0.nt = 0;
            launch_pack<double, double>(g0, du0, H.f.as<double>(), s);
            CKS(solve_prepare(H, b->opts[i], s));
        }
        CK(cudaStreamSynchronize(s));   // before the staging buffers are released
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));
    std::vector<int> hf(8 * (size_t)n);
    std::vector<double> hm(8 * (size_t)n);
    std::vector<mk_status> st(n, MK_OK);
    std::vector<int> finished(n, 0), cycles(n, 0);
    int max_cycles = 0;
    for (int i = 0; i < n; ++i)
        max_cycles = std::max(max_cycles, b->opts[i].max_iters / std::max(1, b->opts[i].restart) + 2);
    for (int c = 0; c < max_cycles; ++c) {
        CK(cudaGraphLaunch(b->graph, s));
        add_launches(b->graph_kernels);
        k_gather_status<<<(n + 127) / 128, 128, 0, s>>>(b->flagptrs.as<const int *>(),
                                                        b->miscptrs.as<const double *>(), n,
                                                        b->gflags.as<int>(), b->gmisc.as<double>());
        count_launch();
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(hf.data(), b->gflags.p, sizeof(int) * 8 * n, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hm.data(), b->gmisc.p, sizeof(double) * 8 * n, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        int left = 0;
        for (int i = 0; i < n; ++i) {
            if (finished[i]) continue;
            ++cycles[i];
            const int *f = &hf[8 * (size_t)i];
            bool stop = false;
            if (f[3]) {
                st[i] = MK_ERR_NONFINITE;
                stop = true;
            } else if (f[0]) {
                finished[i] = 1;   // converged: its kernels exit early from now on
            } else if (f[4] >= b->opts[i].max_iters) {
                st[i] = MK_ERR_NOT_CONVERGED;
                stop = true;
            }
            if (stop) {
                // freeze this problem: its done flag stops its branch in later replays
                finished[i] = 1;
                CK(cudaMemcpyAsync(b->H[i]->lv[0]->ks.flags, &b->one[i], sizeof(int),
                                   cudaMemcpyHostToDevice, s));
            }
            if (!finished[i]) ++left;
        }
        if (left == 0) break;
    }
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    mk_status result = MK_OK;
    for (int i = 0; i < n; ++i) {
        if (!finished[i] && st[i] == MK_OK) st[i] = MK_ERR_NOT_CONVERGED;
        Problem &P = b->probs[i]->P;
        launch_unpack<double, double>(P.g, b->H[i]->u.as<double>(), os[i].dev, s);
        CK(cudaGetLastError());
        CKS(finish_out(os[i], s));
        if (infos) {
            const int *f = &hf[8 * (size_t)i];
            const double *m = &hm[8 * (size_t)i];
            infos[i].iterations = f[4];
            infos[i].restarts = cycles[i];
            infos[i].f_norm = m[3];
            infos[i].rel_residual = m[3] > 0.0 ? m[4] / m[3] : 0.0;
            infos[i].solve_ms = ms;
            infos[i].kernel_launches = (int32_t)(mk_kernel_launch_count() - launches_start);
            infos[i].levels = (int32_t)b->H[i]->lv.size();
        }
        if (result == MK_OK && st[i] != MK_OK) result = st[i];
    }
    CK(cudaStreamSynchronize(s));
    return result;
}

void mk_destroy_batch(mk_batch *b) { delete b; }

// Allocation-free residual: pointer checks only, then one kernel launch (noalloc.cu).
mk_status mk_op_residual_noalloc(const mk_problem *p, const double *f, const double *u, double *r,
                                 double *rnorm, double *rnorm_steps, void *stream) {
    if (!p || !f || !u || !rnorm) return MK_ERR_INVALID;
    if (!is_device_ptr(f) || !is_device_ptr(u) || !is_device_ptr(rnorm)) return MK_ERR_INVALID;
    if ((r && !is_device_ptr(r)) || (rnorm_steps && !is_device_ptr(rnorm_steps)))
        return MK_ERR_INVALID;
    return residual_noalloc(p->P, f, u, r, rnorm, rnorm_steps, (cudaStream_t)stream);
}

}  // extern "C"
