// Schedule autotuner (mk_tune): the knobs the method leaves free -- the number of decoupled
// coarsest slabs N_CGS (Sec. 3.3.2; 0 = the exact coupled coarse solve of Sec. 3.3.1), the
// restart length of FGMRES (Algorithm 2), the fixed inner iteration counts of the
// intermediate levels (Sec. 4.1) and, on request, the number of time levels -- chosen by
// timing complete solves of the caller's own problem.
//
// Built on the public entry points only (mk_solve, mk_problem_shape): a trial is a solve to
// the base tolerance; a candidate that does not converge within base->max_iters, or that
// the library rejects (MK_ERR_INVALID: a slab count that does not divide the coarsest
// level, too few steps for another level), is skipped.  The search: the level count
// (optional), then up to two passes of coordinate descent over the inner iteration counts
// (deepest level first), N_CGS and the restart length.  Each candidate first runs one
// restart cycle (max_iters 1): the first solve of new options builds their hierarchy,
// autotunes its tiles and captures its graph, all of which would otherwise fall inside
// solve_ms.  The timed solve follows; one within 30% of the best so far is solved once more
// and keeps the faster time.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "mk.h"
#include "mk_internal.h"

namespace {

struct Tuner {
    mk_problem *p;
    const double *u0;
    double *u;       // trial solution buffer (device)
    void *stream;
    int max_trials;
    int trials = 0;
    double best_ms = 1e300;
    int best_it = 0;
    mk_solve_opts best;
    mk_status hard = MK_OK;   // a failure other than "invalid" or "not converged"

    // time of a converged solve with o, or a negative value when the candidate is skipped
    double trial(const mk_solve_opts &o) {
        if (hard != MK_OK || (max_trials > 0 && trials >= max_trials)) return -1.0;
        mk_solve_info info;
        {
            mk_solve_opts w = o;
            w.max_iters = 1;
            const mk_status sw = mk_solve(p, u0, &w, u, &info, stream);
            if (sw == MK_ERR_INVALID || sw == MK_ERR_NONFINITE) return -1.0;
            if (sw != MK_OK && sw != MK_ERR_NOT_CONVERGED) {
                hard = sw;
                return -1.0;
            }
        }
        ++trials;
        mk_status st = mk_solve(p, u0, &o, u, &info, stream);
        if (st == MK_ERR_INVALID || st == MK_ERR_NOT_CONVERGED || st == MK_ERR_NONFINITE) return -1.0;
        if (st != MK_OK) {
            hard = st;
            return -1.0;
        }
        double ms = info.solve_ms;
        int it = info.iterations;
        if (ms < 1.3 * best_ms && (max_trials <= 0 || trials < max_trials)) {
            mk_solve_info i2;
            ++trials;
            st = mk_solve(p, u0, &o, u, &i2, stream);
            if (st != MK_OK) {
                if (st != MK_ERR_NOT_CONVERGED) hard = st;
                return -1.0;
            }
            if (i2.solve_ms < ms) ms = i2.solve_ms;
            it = i2.iterations;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best_it = it;
            best = o;
        }
        return ms;
    }
};

void default_inner(mk_solve_opts &o) {
    // 2 fixed iterations on intermediate levels, 1 on the level above the coarsest (Sec. 4.2)
    for (int l = 0; l + 2 < o.levels; ++l) o.m_inner[l] = (l + 3 == o.levels) ? 1 : 2;
}

}  // namespace

extern "C" mk_status mk_tune(mk_problem *p, const double *u0, const mk_solve_opts *base,
                             int32_t flags, int32_t max_trials, mk_solve_opts *best,
                             mk_tune_info *info, void *stream) {
    if (!p || !u0 || !best) return MK_ERR_INVALID;
    int32_t dim = 0, nx = 0, ny = 0, nt = 0;
    mk_status st = mk_problem_shape(p, &dim, &nx, &ny, &nt, nullptr, nullptr, nullptr);
    if (st != MK_OK) return st;
    mk_solve_opts b;
    if (base) b = *base;
    else mk_default_opts(&b);
    b.autotune = 1;
    const auto t0 = std::chrono::steady_clock::now();
    double *u = nullptr;
    const size_t n = (size_t)nx * (size_t)(dim == 2 ? ny : 1) * (size_t)(nt + 1);
    if (cudaMalloc(&u, sizeof(double) * n) != cudaSuccess) return MK_ERR_NOMEM;
    Tuner T{p, u0, u, stream, max_trials};
    T.best = b;
    // the FP64 path has no parallel-in-time solver for the coupled 1D coarse march (it steps
    // sequentially), so the exact coarse solve is a candidate only in the mixed path and in 2D
    const bool try_exact = !(b.precision == 0 && dim == 1);
    auto ncgs_values = [&](const mk_solve_opts &o) {
        std::vector<int> v = {o.n_cgs, 16, 8, 4, 2, 1};
        if (try_exact) v.push_back(0);
        std::vector<int> u2;
        for (int x : v)
            if (std::find(u2.begin(), u2.end(), x) == u2.end()) u2.push_back(x);
        return u2;
    };
    T.trial(b);
    if (flags & MK_TUNE_LEVELS) {
        for (int L = 2; L < b.levels; ++L) {
            mk_solve_opts o = b;
            o.levels = L;
            default_inner(o);
            o.n_cgs = try_exact ? 0 : b.n_cgs;
            T.trial(o);
        }
    }
    // coordinate descent: inner counts (deepest intermediate level first, +1 then -1), then
    // N_CGS, then the restart length; a second pass when the first improved anything (the
    // knobs interact: a coupled coarse solve pays off only once the level above it iterates
    // enough), within the trial budget
    for (int pass = 0; pass < 2; ++pass) {
        const double start_ms = T.best_ms;
        for (int l = T.best.levels - 3; l >= 0; --l) {
            for (int d : {+1, -1}) {
                const mk_solve_opts c = T.best;
                mk_solve_opts o = c;
                o.m_inner[l] = c.m_inner[l] + d;
                if (o.m_inner[l] < 1 || o.m_inner[l] > mk::MK_MAX_INNER) continue;
                T.trial(o);
            }
        }
        {
            const mk_solve_opts c = T.best;
            for (int v : ncgs_values(c)) {
                if (v == c.n_cgs) continue;
                mk_solve_opts o = T.best;
                o.n_cgs = v;
                T.trial(o);
            }
        }
        {
            const mk_solve_opts c = T.best;
            for (int r : {8, 12, 16, 24, 32, 40, 64}) {
                if (r == c.restart || r > mk::MK_MAX_RESTART) continue;
                if ((flags & MK_TUNE_RESTART_CAP) && r > b.restart) continue;
                mk_solve_opts o = T.best;
                o.restart = r;
                T.trial(o);
            }
        }
        if (!(T.best_ms < start_ms)) break;
    }
    cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(u);
    mk_trim(p);   // the last trial's workspace
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) {
        info->trials = T.trials;
        info->best_iterations = T.best_it;
        info->best_ms = T.best_ms < 1e300 ? T.best_ms : 0.0;
        info->tune_ms = ms;
    }
    if (T.hard != MK_OK) return T.hard;
    *best = T.best;
    return T.best_ms < 1e300 ? MK_OK : MK_ERR_NOT_CONVERGED;
}
