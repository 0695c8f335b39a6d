// Algorithm 1 (Fisher-BT) on the host, over the device evaluators mle_loglik / mle_eval.
//
// Sec. 2.1: start from the given theta^(0) or the best of the L9 design (Table 1); each
// iteration computes phi = I^-1 grad l, halves phi until the relaxed Armijo condition
//   l(theta + phi) >= l(theta) + c grad l . phi - slack        (Eq. 5, c = slack = 0.001)
// holds, moves theta <- theta + phi and runs the next Fisher scoring iteration; it stops when
// ||grad l||_2 <= 0.001 and shifts to Nelder-Mead when l has been computed more than 60 times or
// grad l more than 20 times.  Nelder-Mead stops when the simplex's l values differ by less
// than 1e-9, then one Fisher evaluation gives I(theta_hat).
//
// Readings where the paper is silent: every mle_loglik or mle_eval call counts as an l call and
// every mle_eval call as a gradient call (the L9 start included); a candidate outside the
// domain or with a non-PD covariance has l = -inf; the shift rule is checked after each Fisher
// iteration; a 3x3 Fisher matrix that is not positive definite shifts at once; Nelder-Mead uses
// coefficients (1, 2, 1/2, 1/2) and an initial simplex of theta and theta + 0.05 theta_i e_i.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "../../include/fbt.h"
#include "fbt_ctx_access.h"

namespace {

// Table 1: weight of the lower corner theta^(l) per parameter (1/2, 5/6 or 1/6).
const double kM = 0.5, kL = 5.0 / 6.0, kU = 1.0 / 6.0;
const double kL9[9][3] = {{kM, kM, kM}, {kM, kL, kL}, {kM, kU, kU}, {kL, kM, kL}, {kL, kL, kU},
                          {kL, kU, kM}, {kU, kM, kU}, {kU, kL, kM}, {kU, kU, kL}};

bool armijo_ok(double ll_new, const fbt_state* st, const double phi[3], const fbt_bt_opts& bt) {
    if (!isfinite(ll_new)) return false;
    const double gphi = st->score[0] * phi[0] + st->score[1] * phi[1] + st->score[2] * phi[2];
    return ll_new - (st->loglik + bt.armijo_c * gphi) >= -bt.slack;
}

// phi = I^-1 g by a 3x3 Cholesky factorisation; false if I is not positive definite.
bool fisher_solve(const double I[9], const double g[3], double phi[3]) {
    double L[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int j = 0; j < 3; ++j) {
        double d = I[3 * j + j];
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        if (!(d > 0.0) || !isfinite(d)) return false;
        L[j][j] = sqrt(d);
        for (int i = j + 1; i < 3; ++i) {
            double s = I[3 * i + j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            L[i][j] = s / L[j][j];
        }
    }
    double y[3];
    for (int i = 0; i < 3; ++i) {
        double s = g[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
        y[i] = s / L[i][i];
    }
    for (int i = 2; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 3; ++k) s -= L[k][i] * phi[k];
        phi[i] = s / L[i][i];
    }
    return true;
}

bool hard_error(fbt_status s) {
    return s == FBT_ERR_CUDA || s == FBT_ERR_OOM || s == FBT_ERR_ARG || s == FBT_ERR_TIMEOUT;
}

// One Fisher scoring iteration at st->theta (l, grad l, I, then phi).
fbt_status fisher_iteration(fbt_ctx* ctx, fbt_state* st, const fbt_bt_opts& bt) {
    double ll, g[3], I[9];
    fbt_status s = mle_eval(ctx, st->theta, &ll, g, I);
    st->n_ll += 1;
    st->n_grad += 1;
    if (s != FBT_OK) {
        st->state = FBT_FAILED;
        return s;
    }
    st->loglik = ll;
    memcpy(st->score, g, sizeof g);
    memcpy(st->fisher, I, sizeof I);
    if (sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) <= bt.grad_tol) {
        st->state = FBT_CONVERGED;
        return FBT_OK;
    }
    double phi[3];
    if (!fisher_solve(I, g, phi)) {
        st->state = FBT_SHIFT;
        return FBT_OK;
    }
    memcpy(st->phi, phi, sizeof phi);
    if (st->n_ll > bt.max_ll_calls || st->n_grad > bt.max_grad_calls) st->state = FBT_SHIFT;
    return FBT_OK;
}

// -l(theta) for Nelder-Mead (minimisation); +inf outside the domain or on failure.
struct NegLL {
    fbt_ctx* ctx;
    fbt_status err = FBT_OK;
    double operator()(const double th[3]) {
        if (!(th[0] > 0 && th[1] > 0 && th[2] > 0)) return INFINITY;
        double ll;
        fbt_status s = mle_loglik(ctx, th, &ll);
        if (hard_error(s)) err = s;
        return (s == FBT_OK && isfinite(ll)) ? -ll : INFINITY;
    }
};

// Nelder-Mead from x0; returns the number of function calls.
int nelder_mead(NegLL& f, const double x0[3], double xbest[3], const fbt_bt_opts& bt) {
    std::vector<std::vector<double>> sx(4, std::vector<double>(x0, x0 + 3));
    for (int i = 0; i < 3; ++i) sx[i + 1][i] += 0.05 * (x0[i] != 0 ? x0[i] : 1.0);
    std::vector<double> fs(4);
    for (int i = 0; i < 4; ++i) fs[i] = f(sx[i].data());
    int calls = 4;
    while (calls < bt.nm_max_calls && f.err == FBT_OK) {
        std::vector<int> ord(4);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return fs[a] < fs[b]; });
        std::vector<std::vector<double>> s2(4);
        std::vector<double> f2(4);
        for (int i = 0; i < 4; ++i) { s2[i] = sx[ord[i]]; f2[i] = fs[ord[i]]; }
        sx = s2;
        fs = f2;
        if (isfinite(fs[3]) && fs[3] - fs[0] < bt.nm_ftol) break;
        double c[3], xr[3], xe[3], xc[3];
        for (int d = 0; d < 3; ++d) c[d] = (sx[0][d] + sx[1][d] + sx[2][d]) / 3.0;
        for (int d = 0; d < 3; ++d) xr[d] = c[d] + (c[d] - sx[3][d]);
        const double fr = f(xr);
        ++calls;
        if (fr < fs[0]) {
            for (int d = 0; d < 3; ++d) xe[d] = c[d] + 2.0 * (c[d] - sx[3][d]);
            const double fe = f(xe);
            ++calls;
            if (fe < fr) { sx[3].assign(xe, xe + 3); fs[3] = fe; }
            else { sx[3].assign(xr, xr + 3); fs[3] = fr; }
        } else if (fr < fs[2]) {
            sx[3].assign(xr, xr + 3);
            fs[3] = fr;
        } else {
            bool ok;
            double fc;
            if (fr < fs[3]) {
                for (int d = 0; d < 3; ++d) xc[d] = c[d] + 0.5 * (xr[d] - c[d]);
                fc = f(xc);
                ++calls;
                ok = fc <= fr;
            } else {
                for (int d = 0; d < 3; ++d) xc[d] = c[d] + 0.5 * (sx[3][d] - c[d]);
                fc = f(xc);
                ++calls;
                ok = fc < fs[3];
            }
            if (ok) {
                sx[3].assign(xc, xc + 3);
                fs[3] = fc;
            } else {
                for (int i = 1; i < 4; ++i) {
                    for (int d = 0; d < 3; ++d) sx[i][d] = sx[0][d] + 0.5 * (sx[i][d] - sx[0][d]);
                    fs[i] = f(sx[i].data());
                    ++calls;
                }
            }
        }
    }
    int best = 0;
    for (int i = 1; i < 4; ++i)
        if (fs[i] < fs[best]) best = i;
    for (int d = 0; d < 3; ++d) xbest[d] = sx[best][d];
    return calls;
}

}  // namespace

extern "C" {

void fbt_default_bt_opts(fbt_bt_opts* o) {
    if (!o) return;
    o->armijo_c = 0.001;
    o->rho = 0.5;
    o->slack = 0.001;
    o->grad_tol = 0.001;
    o->nm_ftol = 1e-9;
    o->max_ll_calls = 60;
    o->max_grad_calls = 20;
    o->nm_max_calls = 1000;
    o->max_halvings = 64;
    o->polish_step = 1e-4;
}

fbt_status fisher_bt_start(fbt_ctx* ctx, const double* theta0, const double* lo, const double* hi,
                           const fbt_bt_opts* bto, fbt_state* st) {
    if (!ctx || !st || (!theta0 && (!lo || !hi))) return FBT_ERR_ARG;
    fbt_bt_opts bt;
    fbt_default_bt_opts(&bt);
    if (bto) bt = *bto;
    memset(st, 0, sizeof *st);
    st->loglik = -INFINITY;
    st->polish_iter = -1;
    if (theta0) {
        memcpy(st->theta, theta0, 3 * sizeof(double));
    } else {
        double best = -INFINITY;
        int arg = 0;
        for (int c = 0; c < 9; ++c) {
            double th[3], ll;
            for (int d = 0; d < 3; ++d) th[d] = kL9[c][d] * lo[d] + (1.0 - kL9[c][d]) * hi[d];
            fbt_status s = mle_loglik(ctx, th, &ll);
            st->n_ll += 1;
            if (hard_error(s)) return s;
            if (s == FBT_OK && ll > best) { best = ll; arg = c; }
        }
        for (int d = 0; d < 3; ++d) st->theta[d] = kL9[arg][d] * lo[d] + (1.0 - kL9[arg][d]) * hi[d];
    }
    st->state = FBT_RUNNING;
    return fisher_iteration(ctx, st, bt);
}

fbt_status fisher_bt_step(fbt_ctx* ctx, fbt_state* st, const fbt_bt_opts* bto) {
    if (!ctx || !st) return FBT_ERR_ARG;
    if (st->state != FBT_RUNNING) return FBT_ERR_STATE;
    fbt_bt_opts bt;
    fbt_default_bt_opts(&bt);
    if (bto) bt = *bto;
    double cand[3];
    bool accepted = false;
    st->halvings = 0;
    for (int it = 0; it <= bt.max_halvings; ++it) {
        for (int d = 0; d < 3; ++d) cand[d] = st->theta[d] + st->phi[d];
        double ll;
        // the accepted candidate is evaluated next by Algorithm 3: keep its partials
        fbt_status s = fbt::loglik_keep_partials(ctx, cand, &ll);
        st->n_ll += 1;
        if (hard_error(s)) return s;
        if (armijo_ok(s == FBT_OK ? ll : -INFINITY, st, st->phi, bt)) { accepted = true; break; }
        for (int d = 0; d < 3; ++d) st->phi[d] *= bt.rho;
        st->halvings += 1;
    }
    if (!accepted) {
        st->state = FBT_FAILED;
        return FBT_OK;
    }
    memcpy(st->theta, cand, sizeof cand);
    st->iter += 1;
    return fisher_iteration(ctx, st, bt);
}

}  // extern "C"

namespace {

// The mixed phase of a run on an FBT_PREC_MIXED context ends when the Fisher direction is small
// against theta, when the stopping or the shift rule holds on a mixed evaluation, or when the
// last line search halved four times or more (the mixed l may then be too coarse for the
// Armijo slack of 0.001).
bool mixed_phase_done(const fbt_state* st, const fbt_bt_opts& bt) {
    if (st->state != FBT_RUNNING) return true;
    if (st->iter > 0 && st->halvings >= 4) return true;
    double rel = 0.0;
    for (int d = 0; d < 3; ++d) rel = fmax(rel, fabs(st->phi[d]) / fabs(st->theta[d]));
    return rel <= bt.polish_step;
}

fbt_status run_steps(fbt_ctx* ctx, fbt_state* st, const fbt_bt_opts& bt, bool mixed_phase) {
    for (int i = 0; i < 200 && st->state == FBT_RUNNING; ++i) {
        if (mixed_phase && mixed_phase_done(st, bt)) return FBT_OK;
        fbt_status s = fisher_bt_step(ctx, st, &bt);
        if (s != FBT_OK) return s;
    }
    return FBT_OK;
}

fbt_status run_algorithm1(fbt_ctx* ctx, const double* theta0, const double* lo, const double* hi,
                          const fbt_bt_opts& bt, fbt_state* st) {
    const double tol0 = fbt_get_mixed_tol(ctx);
    const bool polish = fbt::ctx_is_mixed(ctx) && tol0 > 0.0 && bt.polish_step >= 0.0;
    fbt_status s = fisher_bt_start(ctx, theta0, lo, hi, &bt, st);
    if (s != FBT_OK) return s;
    if (polish) {
        // mixed phase; a failed line search (FBT_FAILED) ends the run as on any context
        if ((s = run_steps(ctx, st, bt, true)) != FBT_OK) return s;
        if (st->state == FBT_FAILED) return FBT_OK;
        // polish: FP64-accurate products from here on, starting with the Fisher scoring
        // iteration at the current theta
        st->polish_iter = st->iter;
        memcpy(st->theta_mixed, st->theta, sizeof st->theta);
        if ((s = fbt_set_mixed_tol(ctx, 0.0)) != FBT_OK) return s;
        st->state = FBT_RUNNING;
        if ((s = fisher_iteration(ctx, st, bt)) != FBT_OK) return s;
    }
    return run_steps(ctx, st, bt, false);
}

// Nelder-Mead from the current theta, then one Fisher evaluation at its result (Sec. 2.1).
fbt_status nelder_mead_phase(fbt_ctx* ctx, fbt_state* st, const fbt_bt_opts& bt) {
    NegLL f{ctx};
    double th[3];
    const int calls = nelder_mead(f, st->theta, th, bt);
    st->n_ll += calls;
    if (f.err != FBT_OK) return f.err;
    memcpy(st->theta, th, sizeof th);
    double ll, g[3], I[9];
    const fbt_status s = mle_eval(ctx, th, &ll, g, I);
    st->n_ll += 1;
    st->n_grad += 1;
    if (s != FBT_OK) {
        st->state = FBT_FAILED;
        return hard_error(s) ? s : FBT_OK;
    }
    st->loglik = ll;
    memcpy(st->score, g, sizeof g);
    memcpy(st->fisher, I, sizeof I);
    st->state = FBT_DONE_NM;
    return FBT_OK;
}

}  // namespace

extern "C" {

fbt_status fisher_bt_run(fbt_ctx* ctx, const double* theta0, const double* lo, const double* hi,
                         const fbt_bt_opts* bto, fbt_state* st) {
    fbt_bt_opts bt;
    fbt_default_bt_opts(&bt);
    if (bto) bt = *bto;
    if (!ctx || !st) return FBT_ERR_ARG;
    const double tol0 = fbt_get_mixed_tol(ctx);
    fbt_status s = run_algorithm1(ctx, theta0, lo, hi, bt, st);
    if (s == FBT_OK && st->state == FBT_SHIFT) s = nelder_mead_phase(ctx, st, bt);
    // a polished mixed run leaves the context at the tolerance it had
    if (fbt::ctx_is_mixed(ctx) && fbt_get_mixed_tol(ctx) != tol0) {
        const fbt_status r = fbt_set_mixed_tol(ctx, tol0);
        if (s == FBT_OK) s = r;
    }
    return s;
}

}  // extern "C"
