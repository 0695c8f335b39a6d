// Many independent fields (the batched workload): each field keeps its own context, and a pool of
// host threads drives them, every thread on its own CUDA stream, so that the launch-latency-bound
// steps of small fields (diagonal factorisations, strip solves, TRSV) of different fields overlap
// on the GPU while the tile updates of large ones fill it.  Fields are taken largest first
// (longest-processing-time order); nothing is exchanged between fields.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "fbt.h"
#include "fbt_ctx_access.h"

namespace {

bool hard_error(fbt_status s) {
    return s == FBT_ERR_CUDA || s == FBT_ERR_OOM || s == FBT_ERR_TIMEOUT || s == FBT_ERR_ARG ||
           s == FBT_ERR_STATE;
}

// Runs work(f, ctx) once per field; returns the first hard error of any field, else FBT_OK.
template <class Work>
fbt_status run_pool(fbt_ctx* const* ctxs, int nfields, int nthreads, Work&& work) {
    if (nfields < 0 || (nfields > 0 && !ctxs)) return FBT_ERR_ARG;
    if (nfields == 0) return FBT_OK;
    std::vector<fbt_ctx*> uniq(ctxs, ctxs + nfields);
    for (fbt_ctx* c : uniq)
        if (!c) return FBT_ERR_ARG;
    std::sort(uniq.begin(), uniq.end());
    if (std::adjacent_find(uniq.begin(), uniq.end()) != uniq.end()) return FBT_ERR_ARG;   // shared context
    const int device = fbt::ctx_device(ctxs[0]);
    for (int f = 1; f < nfields; ++f)
        if (fbt::ctx_device(ctxs[f]) != device) return FBT_ERR_ARG;
    std::vector<int> order(nfields);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return fbt::ctx_n(ctxs[a]) > fbt::ctx_n(ctxs[b]); });
    if (nthreads <= 0) nthreads = FBT_BATCH_DEFAULT_THREADS;
    nthreads = std::min(nthreads, nfields);
    std::atomic<int> next{0};
    std::atomic<int> first_err{FBT_OK};
    auto body = [&]() {
        if (cudaSetDevice(device) != cudaSuccess) { int z = FBT_OK; first_err.compare_exchange_strong(z, FBT_ERR_CUDA); return; }
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            int z = FBT_OK;
            first_err.compare_exchange_strong(z, FBT_ERR_CUDA);
            if (s) cudaStreamDestroy(s);
            return;
        }
        for (;;) {
            const int q = next.fetch_add(1);
            if (q >= nfields) break;
            const int f = order[q];
            fbt_ctx* c = ctxs[f];
            // the field's work runs on this thread's stream, ordered after and before the
            // context's own stream
            cudaStream_t own = fbt::ctx_swap_stream(c, s);
            cudaEventRecord(ev, own);
            cudaStreamWaitEvent(s, ev, 0);
            const fbt_status st = work(f, c);
            cudaEventRecord(ev, s);
            cudaStreamWaitEvent(own, ev, 0);
            fbt::ctx_swap_stream(c, own);
            if (hard_error(st)) {
                int z = FBT_OK;
                first_err.compare_exchange_strong(z, (int)st);
            }
        }
        cudaStreamSynchronize(s);
        cudaEventDestroy(ev);
        cudaStreamDestroy(s);
    };
    std::vector<std::thread> pool;
    pool.reserve(nthreads);
    for (int t = 0; t < nthreads; ++t) pool.emplace_back(body);
    for (auto& t : pool) t.join();
    return (fbt_status)first_err.load();
}

}  // namespace

extern "C" {

fbt_status mle_eval_batch(fbt_ctx* const* ctxs, int nfields, const double* thetas, int k, int flags,
                          double* out, int* status, int nthreads) {
    if (k < 1 || !thetas || !out || !status || (flags & ~FBT_BATCH_EVAL)) return FBT_ERR_ARG;
    const bool full = flags & FBT_BATCH_EVAL;
    const int stride = full ? 13 : 1;
    return run_pool(ctxs, nfields, nthreads, [&](int f, fbt_ctx* c) {
        fbt_status worst = FBT_OK;
        for (int j = 0; j < k; ++j) {
            const long long u = (long long)f * k + j;
            const double* th = thetas + 3 * u;
            double* o = out + stride * u;
            fbt_status s = full ? mle_eval(c, th, o, o + 1, o + 4) : mle_loglik(c, th, o);
            status[u] = (int)s;
            if (hard_error(s)) return s;
            if (s != FBT_OK) worst = s;
        }
        return worst;
    });
}

fbt_status fisher_bt_start_batch(fbt_ctx* const* ctxs, int nfields, const double* theta0s,
                                 const double* theta_lo, const double* theta_hi, const fbt_bt_opts* bt,
                                 fbt_state* states, int* status, int nthreads) {
    if (!states || !status || (!theta0s && (!theta_lo || !theta_hi))) return FBT_ERR_ARG;
    return run_pool(ctxs, nfields, nthreads, [&](int f, fbt_ctx* c) {
        const double* t0 = theta0s ? theta0s + 3 * (long long)f : nullptr;
        const double* lo = theta_lo ? theta_lo + 3 * (long long)f : nullptr;
        const double* hi = theta_hi ? theta_hi + 3 * (long long)f : nullptr;
        fbt_status s = fisher_bt_start(c, t0, lo, hi, bt, &states[f]);
        status[f] = (int)s;
        return s;
    });
}

fbt_status fisher_bt_step_batch(fbt_ctx* const* ctxs, int nfields, fbt_state* states,
                                const fbt_bt_opts* bt, int* status, int nthreads) {
    if (!states || !status) return FBT_ERR_ARG;
    return run_pool(ctxs, nfields, nthreads, [&](int f, fbt_ctx* c) {
        if (states[f].state != FBT_RUNNING) {       // finished fields are left as they are
            status[f] = (int)FBT_OK;
            return FBT_OK;
        }
        fbt_status s = fisher_bt_step(c, &states[f], bt);
        status[f] = (int)s;
        return s;
    });
}

fbt_status fisher_bt_run_batch(fbt_ctx* const* ctxs, int nfields, const double* theta0s,
                               const double* theta_lo, const double* theta_hi, const fbt_bt_opts* bt,
                               fbt_state* states, int* status, int nthreads) {
    if (!states || !status || (!theta0s && (!theta_lo || !theta_hi))) return FBT_ERR_ARG;
    return run_pool(ctxs, nfields, nthreads, [&](int f, fbt_ctx* c) {
        const double* t0 = theta0s ? theta0s + 3 * (long long)f : nullptr;
        const double* lo = theta_lo ? theta_lo + 3 * (long long)f : nullptr;
        const double* hi = theta_hi ? theta_hi + 3 * (long long)f : nullptr;
        fbt_status s = fisher_bt_run(c, t0, lo, hi, bt, &states[f]);
        status[f] = (int)s;
        return s;
    });
}

// ------------------------------------------------------------------------------------------
// Autotuning.  The choices are measured, not modelled: each candidate runs the same work on the
// caller's data and the fastest wins.
// ------------------------------------------------------------------------------------------
static double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

fbt_status fbt_tune_batch_threads(fbt_ctx* const* ctxs, int nfields, const double* thetas, const int* candidates,
                                  int ncand, int* best, double* seconds) {
    if (!ctxs || nfields < 1 || !thetas || !candidates || ncand < 1 || !best || !seconds) return FBT_ERR_ARG;
    for (int i = 0; i < ncand; ++i)
        if (candidates[i] < 1) return FBT_ERR_ARG;
    std::vector<double> out(nfields);
    std::vector<int> st(nfields);
    // two untimed passes: the first runs each context's launch sequence directly, the second
    // captures it as a graph, later ones replay it (as every timed pass does)
    for (int w = 0; w < 2; ++w) {
        fbt_status s = mle_eval_batch(ctxs, nfields, thetas, 1, FBT_BATCH_LOGLIK, out.data(), st.data(), candidates[0]);
        if (hard_error(s)) return s;
    }
    int arg = 0;
    for (int i = 0; i < ncand; ++i) {
        const auto t0 = std::chrono::steady_clock::now();
        fbt_status s = mle_eval_batch(ctxs, nfields, thetas, 1, FBT_BATCH_LOGLIK, out.data(), st.data(), candidates[i]);
        seconds[i] = seconds_since(t0);           // the batched call returns with every stream idle
        if (hard_error(s)) return s;
        if (seconds[i] < seconds[arg]) arg = i;
    }
    *best = candidates[arg];
    return FBT_OK;
}

namespace {
struct TuneRecord {
    int precision, nb;
    double seconds[2];
};
std::mutex g_tune_mutex;
std::map<std::pair<int, long long>, TuneRecord> g_tune_cache;     // (device, size band) -> choice
}  // namespace

fbt_status fbt_autotune(const double* locs, const double* z, long long n, const double theta[3], int reps,
                        fbt_opts* opts, double seconds[2], int* cached) {
    if (!locs || !z || n < 1 || !theta || !opts || !seconds || reps < 1) return FBT_ERR_ARG;
    if (opts->precision != FBT_PREC_FP64 && opts->precision != FBT_PREC_FP64_EMULATED) return FBT_ERR_ARG;
    long long band = 1;
    while (band < n) band <<= 1;
    const std::pair<int, long long> key{opts->device, band};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            opts->precision = it->second.precision;
            opts->nb = it->second.nb;
            seconds[0] = it->second.seconds[0];
            seconds[1] = it->second.seconds[1];
            if (cached) *cached = 1;
            return FBT_OK;
        }
    }
    // the two FP64-accurate configurations: FP64 DFMA tiles of 64, tensor-core tiles of 128
    const int prec[2] = {FBT_PREC_FP64, FBT_PREC_FP64_EMULATED};
    const int nbs[2] = {64, 128};
    for (int c = 0; c < 2; ++c) {
        fbt_opts o = *opts;
        o.precision = prec[c];
        o.nb = nbs[c];
        fbt_ctx* ctx = nullptr;
        fbt_status s = fbt_create(&ctx, locs, 0, z, 0, n, &o, nullptr, 0, nullptr);
        if (s != FBT_OK) return s;
        double ll, g[3], I[9];
        s = mle_eval(ctx, theta, &ll, g, I);          // untimed: direct launches
        if (hard_error(s)) { fbt_destroy(ctx); return s; }
        s = mle_eval(ctx, theta, &ll, g, I);          // untimed: captures the graph
        if (hard_error(s)) { fbt_destroy(ctx); return s; }
        const auto t0 = std::chrono::steady_clock::now();
        for (int r = 0; r < reps && !hard_error(s); ++r) s = mle_eval(ctx, theta, &ll, g, I);
        seconds[c] = seconds_since(t0) / reps;        // each evaluation synchronises
        fbt_destroy(ctx);
        if (hard_error(s)) return s;
    }
    const int arg = seconds[1] <= seconds[0] ? 1 : 0;
    opts->precision = prec[arg];
    opts->nb = nbs[arg];
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = TuneRecord{prec[arg], nbs[arg], {seconds[0], seconds[1]}};
    if (cached) *cached = 0;
    return FBT_OK;
}

}  // extern "C"
