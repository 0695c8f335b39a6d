// C ABI of libfbt: context management, the evaluation pipelines of Algorithm 2 (mle_loglik)
// and Algorithm 3 (mle_eval), per-kernel profiling and test hooks.  See include/fbt.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/fbt.h"

#include "fbt_kernels.cuh"
#include "fbt_ctx_access.h"

using namespace fbt;

// ------------------------------------------------------------------------------------------
// profiling
// ------------------------------------------------------------------------------------------
namespace fbt {

struct FamilyStat {
    std::string name;
    long long groups = 0, launches = 0;
    double ms = 0.0, flops = 0.0, bytes = 0.0;
};
struct Pending {
    int fam;
    cudaEvent_t a, b;
    double flops, bytes;
    int launches;
};
struct Profiler {
    std::vector<FamilyStat> fams;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    int family_id(const char* name) {
        for (size_t i = 0; i < fams.size(); ++i)
            if (fams[i].name == name) return (int)i;
        fams.push_back(FamilyStat{name});
        return (int)fams.size() - 1;
    }
    cudaEvent_t get_event() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    void flush() {
        for (auto& p : pending) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p.a, p.b);
            auto& f = fams[p.fam];
            f.groups += 1;
            f.launches += p.launches;
            f.ms += ms;
            f.flops += p.flops;
            f.bytes += p.bytes;
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
    }
    ~Profiler() {
        for (auto& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

void ensure_smem(const void* kernel, int bytes) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> set;
    std::lock_guard<std::mutex> lock(mu);
    int& have = set[kernel];
    if (have >= bytes) return;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess) have = bytes;
}

static thread_local cudaEvent_t tl_start;

void Launcher::begin(const char* family_name) {
    launches_in_group = 0;
    if (prof) {
        family = prof->family_id(family_name);
        tl_start = prof->get_event();
        cudaEventRecord(tl_start, stream);
    }
}

int Launcher::end(double flops, double bytes) {
    cudaError_t e = cudaGetLastError();
    if (prof) {
        cudaEvent_t stop = prof->get_event();
        cudaEventRecord(stop, stream);
        prof->pending.push_back(Pending{family, tl_start, stop, flops, bytes, launches_in_group});
    }
    return (int)e;
}

}  // namespace fbt

// ------------------------------------------------------------------------------------------
// context
// ------------------------------------------------------------------------------------------
struct fbt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    fbt_opts opts;
    Geom g;
    int nstrips = 0;
    bool own_ws = false;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    double *X = nullptr, *Y = nullptr, *Z = nullptr, *vy = nullptr, *vw = nullptr, *bbox = nullptr;
    long long* perm = nullptr;
    ThetaConsts* tc = nullptr;
    QuadTables* qt = nullptr;
    Slots slots{};
    int* status = nullptr;
    EvalOut* out = nullptr;
    double *S = nullptr, *SA = nullptr, *SN = nullptr;
    unsigned char* slices = nullptr;         // digit planes of L (emulated-FP64 tile updates)
    unsigned char* slice_scratch = nullptr;  // digit planes of transform panels / rows
    double* winv = nullptr;                  // inverses of the diagonal factor tiles
    unsigned char* wsl = nullptr;            // their digit planes
    unsigned char* wcs = nullptr;            // their digit planes, column-sliced
    double* yscratch = nullptr;              // two scratch tiles
    double* vx = nullptr;                    // one solved block of a triangular solve
    unsigned long long* tier_counts = nullptr;   // mixed path: tasks per tier (device, 4)
    long long* task_list = nullptr;          // mixed path: classified tasks of the current launch
    unsigned* task_count = nullptr;
    long long task_cap = 0;
    double mixed_tol = 0.0;                  // mixed path: the current tolerance (0: all planes)
    long long spin_budget = 0;               // mbarrier wait limit of the tensor-core kernel (0: default)
    Profiler* prof = nullptr;
    long long launches = 0;
    long long h2d_bytes = 0, d2h_bytes = 0;
    EvalOut host_out{};
    // The S slab holds the Cholesky factor of Sigma(factor_theta) after every successful
    // evaluation; an Algorithm 3 evaluation at the same theta (the Fisher iteration at the point
    // the line search just accepted) reuses it instead of regenerating and refactoring Sigma.
    bool factor_valid = false;
    double factor_theta[3] = {0.0, 0.0, 0.0};
    // SA and SN hold Sigma_alpha, Sigma_nu at partials_theta (written together with Sigma by a
    // line-search evaluation, so that Algorithm 3 at the accepted point generates nothing)
    bool partials_valid = false;
    double partials_theta[3] = {0.0, 0.0, 0.0};
    long long factor_reuses = 0;
    // Launch sequences of the evaluation variants (see Variant), captured once as CUDA graphs
    // and replayed: theta reaches the device through dtheta (copied from pin_theta by the
    // sequence itself), the result comes back into pin_out.
    double* dtheta = nullptr;
    double* pin_theta = nullptr;               // pinned host: sigma^2, alpha, nu, jitter
    EvalOut* pin_out = nullptr;                // pinned host: the result record
    bool graphs = true;
    cudaStream_t side_stream = nullptr;       // the Cholesky's lookahead (emulated path)
    cudaEvent_t side_ev[2] = {nullptr, nullptr};
    cudaStream_t cap_stream = nullptr;        // private stream for captures (the caller's may be
                                              // the legacy default stream, which cannot capture)
    cudaGraphExec_t gexec[5] = {};
    long long glaunches[5] = {};
    int gseen[5] = {};
};

static thread_local std::string tl_cuda_error;

static fbt_status cuda_fail(cudaError_t e, const char* where) {
    tl_cuda_error = std::string(where) + ": " + cudaGetErrorString(e);
    return FBT_ERR_CUDA;
}
namespace fbt {
fbt_status record_cuda_error(cudaError_t e, const char* where) { return cuda_fail(e, where); }
}  // namespace fbt
#define CK(call, where)                                              \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);          \
    } while (0)

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Computes the workspace layout; when base is non-null, also assigns the context's pointers.
static size_t carve(long long n, const fbt_opts& o, char* base, fbt_ctx* c) {
    const int nb = o.nb;
    const long long T = (n + nb - 1) / nb;
    const long long npad = T * nb;
    const long long tiles = T * (T + 1) / 2;
    const int ns = nb / 32;
    const size_t slab = (size_t)tiles * nb * nb * sizeof(double);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align256(off + bytes);
        return base ? base + at : nullptr;
    };
    char* pX = take(npad * 8);
    char* pY = take(npad * 8);
    char* pZ = take(npad * 8);
    char* pvy = take(npad * 8);
    char* pvw = take(npad * 8);
    char* pperm = take((size_t)n * 8);
    char* pbbox = take(4 * 8);
    char* ptc = take(sizeof(ThetaConsts));
    char* pth = take(4 * sizeof(double));                  // theta and jitter for prep_theta
    char* pqt = take(sizeof(QuadTables));
    char* pld = take((size_t)T * 8);
    char* pqf = take((size_t)tiles * 2 * 8);
    char* pdg = take((size_t)T * ns * 5 * 8);
    char* pod = take((size_t)tiles * ns * 3 * 8);
    char* pst = take(sizeof(int) * 4);
    char* ptier = take(4 * sizeof(unsigned long long));
    char* pout = take(sizeof(EvalOut));
    char* pS = take(slab);
    char* pSA = o.with_derivatives ? take(slab) : nullptr;
    char* pSN = o.with_derivatives ? take(slab) : nullptr;
    // emulated FP64: digit planes of every strictly-lower tile of L (kept from the Cholesky for
    // the two-sided transforms), plus scratch for two panels / rows and two diagonal tiles
    const bool emu = o.precision == FBT_PREC_FP64_EMULATED || o.precision == FBT_PREC_MIXED;
    const long long nL = T * (T - 1) / 2 > 0 ? T * (T - 1) / 2 : 1;
    const long long nX = 2 * (T > 1 ? T - 1 : 1) + 6;
    char* psl = emu ? take((size_t)nL * ozaki_tile_bytes()) : nullptr;
    const bool ed = emu && o.with_derivatives;
    char* psx = ed ? take((size_t)nX * ozaki_tile_bytes()) : nullptr;
    char* pwi = ed ? take((size_t)T * nb * nb * sizeof(double)) : nullptr;       // W_k = L_kk^-1
    char* pws = ed ? take((size_t)T * ozaki_tile_bytes()) : nullptr;             // digit planes of W_k
    char* pwc = ed ? take((size_t)T * ozaki_tile_bytes()) : nullptr;             // W_k, column-sliced
    char* pyy = ed ? take((size_t)2 * nb * nb * sizeof(double)) : nullptr;       // two scratch tiles
    char* pvx = ed ? take((size_t)nb * sizeof(double)) : nullptr;                // one solved block
    const bool mix = o.precision == FBT_PREC_MIXED;
    const long long cap = mixed_list_capacity((int)T);
    char* plist = mix ? take((size_t)cap * sizeof(long long)) : nullptr;         // classified tasks
    char* pcount = mix ? take(sizeof(unsigned)) : nullptr;
    if (base && c) {
        c->slices = (unsigned char*)psl;
        c->slice_scratch = (unsigned char*)psx;
        c->winv = (double*)pwi;
        c->wsl = (unsigned char*)pws;
        c->wcs = (unsigned char*)pwc;
        c->yscratch = (double*)pyy;
        c->vx = (double*)pvx;
        c->X = (double*)pX; c->Y = (double*)pY; c->Z = (double*)pZ;
        c->vy = (double*)pvy; c->vw = (double*)pvw;
        c->perm = (long long*)pperm; c->bbox = (double*)pbbox;
        c->tc = (ThetaConsts*)ptc; c->qt = (QuadTables*)pqt;
        c->dtheta = (double*)pth;
        c->slots.logdet = (double*)pld; c->slots.qform = (double*)pqf;
        c->slots.diag = (double*)pdg; c->slots.offd = (double*)pod;
        c->status = (int*)pst; c->out = (EvalOut*)pout;
        c->tier_counts = (unsigned long long*)ptier;
        c->task_list = (long long*)plist;
        c->task_count = (unsigned*)pcount;
        c->task_cap = mix ? cap : 0;
        c->S = (double*)pS; c->SA = (double*)pSA; c->SN = (double*)pSN;
    }
    return off;
}

static bool opts_valid(const fbt_opts& o) {
    return (o.nb == 64 || o.nb == 128) && o.jitter >= 0.0 && isfinite(o.jitter) && o.device >= 0 &&
           (o.precision == FBT_PREC_FP64 ||
            ((o.precision == FBT_PREC_FP64_EMULATED || o.precision == FBT_PREC_MIXED) && o.nb == 128)) &&
           (o.precision != FBT_PREC_MIXED || (o.mixed_tol > 0.0 && o.mixed_tol < 1.0));
}

extern "C" {

void fbt_default_opts(fbt_opts* o) {
    if (!o) return;
    o->jitter = 1e-8;
    o->nb = 128;
    o->reorder = 1;
    o->with_derivatives = 1;
    o->device = 0;
    o->precision = FBT_PREC_FP64;
    o->mixed_tol = 1e-12;
}

size_t fbt_workspace_bytes(long long n, const fbt_opts* opts) {
    fbt_opts o;
    fbt_default_opts(&o);
    if (opts) o = *opts;
    if (o.nb == 0) o.nb = 128;
    if (n < 1 || !opts_valid(o)) return 0;
    return carve(n, o, nullptr, nullptr);
}

static Launcher launcher(fbt_ctx* c) {
    Launcher L;
    L.stream = c->stream;
    L.prof = c->prof;
    L.launches = &c->launches;
    L.spin = c->spin_budget;
    return L;
}

fbt_status fbt_create(fbt_ctx** out, const double* locs, int locs_on_device, const double* z,
                      int z_on_device, long long n, const fbt_opts* opts, void* workspace,
                      size_t workspace_bytes, void* stream) {
    if (!out) return FBT_ERR_ARG;
    *out = nullptr;
    if (!locs || !z || n < 1 || n > (1ll << 31)) return FBT_ERR_ARG;
    fbt_opts o;
    fbt_default_opts(&o);
    if (opts) o = *opts;
    if (o.nb == 0) o.nb = 128;
    if (!opts_valid(o)) return FBT_ERR_ARG;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (o.device >= ndev) return FBT_ERR_ARG;
    CK(cudaSetDevice(o.device), "cudaSetDevice");
    const size_t need = carve(n, o, nullptr, nullptr);
    fbt_ctx* c = new fbt_ctx();
    c->device = o.device;
    c->stream = (cudaStream_t)stream;
    c->opts = o;
    c->g.n = n;
    c->g.nb = o.nb;
    c->g.T = (int)((n + o.nb - 1) / o.nb);
    c->g.npad = (long long)c->g.T * o.nb;
    c->nstrips = strips_per_tile(o.nb);
    if (workspace) {
        if (workspace_bytes < need || ((uintptr_t)workspace & 255)) { delete c; return FBT_ERR_OOM; }
        c->ws = (char*)workspace;
        c->ws_bytes = workspace_bytes;
    } else {
        cudaError_t e = cudaMalloc((void**)&c->ws, need);
        if (e != cudaSuccess) { cudaGetLastError(); delete c; return FBT_ERR_OOM; }
        c->own_ws = true;
        c->ws_bytes = need;
    }
    carve(n, o, c->ws, c);
    c->mixed_tol = o.precision == FBT_PREC_MIXED ? o.mixed_tol : 0.0;
    {
        void* pin = nullptr;
        if (cudaHostAlloc(&pin, 4 * sizeof(double) + sizeof(EvalOut), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            fbt_destroy(c);
            return FBT_ERR_OOM;
        }
        c->pin_theta = (double*)pin;
        c->pin_out = (EvalOut*)(c->pin_theta + 4);
    }
    if (c->winv && c->wsl) {
        if (cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->side_ev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->side_ev[1], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            fbt_destroy(c);
            return FBT_ERR_CUDA;
        }
    }
    // staging inside the (not yet used) Sigma slab: sort keys, raw locations, raw field
    long long npow2 = 1;
    while (npow2 < n) npow2 <<= 1;
    unsigned long long* keys = (unsigned long long*)c->S;
    double* raw_locs = (double*)(keys + npow2);
    double* raw_z = raw_locs + 2 * n;
    fbt_status st = FBT_OK;
    do {
        cudaError_t e;
        e = cudaMemcpyAsync(raw_locs, locs, (size_t)n * 2 * sizeof(double),
                            locs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) { st = cuda_fail(e, "copy locations"); break; }
        e = cudaMemcpyAsync(raw_z, z, (size_t)n * sizeof(double),
                            z_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) { st = cuda_fail(e, "copy field"); break; }
        c->h2d_bytes += (locs_on_device ? 0 : 16ll * n) + (z_on_device ? 0 : 8ll * n);
        e = cudaMemsetAsync(c->tier_counts, 0, 4 * sizeof(unsigned long long), c->stream);
        if (e != cudaSuccess) { st = cuda_fail(e, "clear counters"); break; }
        Launcher L = launcher(c);
        int rc = launch_reorder(L, raw_locs, raw_z, n, c->g.npad, o.reorder, keys, c->bbox, c->X,
                                c->Y, c->Z, c->perm);
        if (rc) { st = cuda_fail((cudaError_t)rc, "reorder"); break; }
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) { st = cuda_fail(e, "reorder sync"); break; }
    } while (0);
    if (st != FBT_OK) { fbt_destroy(c); return st; }
    *out = c;
    return FBT_OK;
}

fbt_status fbt_set_field(fbt_ctx* c, const double* z, int z_on_device) {
    if (!c || !z) return FBT_ERR_ARG;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    double* raw_z = c->vw;    // staging: the w vector is rebuilt by every evaluation
    CK(cudaMemcpyAsync(raw_z, z, (size_t)c->g.n * sizeof(double),
                       z_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream),
       "copy field");
    if (!z_on_device) c->h2d_bytes += 8ll * c->g.n;
    Launcher L = launcher(c);
    int rc = launch_permute_field(L, raw_z, c->perm, c->g.n, c->g.npad, c->Z);
    if (rc) return cuda_fail((cudaError_t)rc, "permute field");
    CK(cudaStreamSynchronize(c->stream), "set_field sync");
    return FBT_OK;
}

static bool theta_ok(const double* th) {
    return th && isfinite(th[0]) && isfinite(th[1]) && isfinite(th[2]) && th[0] > 0 && th[1] > 0 &&
           th[2] > 0;
}

static bool same_theta(const double a[3], const double b[3]) {
    return a[0] == b[0] && a[1] == b[1] && a[2] == b[2];
}

// The inverted diagonal factor tiles, when this context's Cholesky computes them (emulated and
// mixed paths with the derivative workspace; the inverses of the same factor are bitwise equal
// wherever they are computed), else nullptr
static const double* winv_valid(const fbt_ctx* c) {
    return (c->opts.precision != FBT_PREC_FP64 && c->winv && c->wsl && c->g.nb == 128) ? c->winv : nullptr;
}

// The launch sequence of one evaluation depends only on these flags (and the context), not on
// theta, so each variant is captured once as a CUDA graph.
enum Variant : int { V_LOGLIK = 0, V_LOGLIK_KEEP = 1, V_EVAL = 2, V_EVAL_REUSE = 3, V_EVAL_REUSE_PARTIALS = 4 };
struct EvalFlags {
    bool deriv, reuse, have_partials, gen_partials;
    int variant() const {
        if (!deriv) return gen_partials ? V_LOGLIK_KEEP : V_LOGLIK;
        if (!reuse) return V_EVAL;
        return have_partials ? V_EVAL_REUSE_PARTIALS : V_EVAL_REUSE;
    }
};

#define EQ(call, what)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// The digit-plane thresholds of the mixed path at theta.  With tau = mixed_tol * sigma^2 and a
// tile product C -= A B^T over K = 128 whose operand entries are below 2^ea and 2^eb (e = ea + eb):
//   * 1 plane (8-bit digits, truncation below 2^-8 of each row's scale) errs by at most
//     2 * 128 * 2^-8 * 2^e = 2^e per entry: used when e < floor(log2 tau) - 1;
//   * 3 planes (24 bits) err by at most 2^(e - 16): used when e < floor(log2 tau) + 13;
//   * every entry of the product is below 128 * 2^e: skipped when e < floor(log2 tau) - 7.
// So every tile product is computed to within tau / 2 of its exact value.  mixed_tol = 0 (the
// polish phase of Algorithm 1) keeps all 7 planes: the emulated-FP64 arithmetic exactly.
static MixedPolicy mixed_policy(const fbt_ctx* c, const double theta[3]) {
    MixedPolicy pol;
    if (c->opts.precision != FBT_PREC_MIXED || !(c->mixed_tol > 0.0)) return pol;
    const int l2 = (int)floor(log2(c->mixed_tol * theta[0]));
    pol.on = 1;
    pol.e_skip = l2 - 7;
    pol.e_fp32 = l2 - 1;
    pol.e_fp64 = l2 + 13;
    pol.counts = c->tier_counts;
    pol.task_list = c->task_list;
    pol.task_count = c->task_count;
    pol.task_cap = c->task_cap;
    return pol;
}

// Enqueue the device work of one evaluation on c->stream (no host synchronisation).
static fbt_status enqueue_eval(fbt_ctx* c, const EvalFlags& f, const MixedPolicy& pol) {
    Launcher L = launcher(c);
    const Geom& g = c->g;
    int rc = 0;
    EQ(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream), "clear status");
    EQ(cudaMemcpyAsync(c->dtheta, c->pin_theta, 4 * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy theta");
    if ((rc = launch_prep_theta_dev(L, c->dtheta, c->tc, c->qt))) return cuda_fail((cudaError_t)rc, "prep_theta");
    if (!f.have_partials &&
        (rc = launch_generate(L, g, c->X, c->Y, c->tc, c->qt, f.reuse ? nullptr : c->S, c->SA, c->SN, f.gen_partials,
                              c->status)))
        return cuda_fail((cudaError_t)rc, "generate");
    if (!f.reuse && (rc = launch_potrf(L, g, c->S, c->slots.logdet, c->status, c->opts.precision, c->slices, pol, c->winv, c->wsl, c->side_stream, c->side_ev)))
        return cuda_fail((cudaError_t)rc, "potrf");
    EQ(cudaMemcpyAsync(c->vy, c->Z, (size_t)g.npad * 8, cudaMemcpyDeviceToDevice, c->stream), "copy z");
    if ((rc = launch_trsv(L, g, c->S, c->vy, false, winv_valid(c), c->vx))) return cuda_fail((cudaError_t)rc, "trsv forward");
    if (f.deriv) {
        EQ(cudaMemcpyAsync(c->vw, c->vy, (size_t)g.npad * 8, cudaMemcpyDeviceToDevice, c->stream), "copy y");
        if ((rc = launch_trsv(L, g, c->S, c->vw, true, winv_valid(c), c->vx))) return cuda_fail((cudaError_t)rc, "trsv backward");
        if ((rc = launch_qform(L, g, c->SA, c->SN, c->vw, c->slots.qform))) return cuda_fail((cudaError_t)rc, "qform");
        // the off-diagonal product slots are indexed by tile; those of diagonal tiles are never
        // written by the transform and must read as zero in the assembly
        EQ(cudaMemsetAsync(c->slots.offd, 0, (size_t)num_tiles(g.T) * c->nstrips * 3 * sizeof(double), c->stream),
           "clear slots");
        if ((rc = launch_sygst(L, g, c->S, c->SA, c->SN, c->slots.diag, c->slots.offd, c->status,
                               c->opts.precision, c->slices, c->slice_scratch, c->winv, c->wsl,
                               c->yscratch, pol)))
            return cuda_fail((cudaError_t)rc, "sygst");
    }
    if ((rc = launch_assemble(L, g, c->vy, c->slots, f.deriv, c->tc, c->status, c->out)))
        return cuda_fail((cudaError_t)rc, "assemble");
    EQ(cudaMemcpyAsync(c->pin_out, c->out, sizeof(EvalOut), cudaMemcpyDeviceToHost, c->stream), "copy result");
    return FBT_OK;
}

// Run one evaluation's device work: directly the first time a variant is seen (and whenever
// profiling is on or the mixed path bakes a theta-dependent policy into the launches), as a
// captured graph from then on.  A capture that fails switches the context to direct launches.
static fbt_status run_eval(fbt_ctx* c, const EvalFlags& f, const MixedPolicy& pol) {
    const int v = f.variant();
    const bool graphable = c->graphs && !c->prof && !pol.on;
    if (graphable && c->gseen[v] >= 1 && !c->gexec[v]) {
        const long long before = c->launches;
        fbt_status est = FBT_OK;
        cudaGraph_t graph = nullptr;
        if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            c->cap_stream = nullptr;
        const cudaStream_t own = c->stream;
        const cudaError_t eb = c->cap_stream ? cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal)
                                             : cudaErrorInvalidResourceHandle;
        if (eb == cudaSuccess) {
            c->stream = c->cap_stream;            // nothing runs while capturing
            est = enqueue_eval(c, f, pol);
            c->stream = own;
            const cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &graph);
            const cudaError_t ei = (est == FBT_OK && ee == cudaSuccess && graph)
                                       ? cudaGraphInstantiate(&c->gexec[v], graph, 0) : cudaErrorUnknown;
            if (ei == cudaSuccess) {
                c->glaunches[v] = c->launches - before;
            } else {
                tl_cuda_error = std::string("graph capture: ") + cudaGetErrorString(ee != cudaSuccess ? ee : ei);
                c->gexec[v] = nullptr;
                c->graphs = false;
            }
            if (graph) cudaGraphDestroy(graph);
        } else {
            tl_cuda_error = std::string("graph capture: ") + cudaGetErrorString(eb);
            c->graphs = false;
        }
        c->launches = before;
        cudaGetLastError();
    }
    c->gseen[v] += 1;
    if (graphable && c->graphs && c->gexec[v]) {
        EQ(cudaGraphLaunch(c->gexec[v], c->stream), "graph launch");
        c->launches += c->glaunches[v];
        return FBT_OK;
    }
    return enqueue_eval(c, f, pol);
}

// Shared pipeline of Algorithms 2 and 3.  keep_partials (Algorithm 2 only): generate Sigma_alpha
// and Sigma_nu together with Sigma (the same exponentials serve all three) and keep them for an
// Algorithm 3 evaluation at the same theta.
static fbt_status evaluate(fbt_ctx* c, const double theta[3], bool deriv, bool keep_partials = false) {
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const bool reuse = deriv && c->factor_valid && same_theta(theta, c->factor_theta);
    const bool have_partials = reuse && c->partials_valid && same_theta(theta, c->partials_theta);
    const bool gen_partials = deriv ? !have_partials : (keep_partials && c->opts.with_derivatives);
    const EvalFlags f{deriv, reuse, have_partials, gen_partials};
    c->factor_valid = false;
    if (deriv || gen_partials) c->partials_valid = false;     // SA, SN are about to change
    const MixedPolicy pol = mixed_policy(c, theta);
    for (int i = 0; i < 3; ++i) c->pin_theta[i] = theta[i];
    c->pin_theta[3] = c->opts.jitter;
    if (reuse) c->factor_reuses += 1;
    fbt_status est = run_eval(c, f, pol);
    if (est != FBT_OK) return est;
    c->h2d_bytes += 4 * (long long)sizeof(double);
    c->d2h_bytes += (long long)sizeof(EvalOut);
    CK(cudaStreamSynchronize(c->stream), "evaluation sync");
    c->host_out = *c->pin_out;
    if (c->prof) c->prof->flush();
    if (c->host_out.status & ST_TIMEOUT) return FBT_ERR_TIMEOUT;
    if (c->host_out.status & ST_NOT_PD) return FBT_ERR_NOT_PD;
    if (c->host_out.status & ST_BESSEL) return FBT_ERR_BESSEL;
    c->factor_valid = true;
    for (int i = 0; i < 3; ++i) c->factor_theta[i] = theta[i];
    if (!deriv && gen_partials) {
        c->partials_valid = true;
        for (int i = 0; i < 3; ++i) c->partials_theta[i] = theta[i];
    }
    return FBT_OK;
}

// Adjoint pipeline: l and grad l through Sigma^-1 (no Fisher information, no stored partials).
static fbt_status evaluate_adjoint(fbt_ctx* c, const double theta[3]) {
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    Launcher L = launcher(c);
    const Geom& g = c->g;
    int rc = 0;
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream), "clear status");
    const bool reuse = c->factor_valid && same_theta(theta, c->factor_theta);
    c->factor_valid = false;
    c->partials_valid = false;            // SA, SN receive L^-1 and Sigma^-1
    const MixedPolicy pol = mixed_policy(c, theta);
    if ((rc = launch_prep_theta(L, theta, c->opts.jitter, c->tc, c->qt))) return cuda_fail((cudaError_t)rc, "prep_theta");
    if (reuse) {
        c->factor_reuses += 1;
    } else {
        if ((rc = launch_generate(L, g, c->X, c->Y, c->tc, c->qt, c->S, nullptr, nullptr, false, c->status)))
            return cuda_fail((cudaError_t)rc, "generate");
        if ((rc = launch_potrf(L, g, c->S, c->slots.logdet, c->status, c->opts.precision, c->slices, pol, c->winv, c->wsl, c->side_stream, c->side_ev)))
            return cuda_fail((cudaError_t)rc, "potrf");
    }
    CK(cudaMemcpyAsync(c->vy, c->Z, (size_t)g.npad * 8, cudaMemcpyDeviceToDevice, c->stream), "copy z");
    if ((rc = launch_trsv(L, g, c->S, c->vy, false, winv_valid(c), c->vx))) return cuda_fail((cudaError_t)rc, "trsv forward");
    CK(cudaMemcpyAsync(c->vw, c->vy, (size_t)g.npad * 8, cudaMemcpyDeviceToDevice, c->stream), "copy y");
    if ((rc = launch_trsv(L, g, c->S, c->vw, true, winv_valid(c), c->vx))) return cuda_fail((cudaError_t)rc, "trsv backward");
    // Sigma^-1 into SN (W = L^-1 in SA on the way)
    // all digit planes: the plane choice is scaled to Sigma's entries, not to its inverse's
    if ((rc = launch_inverse_from_factor(L, g, c->S, c->SA, c->SN, c->status, c->slices, c->slice_scratch,
                                         c->winv, c->wsl, c->wcs, MixedPolicy{})))
        return cuda_fail((cudaError_t)rc, "inverse");
    // the reduction's partials go to the quadratic-form slots; traces and Frobenius slots read 0,
    // so the assembly's score_i = -tr/2 + q/2 is exactly the adjoint sum / 2
    CK(cudaMemsetAsync(c->slots.diag, 0, (size_t)g.T * c->nstrips * 5 * sizeof(double), c->stream), "clear slots");
    CK(cudaMemsetAsync(c->slots.offd, 0, (size_t)num_tiles(g.T) * c->nstrips * 3 * sizeof(double), c->stream),
       "clear slots");
    if ((rc = launch_adjoint_reduce(L, g, c->X, c->Y, c->SN, c->vw, c->tc, c->qt, c->slots.qform, c->status)))
        return cuda_fail((cudaError_t)rc, "adjoint reduce");
    if ((rc = launch_assemble(L, g, c->vy, c->slots, true, c->tc, c->status, c->out)))
        return cuda_fail((cudaError_t)rc, "assemble");
    CK(cudaMemcpyAsync(&c->host_out, c->out, sizeof(EvalOut), cudaMemcpyDeviceToHost, c->stream), "copy result");
    c->d2h_bytes += (long long)sizeof(EvalOut);
    CK(cudaStreamSynchronize(c->stream), "adjoint sync");
    if (c->prof) c->prof->flush();
    if (c->host_out.status & ST_TIMEOUT) return FBT_ERR_TIMEOUT;
    if (c->host_out.status & ST_NOT_PD) return FBT_ERR_NOT_PD;
    if (c->host_out.status & ST_BESSEL) return FBT_ERR_BESSEL;
    c->factor_valid = true;
    for (int i = 0; i < 3; ++i) c->factor_theta[i] = theta[i];
    return FBT_OK;
}

fbt_status mle_loglik_grad(fbt_ctx* c, const double theta[3], double* loglik, double grad[3]) {
    if (!c || !theta || !loglik || !grad) return FBT_ERR_ARG;
    if (!c->opts.with_derivatives || c->g.nb != 128 ||
        (c->opts.precision != FBT_PREC_FP64_EMULATED && c->opts.precision != FBT_PREC_MIXED))
        return FBT_ERR_ARG;
    if (!theta_ok(theta)) { *loglik = -INFINITY; return FBT_ERR_DOMAIN; }
    fbt_status st = evaluate_adjoint(c, theta);
    if (st != FBT_OK) { *loglik = -INFINITY; return st; }
    *loglik = c->host_out.loglik;
    for (int i = 0; i < 3; ++i) grad[i] = c->host_out.score[i];
    return FBT_OK;
}

fbt_status mle_loglik(fbt_ctx* c, const double theta[3], double* loglik) {
    if (!c || !theta || !loglik) return FBT_ERR_ARG;
    if (!theta_ok(theta)) { *loglik = -INFINITY; return FBT_ERR_DOMAIN; }
    fbt_status st = evaluate(c, theta, false);
    *loglik = st == FBT_OK ? c->host_out.loglik : -INFINITY;
    return st;
}

fbt_status mle_eval(fbt_ctx* c, const double theta[3], double* loglik, double score[3],
                    double fisher[9]) {
    if (!c || !theta || !loglik || !score || !fisher) return FBT_ERR_ARG;
    if (!c->opts.with_derivatives) return FBT_ERR_ARG;
    if (!theta_ok(theta)) { *loglik = -INFINITY; return FBT_ERR_DOMAIN; }
    fbt_status st = evaluate(c, theta, true);
    if (st != FBT_OK) { *loglik = -INFINITY; return st; }
    *loglik = c->host_out.loglik;
    for (int i = 0; i < 3; ++i) score[i] = c->host_out.score[i];
    for (int i = 0; i < 9; ++i) fisher[i] = c->host_out.fisher[i];
    return FBT_OK;
}

fbt_status fbt_generate(fbt_ctx* c, const double theta[3], int with_derivatives) {
    if (!c || !theta) return FBT_ERR_ARG;
    if (with_derivatives && !c->opts.with_derivatives) return FBT_ERR_ARG;
    if (!theta_ok(theta)) return FBT_ERR_DOMAIN;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    Launcher L = launcher(c);
    int rc;
    c->factor_valid = false;
    c->partials_valid = false;
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream), "clear status");
    if ((rc = launch_prep_theta(L, theta, c->opts.jitter, c->tc, c->qt))) return cuda_fail((cudaError_t)rc, "prep_theta");
    if ((rc = launch_generate(L, c->g, c->X, c->Y, c->tc, c->qt, c->S, c->SA, c->SN,
                              with_derivatives != 0, c->status)))
        return cuda_fail((cudaError_t)rc, "generate");
    int hs = 0;
    CK(cudaMemcpyAsync(&hs, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "copy status");
    CK(cudaStreamSynchronize(c->stream), "generate sync");
    if (c->prof) c->prof->flush();
    return (hs & ST_BESSEL) ? FBT_ERR_BESSEL : FBT_OK;
}

fbt_status fbt_geometry(fbt_ctx* c, long long* n, long long* npad, int* nb, int* tiles) {
    if (!c) return FBT_ERR_ARG;
    if (n) *n = c->g.n;
    if (npad) *npad = c->g.npad;
    if (nb) *nb = c->g.nb;
    if (tiles) *tiles = c->g.T;
    return FBT_OK;
}

fbt_status fbt_copy_slab(fbt_ctx* c, int which, double* dst, int dst_on_device) {
    if (!c || !dst || which < 0 || which > 2) return FBT_ERR_ARG;
    const double* src = which == 0 ? c->S : which == 1 ? c->SA : c->SN;
    if (!src) return FBT_ERR_ARG;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const size_t bytes = (size_t)num_tiles(c->g.T) * c->g.nb * c->g.nb * sizeof(double);
    CK(cudaMemcpyAsync(dst, src, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->stream), "copy slab");
    CK(cudaStreamSynchronize(c->stream), "copy slab sync");
    return FBT_OK;
}

fbt_status fbt_copy_perm(fbt_ctx* c, long long* perm) {
    if (!c || !perm) return FBT_ERR_ARG;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(perm, c->perm, (size_t)c->g.n * sizeof(long long), cudaMemcpyDeviceToHost, c->stream),
       "copy perm");
    CK(cudaStreamSynchronize(c->stream), "copy perm sync");
    return FBT_OK;
}

fbt_status fbt_set_graphs(fbt_ctx* c, int enable) {
    if (!c) return FBT_ERR_ARG;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(c->stream), "graphs sync");
    for (int v = 0; v < 5; ++v) {
        if (c->gexec[v]) cudaGraphExecDestroy(c->gexec[v]);
        c->gexec[v] = nullptr;
        c->gseen[v] = 0;
    }
    c->graphs = enable != 0;
    return FBT_OK;
}

int fbt_graph_count(fbt_ctx* c) {
    if (!c) return 0;
    int k = 0;
    for (cudaGraphExec_t x : c->gexec) k += x != nullptr;
    return k;
}

fbt_status fbt_set_mixed_tol(fbt_ctx* c, double tol) {
    if (!c || c->opts.precision != FBT_PREC_MIXED || !(tol >= 0.0 && tol < 1.0)) return FBT_ERR_ARG;
    if (tol == c->mixed_tol) return FBT_OK;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(c->stream), "mixed_tol sync");
    // graphs captured under the previous policy would replay it: drop them
    for (int v = 0; v < 5; ++v) {
        if (c->gexec[v]) cudaGraphExecDestroy(c->gexec[v]);
        c->gexec[v] = nullptr;
        c->gseen[v] = 0;
    }
    c->mixed_tol = tol;
    // the kept factor and partials were computed under the previous policy
    c->factor_valid = false;
    c->partials_valid = false;
    return FBT_OK;
}

double fbt_get_mixed_tol(fbt_ctx* c) { return c ? c->mixed_tol : -1.0; }

fbt_status fbt_set_spin_budget(fbt_ctx* c, long long iterations) {
    if (!c) return FBT_ERR_ARG;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(c->stream), "spin budget sync");
    for (int v = 0; v < 5; ++v) {           // captured graphs carry the old budget
        if (c->gexec[v]) cudaGraphExecDestroy(c->gexec[v]);
        c->gexec[v] = nullptr;
        c->gseen[v] = 0;
    }
    c->spin_budget = iterations > 0 ? iterations : 0;
    return FBT_OK;
}

fbt_status fbt_mixed_counts(fbt_ctx* c, long long counts[4], int reset) {
    if (!c || !counts) return FBT_ERR_ARG;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    unsigned long long h[4];
    CK(cudaMemcpyAsync(h, c->tier_counts, sizeof h, cudaMemcpyDeviceToHost, c->stream), "read counters");
    CK(cudaStreamSynchronize(c->stream), "counters sync");
    for (int i = 0; i < 4; ++i) counts[i] = (long long)h[i];
    if (reset) {
        CK(cudaMemsetAsync(c->tier_counts, 0, sizeof h, c->stream), "clear counters");
        CK(cudaStreamSynchronize(c->stream), "counters sync");
    }
    return FBT_OK;
}

fbt_status fbt_profile(fbt_ctx* c, int enable) {
    if (!c) return FBT_ERR_ARG;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(c->stream), "profile sync");
    delete c->prof;
    c->prof = enable ? new Profiler() : nullptr;
    return FBT_OK;
}

fbt_status fbt_profile_read(fbt_ctx* c, fbt_kernel_stat* out, int cap, int* count) {
    if (!c || !count) return FBT_ERR_ARG;
    if (!c->prof) { *count = 0; return FBT_OK; }
    CK(cudaStreamSynchronize(c->stream), "profile sync");
    c->prof->flush();
    const int nf = (int)c->prof->fams.size();
    *count = nf;
    for (int i = 0; i < nf && i < cap && out; ++i) {
        const FamilyStat& f = c->prof->fams[i];
        out[i].name = f.name.c_str();
        out[i].launches = f.groups;
        out[i].ms = f.ms;
        out[i].flops = f.flops;
        out[i].bytes = f.bytes;
    }
    return FBT_OK;
}

long long fbt_factor_reuses(fbt_ctx* c) { return c ? c->factor_reuses : -1; }

fbt_status fbt_transfer_bytes(fbt_ctx* c, long long* h2d, long long* d2h, int reset) {
    if (!c) return FBT_ERR_ARG;
    if (h2d) *h2d = c->h2d_bytes;
    if (d2h) *d2h = c->d2h_bytes;
    if (reset) c->h2d_bytes = c->d2h_bytes = 0;
    return FBT_OK;
}

long long fbt_launch_count(fbt_ctx* c, int reset) {
    if (!c) return -1;
    long long v = c->launches;
    if (reset) c->launches = 0;
    return v;
}

void fbt_destroy(fbt_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (cudaGraphExec_t& x : c->gexec)
        if (x) cudaGraphExecDestroy(x);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side_stream) cudaStreamDestroy(c->side_stream);
    for (cudaEvent_t& e : c->side_ev)
        if (e) cudaEventDestroy(e);
    if (c->pin_theta) cudaFreeHost(c->pin_theta);
    delete c->prof;
    if (c->own_ws && c->ws) cudaFree(c->ws);
    delete c;
}

const char* fbt_strerror(int s) {
    switch (s) {
        case FBT_OK: return "ok";
        case FBT_ERR_DOMAIN: return "parameter outside the domain (theta_i <= 0 or not finite)";
        case FBT_ERR_NOT_PD: return "covariance matrix not positive definite (Cholesky pivot <= 0)";
        case FBT_ERR_BESSEL: return "non-finite covariance entry";
        case FBT_ERR_TIMEOUT: return "bounded device wait expired";
        case FBT_ERR_CUDA: return "CUDA runtime error";
        case FBT_ERR_OOM: return "device memory unavailable or workspace too small";
        case FBT_ERR_ARG: return "invalid argument";
        case FBT_ERR_STATE: return "Fisher-BT state is not running";
        default: return "unknown status";
    }
}

const char* fbt_last_cuda_error(void) { return tl_cuda_error.c_str(); }

}  // extern "C"

namespace fbt {
fbt_status loglik_keep_partials(fbt_ctx* c, const double theta[3], double* loglik) {
    if (!c || !theta || !loglik) return FBT_ERR_ARG;
    if (!theta_ok(theta)) { *loglik = -INFINITY; return FBT_ERR_DOMAIN; }
    fbt_status st = evaluate(c, theta, false, true);
    *loglik = st == FBT_OK ? c->host_out.loglik : -INFINITY;
    return st;
}
cudaStream_t ctx_swap_stream(fbt_ctx* c, cudaStream_t s) {
    cudaStream_t prev = c->stream;
    c->stream = s;
    return prev;
}
int ctx_device(const fbt_ctx* c) { return c->device; }
bool ctx_is_mixed(const fbt_ctx* c) { return c->opts.precision == FBT_PREC_MIXED; }
long long ctx_n(const fbt_ctx* c) { return c->g.n; }
}  // namespace fbt
