// fbt_loglik_noalloc: Algorithm 2 for small problems without any device allocation.
//
// Some callers cannot allocate device memory when they need a log-likelihood: a process whose
// device memory has been reserved up front by another framework's allocator, or a latency-
// critical loop that must not enter the CUDA allocator (cudaMalloc / cudaFree can synchronise
// the device).  This entry point serves them: all of its scratch (reordered coordinates and
// field, the Sigma tile slab, vectors, partial sums, status and result record) lives in one
// file-scope device array of fixed size, allocated once when the library is loaded and held by
// every GPU that loads it until the process exits.  It runs the same kernels as mle_loglik.
#include <math.h>

#include "../../include/fbt.h"
#include "fbt_ctx_access.h"
#include "fbt_kernels.cuh"

using namespace fbt;

namespace {

constexpr int NA_NB = 64;                         // tile size used by this entry point
constexpr size_t NA_SCRATCH_BYTES = 5u << 20;     // 5 MiB, enough for n <= FBT_NOALLOC_MAX_N

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

constexpr size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

// Bytes of the loglik-only workspace for n points, in the order carve_noalloc takes them
// (constexpr, so that the size bound of FBT_NOALLOC_MAX_N is checked at compile time).
constexpr size_t noalloc_bytes(long long n) {
    const long long T = (n + NA_NB - 1) / NA_NB;
    const size_t npad = (size_t)(T * NA_NB);
    const size_t tiles = (size_t)(T * (T + 1) / 2);
    size_t off = 0;
    const size_t parts[12] = {npad * 8, npad * 8, npad * 8, npad * 8, (size_t)n * 8, 4 * 8,
                              sizeof(ThetaConsts), sizeof(QuadTables), (size_t)T * 8, 4 * sizeof(int),
                              sizeof(EvalOut), tiles * NA_NB * NA_NB * 8};
    for (size_t b : parts) off = a256(off + b);
    return off;
}
static_assert(noalloc_bytes(FBT_NOALLOC_MAX_N) <= NA_SCRATCH_BYTES,
              "the scratch array must hold the workspace of FBT_NOALLOC_MAX_N points");

struct NoallocLayout {
    double *X, *Y, *Z, *vy, *bbox;
    long long* perm;
    ThetaConsts* tc;
    QuadTables* qt;
    Slots slots;
    int* status;
    EvalOut* out;
    double* S;
    size_t bytes;
};

// Carves the loglik-only workspace for n points out of base (same order as noalloc_bytes).
NoallocLayout carve_noalloc(long long n, char* base) {
    const long long T = (n + NA_NB - 1) / NA_NB;
    const long long npad = T * NA_NB;
    const long long tiles = T * (T + 1) / 2;
    size_t off = 0;
    auto take = [&](size_t b) { size_t at = off; off = a256(off + b); return base + at; };
    NoallocLayout L{};
    L.X = (double*)take(npad * 8);
    L.Y = (double*)take(npad * 8);
    L.Z = (double*)take(npad * 8);
    L.vy = (double*)take(npad * 8);
    L.perm = (long long*)take((size_t)n * 8);
    L.bbox = (double*)take(4 * 8);
    L.tc = (ThetaConsts*)take(sizeof(ThetaConsts));
    L.qt = (QuadTables*)take(sizeof(QuadTables));
    L.slots.logdet = (double*)take((size_t)T * 8);
    L.status = (int*)take(4 * sizeof(int));
    L.out = (EvalOut*)take(sizeof(EvalOut));
    L.S = (double*)take((size_t)tiles * NA_NB * NA_NB * 8);
    L.bytes = off;
    return L;
}

// Device address of the scratch array in the current context.  It is looked up on every call,
// not cached: the lookup allocates nothing, and a cached address would be stale after the
// primary context is torn down and created again (cudaDeviceReset), when the module is reloaded.
fbt_status scratch_address(void** ptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return record_cuda_error(e, "noalloc scratch address");
    if (!p) return record_cuda_error(cudaErrorInvalidSymbol, "noalloc scratch address");
    *ptr = p;
    return FBT_OK;
}

}  // namespace

extern "C" {

long long fbt_noalloc_max_n(void) { return FBT_NOALLOC_MAX_N; }

fbt_status fbt_loglik_noalloc(const double* locs, const double* z, int inputs_on_device, long long n,
                              const double theta[3], double jitter, double* loglik, void* stream) {
    if (!locs || !z || !theta || !loglik || n < 1) return FBT_ERR_ARG;
    if (n > FBT_NOALLOC_MAX_N) return FBT_ERR_ARG;
    if (!(jitter >= 0.0) || !isfinite(jitter)) return FBT_ERR_ARG;
    if (!(isfinite(theta[0]) && isfinite(theta[1]) && isfinite(theta[2]) && theta[0] > 0 &&
          theta[1] > 0 && theta[2] > 0)) {
        *loglik = -INFINITY;
        return FBT_ERR_DOMAIN;
    }
    void* base = nullptr;
    fbt_status st = scratch_address(&base);
    if (st != FBT_OK) return st;
    NoallocLayout W = carve_noalloc(n, (char*)base);
    if (W.bytes > NA_SCRATCH_BYTES) return FBT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Geom g;
    g.n = n;
    g.nb = NA_NB;
    g.T = (int)((n + NA_NB - 1) / NA_NB);
    g.npad = (long long)g.T * NA_NB;
    // staging inside the (not yet generated) tile slab: sort keys, raw locations, raw field
    long long npow2 = 1;
    while (npow2 < n) npow2 <<= 1;
    unsigned long long* keys = (unsigned long long*)W.S;
    double* raw_locs = (double*)(keys + npow2);
    double* raw_z = raw_locs + 2 * n;
    const cudaMemcpyKind kind = inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e;
    int rc;
    if ((e = cudaMemcpyAsync(raw_locs, locs, (size_t)n * 16, kind, s)) != cudaSuccess)
        return record_cuda_error(e, "noalloc copy locations");
    if ((e = cudaMemcpyAsync(raw_z, z, (size_t)n * 8, kind, s)) != cudaSuccess)
        return record_cuda_error(e, "noalloc copy field");
    // the array keeps the previous call's contents: the status word must start at zero
    if ((e = cudaMemsetAsync(W.status, 0, sizeof(int), s)) != cudaSuccess)
        return record_cuda_error(e, "noalloc clear status");
    Launcher L;
    L.stream = s;
    if ((rc = launch_reorder(L, raw_locs, raw_z, n, g.npad, 1, keys, W.bbox, W.X, W.Y, W.Z, W.perm)))
        return record_cuda_error((cudaError_t)rc, "noalloc reorder");
    if ((rc = launch_prep_theta(L, theta, jitter, W.tc, W.qt))) return record_cuda_error((cudaError_t)rc, "noalloc prep_theta");
    if ((rc = launch_generate(L, g, W.X, W.Y, W.tc, W.qt, W.S, nullptr, nullptr, false, W.status)))
        return record_cuda_error((cudaError_t)rc, "noalloc generate");
    if ((rc = launch_potrf(L, g, W.S, W.slots.logdet, W.status))) return record_cuda_error((cudaError_t)rc, "noalloc potrf");
    if ((e = cudaMemcpyAsync(W.vy, W.Z, (size_t)g.npad * 8, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return record_cuda_error(e, "noalloc copy field to solve vector");
    if ((rc = launch_trsv(L, g, W.S, W.vy, false))) return record_cuda_error((cudaError_t)rc, "noalloc trsv");
    if ((rc = launch_assemble(L, g, W.vy, W.slots, false, W.tc, W.status, W.out)))
        return record_cuda_error((cudaError_t)rc, "noalloc assemble");
    EvalOut host{};
    if ((e = cudaMemcpyAsync(&host, W.out, sizeof(EvalOut), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return record_cuda_error(e, "noalloc copy result");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return record_cuda_error(e, "noalloc synchronize");
    if (host.status & ST_NOT_PD) { *loglik = -INFINITY; return FBT_ERR_NOT_PD; }
    if (host.status & ST_BESSEL) { *loglik = -INFINITY; return FBT_ERR_BESSEL; }
    *loglik = host.loglik;
    return FBT_OK;
}

}  // extern "C"
