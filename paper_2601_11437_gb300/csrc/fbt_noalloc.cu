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
#include <mutex>

#include "../../include/fbt.h"
#include "fbt_kernels.cuh"

using namespace fbt;

namespace {

constexpr int NA_NB = 64;                         // tile size used by this entry point
constexpr size_t NA_SCRATCH_BYTES = 5u << 20;     // 5 MiB, enough for n <= FBT_NOALLOC_MAX_N

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[NA_MAX_DEVICES] = {nullptr};

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

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

// Carves the loglik-only workspace for n points out of base (base may be null to size it).
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

// Device address of the scratch array on the current device (set up once per device).
fbt_status scratch_address(int dev, void** ptr) {
    if (dev < 0 || dev >= NA_MAX_DEVICES) return FBT_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return FBT_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *ptr = g_noalloc_ptr[dev];
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
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FBT_ERR_CUDA;
    void* base = nullptr;
    fbt_status st = scratch_address(dev, &base);
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
    if (cudaMemcpyAsync(raw_locs, locs, (size_t)n * 16, kind, s) != cudaSuccess) return FBT_ERR_CUDA;
    if (cudaMemcpyAsync(raw_z, z, (size_t)n * 8, kind, s) != cudaSuccess) return FBT_ERR_CUDA;
    // the array keeps the previous call's contents: the status word must start at zero
    if (cudaMemsetAsync(W.status, 0, sizeof(int), s) != cudaSuccess) return FBT_ERR_CUDA;
    Launcher L;
    L.stream = s;
    if (launch_reorder(L, raw_locs, raw_z, n, g.npad, 1, keys, W.bbox, W.X, W.Y, W.Z, W.perm)) return FBT_ERR_CUDA;
    if (launch_prep_theta(L, theta, jitter, W.tc, W.qt)) return FBT_ERR_CUDA;
    if (launch_generate(L, g, W.X, W.Y, W.tc, W.qt, W.S, nullptr, nullptr, false, W.status)) return FBT_ERR_CUDA;
    if (launch_potrf(L, g, W.S, W.slots.logdet, W.status)) return FBT_ERR_CUDA;
    if (cudaMemcpyAsync(W.vy, W.Z, (size_t)g.npad * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return FBT_ERR_CUDA;
    if (launch_trsv(L, g, W.S, W.vy, false)) return FBT_ERR_CUDA;
    if (launch_assemble(L, g, W.vy, W.slots, false, W.tc, W.status, W.out)) return FBT_ERR_CUDA;
    EvalOut host{};
    if (cudaMemcpyAsync(&host, W.out, sizeof(EvalOut), cudaMemcpyDeviceToHost, s) != cudaSuccess) return FBT_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FBT_ERR_CUDA;
    if (host.status & ST_NOT_PD) { *loglik = -INFINITY; return FBT_ERR_NOT_PD; }
    if (host.status & ST_BESSEL) { *loglik = -INFINITY; return FBT_ERR_BESSEL; }
    *loglik = host.loglik;
    return FBT_OK;
}

}  // extern "C"
