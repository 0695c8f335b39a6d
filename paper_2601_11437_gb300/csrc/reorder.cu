// Step a0: Z-order (Morton) reordering of the locations, padded copy of coordinates and field.
//
// The log-likelihood, score and Fisher information are invariant under a simultaneous
// permutation of locations and observations (Eq. 1-3 only involve Sigma through log det,
// quadratic forms and traces).  Ordering the points along a Z-order curve makes points that are
// close in the list close in space, so a tile of Sigma couples two compact groups of points.
#include "fbt_kernels.cuh"

namespace fbt {

// Bounding box of the n locations (row-major n x 2), one block.
__global__ void __launch_bounds__(1024) k_bbox(const double* __restrict__ locs, long long n,
                                               double* __restrict__ bbox) {
    __shared__ double s[4][1024];
    double mnx = 1e300, mny = 1e300, mxx = -1e300, mxy = -1e300;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        double x = locs[2 * i], y = locs[2 * i + 1];
        mnx = fmin(mnx, x); mxx = fmax(mxx, x);
        mny = fmin(mny, y); mxy = fmax(mxy, y);
    }
    s[0][threadIdx.x] = mnx; s[1][threadIdx.x] = mny;
    s[2][threadIdx.x] = mxx; s[3][threadIdx.x] = mxy;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s[0][threadIdx.x] = fmin(s[0][threadIdx.x], s[0][threadIdx.x + w]);
            s[1][threadIdx.x] = fmin(s[1][threadIdx.x], s[1][threadIdx.x + w]);
            s[2][threadIdx.x] = fmax(s[2][threadIdx.x], s[2][threadIdx.x + w]);
            s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) bbox[threadIdx.x] = s[threadIdx.x][0];
}

__device__ inline uint32_t spread16(uint32_t v) {   // 16 bits -> even bit positions
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

// key = (Morton code of the 16-bit quantised position) << 32 | original index; padding keys sort last.
__global__ void k_morton_keys(const double* __restrict__ locs, long long n, long long npow2,
                              const double* __restrict__ bbox, int reorder,
                              unsigned long long* __restrict__ keys) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= npow2) return;
    if (i >= n) { keys[i] = ~0ull; return; }
    uint32_t code = 0;
    if (reorder) {
        double wx = bbox[2] - bbox[0], wy = bbox[3] - bbox[1];
        double fx = wx > 0 ? (locs[2 * i] - bbox[0]) / wx : 0.0;
        double fy = wy > 0 ? (locs[2 * i + 1] - bbox[1]) / wy : 0.0;
        uint32_t qx = (uint32_t)fmin(fmax(fx * 65535.0, 0.0), 65535.0);
        uint32_t qy = (uint32_t)fmin(fmax(fy * 65535.0, 0.0), 65535.0);
        code = spread16(qx) | (spread16(qy) << 1);
    }
    keys[i] = ((unsigned long long)code << 32) | (unsigned long long)i;
}

// One compare-exchange pass of a bitonic sorting network over npow2 keys.
__global__ void k_bitonic_pass(unsigned long long* __restrict__ keys, long long npow2, long long j,
                               long long k) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= npow2) return;
    long long l = i ^ j;
    if (l <= i) return;
    unsigned long long a = keys[i], b = keys[l];
    bool ascending = (i & k) == 0;
    if ((a > b) == ascending) { keys[i] = b; keys[l] = a; }
}

// Reordered, padded SoA coordinates and field; perm[i] = original index of reordered point i.
__global__ void k_gather(const double* __restrict__ locs, const double* __restrict__ z,
                         const unsigned long long* __restrict__ keys, long long n, long long npad,
                         double* __restrict__ X, double* __restrict__ Y, double* __restrict__ Z,
                         long long* __restrict__ perm) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= npad) return;
    if (i < n) {
        long long p = (long long)(keys[i] & 0xFFFFFFFFull);
        X[i] = locs[2 * p];
        Y[i] = locs[2 * p + 1];
        Z[i] = z[p];
        perm[i] = p;
    } else {
        X[i] = 0.0; Y[i] = 0.0; Z[i] = 0.0;
    }
}

__global__ void k_permute_field(const double* __restrict__ z, const long long* __restrict__ perm,
                                long long n, long long npad, double* __restrict__ Z) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= npad) return;
    Z[i] = i < n ? z[perm[i]] : 0.0;
}

static inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

int launch_reorder(Launcher& L, const double* locs_dev, const double* z_dev, long long n,
                   long long npad, int reorder, unsigned long long* keys, double* bbox, double* X,
                   double* Y, double* Z, long long* perm) {
    long long npow2 = 1;
    while (npow2 < n) npow2 <<= 1;
    L.begin("reorder");
    k_bbox<<<1, 1024, 0, L.stream>>>(locs_dev, n, bbox);
    L.count();
    k_morton_keys<<<blocks_for(npow2, 256), 256, 0, L.stream>>>(locs_dev, n, npow2, bbox, reorder, keys);
    L.count();
    for (long long k = 2; k <= npow2; k <<= 1)
        for (long long j = k >> 1; j > 0; j >>= 1) {
            k_bitonic_pass<<<blocks_for(npow2, 256), 256, 0, L.stream>>>(keys, npow2, j, k);
            L.count();
        }
    k_gather<<<blocks_for(npad, 256), 256, 0, L.stream>>>(locs_dev, z_dev, keys, n, npad, X, Y, Z, perm);
    L.count();
    return L.end(0.0, 0.0);
}

int launch_permute_field(Launcher& L, const double* z_dev, const long long* perm, long long n,
                         long long npad, double* Z) {
    L.begin("permute_field");
    k_permute_field<<<blocks_for(npad, 256), 256, 0, L.stream>>>(z_dev, perm, n, npad, Z);
    L.count();
    return L.end(0.0, 16.0 * n);
}

}  // namespace fbt
