// Internal definitions shared by the CUDA translation units of libfbt.
//
// Data layout in HBM (one workspace allocation, carved in fbt_api.cu):
//   * coordinates x[], y[] and field z[] after Z-order reordering, padded to n_pad = T * nb
//   * three lower-tile slabs S, SA, SN (Sigma, Sigma_alpha, Sigma_nu): tile (i, j), i >= j, of
//     T x T tiles of nb x nb doubles, column-major inside the tile, tiles ordered column by
//     column (all tiles of tile-column 0, then tile-column 1, ...).  Padding rows/columns get
//     identity in S and zeros in SA, SN, so the padded problem has the same l, score and Fisher.
//   * vectors y = L^-1 z, w = L^-T y, per-theta constants, quadrature tables, partial-sum
//     slots (reduced in a fixed order, so results are bitwise reproducible), status word and
//     the output record copied back to the host.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fbt {

// ---- status bits set on the device (combined with atomicOr) ----
enum : int { ST_NOT_PD = 1, ST_BESSEL = 2, ST_DOMAIN = 4 };

// ---- trapezoid quadrature of K_nu, K_{nu-1} and dK_nu/dnu (see matern_gen.cu) ----
constexpr int QUAD_LEVELS = 4;
constexpr int QUAD_NODES = 256;

struct ThetaConsts {
    double sigma2, alpha, nu;
    double inv_alpha;
    double norm;     // 1 / (2^(nu-1) Gamma(nu))
    double c_nu;     // log 2 + psi(nu): nu-derivative of log(2^(nu-1) Gamma(nu))
    double jitter;
};

struct QuadTables {
    double st2[QUAD_LEVELS][QUAD_NODES];  // 2 sinh^2(t_j / 2)  (x cosh t = x + x * st2)
    double wa[QUAD_LEVELS][QUAD_NODES];   // w_j cosh(nu t_j)
    double wb[QUAD_LEVELS][QUAD_NODES];   // w_j cosh((nu - 1) t_j)
    double wd[QUAD_LEVELS][QUAD_NODES];   // w_j t_j sinh(nu t_j)
};

// ---- output record of one evaluation (device, copied to the host in one transfer) ----
struct EvalOut {
    double loglik, score[3], fisher[9];
    double logdet, quad, q_alpha, q_nu, t_alpha, t_nu, f_aa, f_an, f_nn;
    int status;
    int pad_;
};

// ---- geometry ----
struct Geom {
    long long n, npad;
    int T, nb;
};

__host__ __device__ inline long long tile_index(int i, int j, int T) {
    return (long long)j * T - (long long)j * (j - 1) / 2 + (i - j);
}
__host__ __device__ inline long long tile_offset(int i, int j, int T, int nb) {
    return tile_index(i, j, T) * (long long)nb * nb;
}
__host__ __device__ inline long long num_tiles(int T) { return (long long)T * (T + 1) / 2; }

// linear index t of the lower triangle (row-major: (0,0),(1,0),(1,1),(2,0),...) -> (r, c), c <= r
__device__ inline void tri_decode(long long t, int& r, int& c) {
    long long rr = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((rr + 1) * (rr + 2) / 2 <= t) ++rr;
    while (rr * (rr + 1) / 2 > t) --rr;
    r = (int)rr;
    c = (int)(t - rr * (rr + 1) / 2);
}

// ---- partial-sum slot layout (doubles) ----
struct Slots {
    double* logdet;     // [T]               sum_j log L_jj of diagonal tile k
    double* qform;      // [ntiles * 2]      w_i^T Sigma_a,b(i,j) w_j per tile (x2 off-diagonal)
    double* diag;       // [T * strips * 5]  tr B_a, tr B_n, <B_a,B_a>, <B_a,B_n>, <B_n,B_n>
    double* offd;       // [ntiles * strips * 3]  <.,.> of off-diagonal tiles (not yet doubled)
};

// ---- launch bookkeeping: launch counter and optional CUDA-event timing per kernel family ----
struct Profiler;
struct Launcher {
    cudaStream_t stream = nullptr;
    Profiler* prof = nullptr;        // non-null while profiling is enabled
    long long* launches = nullptr;   // running count of this library's kernel launches
    int family = -1;
    int launches_in_group = 0;
    void begin(const char* family_name);
    void count(int k = 1) {
        launches_in_group += k;
        if (launches) *launches += k;
    }
    // flops / bytes: algorithmic work of the launches since begin(); returns 0 or a CUDA error code
    int end(double flops, double bytes);
};

// ---- host launchers (one per kernel family), defined next to their kernels ----
int launch_reorder(Launcher& L, const double* locs_dev, const double* z_dev, long long n,
                   long long npad, int reorder, unsigned long long* keys, double* bbox, double* X,
                   double* Y, double* Z, long long* perm);
int launch_permute_field(Launcher& L, const double* z_dev, const long long* perm, long long n,
                         long long npad, double* Z);

int launch_prep_theta(Launcher& L, const double theta[3], double jitter, ThetaConsts* tc,
                      QuadTables* qt);
int launch_generate(Launcher& L, const Geom& g, const double* X, const double* Y,
                    const ThetaConsts* tc, const QuadTables* qt, double* S, double* SA,
                    double* SN, bool deriv, int* status);

// tiled Cholesky of the S slab in place (lower tiles), log-det partials per diagonal tile
int launch_potrf(Launcher& L, const Geom& g, double* S, double* logdet_slots, int* status);
// two-sided transform B = L^-1 M L^-T of both derivative slabs in place, with the trace and
// Frobenius-product partials of the result
int launch_sygst(Launcher& L, const Geom& g, const double* S, double* M0, double* M1,
                 double* diag_slots, double* offd_slots);
int strips_per_tile(int nb);

// v <- L^-1 v (trans = false) or v <- L^-T v (trans = true), tile by tile
int launch_trsv(Launcher& L, const Geom& g, const double* S, double* v, bool trans);
// per-tile partials of w^T M0 w and w^T M1 w over the lower tiles (off-diagonal tiles doubled)
int launch_qform(Launcher& L, const Geom& g, const double* M0, const double* M1, const double* w,
                 double* qform_slots);
int launch_assemble(Launcher& L, const Geom& g, const double* y, const Slots& s, bool deriv,
                    const ThetaConsts* tc, const int* status, EvalOut* out);

}  // namespace fbt
