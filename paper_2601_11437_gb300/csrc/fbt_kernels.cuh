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
enum : int { ST_NOT_PD = 1, ST_BESSEL = 2, ST_DOMAIN = 4, ST_TIMEOUT = 8 };

// ---- arithmetic of the tile updates ----
enum : int { PREC_FP64 = 0, PREC_FP64_OZAKI = 1, PREC_MIXED = 2 };

// Mixed path: a tile product with operand maxima 2^ea, 2^eb uses all 7 digit planes
// (FP64-accurate) if ea + eb >= e_fp64, 3 planes (24 bits, FP32-class) if ea + eb >= e_fp32,
// 1 plane (8 bits, BF16-class) if ea + eb >= e_skip, and is skipped (its entries are all below
// the tolerance) otherwise; the thresholds follow from mixed_tol * sigma^2.  counts (optional,
// device): tasks per tier (skipped, 1, 3, 7 planes), accumulated over launches.
struct MixedPolicy {
    int on = 0;
    int e_fp64 = 0, e_fp32 = 0, e_skip = -100000;
    unsigned long long* counts = nullptr;
    // device scratch of the task classification that precedes every mixed launch: the list of
    // tasks that are not skipped, with their tier, and its length (capacity: mixed_list_capacity)
    long long* task_list = nullptr;
    unsigned* task_count = nullptr;
    long long task_cap = 0;
};
// entries of the classified task list a launch over T x T tiles may need (the largest launch is
// the two-sided transform's trailing update of both matrices: 2 m (m + 1) tasks, m < T)
inline long long mixed_list_capacity(int T) { return 2ll * T * (T + 1) + 64; }

// ---- trapezoid quadrature of K_nu, K_{nu-1} and dK_nu/dnu (see matern_gen.cu) ----
constexpr int QUAD_LEVELS = 5;
constexpr int QUAD_NODES = 256;

struct ThetaConsts {
    double sigma2, alpha, nu;
    double inv_alpha;
    double norm;     // 1 / (2^(nu-1) Gamma(nu))
    double c_nu;     // log 2 + psi(nu): nu-derivative of log(2^(nu-1) Gamma(nu))
    double jitter;
};

constexpr int EXP_TABLE = 256;
// Piecewise polynomials of the three smooth sums e^x K_nu(x), e^x K_(nu-1)(x), e^x dK_nu/dnu(x)
// on [1, 1024): each octave [2^s, 2^(s+1)) cut into IP_SUB equal intervals, on each a polynomial of
// degree IP_DEG - 1 in t in [-1, 1] (see matern_gen.cu).
constexpr int IP_OCTAVES = 10;
constexpr int IP_SUB = 8;
constexpr int IP_DEG = 12;
constexpr int IP_INTERVALS = IP_OCTAVES * IP_SUB;
struct QuadTables {
    double exp2tab[EXP_TABLE];            // 2^(j/256), j = 0..255 (table of the exponential)
    double st2[QUAD_LEVELS][QUAD_NODES];  // 2 sinh^2(t_j / 2)  (x cosh t = x + x * st2)
    double wa[QUAD_LEVELS][QUAD_NODES];   // w_j cosh(nu t_j)
    double wb[QUAD_LEVELS][QUAD_NODES];   // w_j cosh((nu - 1) t_j)
    double wd[QUAD_LEVELS][QUAD_NODES];   // w_j t_j sinh(nu t_j)
    double ipoly[IP_INTERVALS][3][IP_DEG];   // monomial coefficients, constant term first
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

// linear index t of the lower triangle (row-major: (0,0),(1,0),(1,1),(2,0),...) -> (r, c), c <= r.
// The FP32 square root only estimates r (the FP64 pipe is the tile-update epilogue's scarce
// resource, and every thread decodes every task); the integer steps make the result exact.
__device__ inline void tri_decode(long long t, int& r, int& c) {
    long long rr = (long long)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((rr + 1) * (rr + 2) / 2 <= t) ++rr;
    while (rr * (rr + 1) / 2 > t) --rr;
    r = (int)rr;
    c = (int)(t - rr * (rr + 1) / 2);
}

// ---- FP64-accurate tile updates on tensor cores (ozaki.cu) ----
size_t ozaki_tile_bytes();   // digit planes + row scales of one sliced 128 x 128 tile
// position of strictly-lower tile (i, k), i > k, in the column-ordered list of such tiles
__host__ __device__ inline long long strict_lower_pos(int i, int k, int T) {
    return tile_index(i, k, T) - k - 1;
}

// Which tiles a slicing launch reads: block t of the launch slices tile (ti, tj) of src into
// position t of the slice buffer.
enum : int { SLICE_PANEL = 0, SLICE_ROW = 1, SLICE_DIAG = 2, SLICE_PTR = 3 };
struct SliceJob {
    const double* src;
    int mode, k, T;
    // tile t of the launch: (ti, tj) of the slab src; SLICE_PTR: tile t of a contiguous tile array
    __device__ const double* tile_ptr(int t, int nb) const {
        if (mode == SLICE_PTR) return src + (long long)t * nb * nb;
        int ti, tj;
        if (mode == SLICE_PANEL) { ti = k + 1 + t; tj = k; }       // column k below the diagonal
        else if (mode == SLICE_ROW) { ti = k; tj = t; }            // row k left of the diagonal
        else { ti = k; tj = k; }                                    // diagonal tile k
        return src + tile_offset(ti, tj, T, nb);
    }
};

// One task of an update launch: 128 rows x 64 columns of one target tile (two per tile).
enum : int { OZ_POTRF_UPD = 0, OZ_SYGST_UPD = 1, OZ_SYGST_FIX = 2, OZ_SYGST_ROWUPD = 3, OZ_SINGLE = 4,
             OZ_ROWSOLVE = 5, OZ_LAUUM = 6, OZ_POTRF_COL = 7, OZ_POTRF_REST = 8 };
struct OzGemmJob {
    int mode, k, T;
    double* C;                     // target slab
    const unsigned char* slA;      // sliced A operands
    const unsigned char* slB;      // sliced B operands
    size_t tile_bytes;
    double mult;
    int assign;                    // 1: C = -mult * A B^T (overwrite); 0: C -= mult * A B^T
    int mixed = 0;                 // 1: digit planes per task from the operand magnitudes
    int e_fp64 = 0, e_fp32 = 0;    // exponent thresholds of the mixed path (see task_planes)
    int e_skip = -100000;
    unsigned long long* counts = nullptr;   // tasks per tier (mixed path, optional)
    long long* task_list = nullptr;         // mixed path: classified task list (see MixedPolicy)
    unsigned* task_count = nullptr;
    long long task_cap = 0;
    __device__ void task(long long bid, const unsigned char*& sa, const unsigned char*& sb,
                         double*& Ct, int& c0, double& m) const {
        const long long tsk = bid >> 1;
        c0 = (int)(bid & 1) * 64;
        m = mult;
        if (mode == OZ_POTRF_UPD || mode == OZ_SYGST_UPD || mode == OZ_POTRF_REST) {
            // OZ_POTRF_REST: the trailing update without its first column (jj >= 1)
            int ii, jj;
            tri_decode(tsk, ii, jj);
            if (mode == OZ_POTRF_REST) { ++ii; ++jj; }
            Ct = C + tile_offset(k + 1 + ii, k + 1 + jj, T, 128);
            sa = slA + (size_t)ii * tile_bytes;
            sb = slB + (size_t)jj * tile_bytes;
        } else if (mode == OZ_POTRF_COL) {      // the trailing update's first column: (k+1+ii, k+1)
            Ct = C + tile_offset(k + 1 + (int)tsk, k + 1, T, 128);
            sa = slA + (size_t)tsk * tile_bytes;
            sb = slB;
        } else if (mode == OZ_SYGST_FIX) {
            Ct = C + tile_offset(k + 1 + (int)tsk, k, T, 128);
            sa = slA + (size_t)tsk * tile_bytes;
            sb = slB;
        } else if (mode == OZ_SYGST_ROWUPD) {   // m = k: targets (i, kk), i > m > kk
            const int kk = (int)(tsk % k), ii = (int)(tsk / k);
            Ct = C + tile_offset(k + 1 + ii, kk, T, 128);
            sa = slA + (size_t)ii * tile_bytes;
            sb = slB + (size_t)kk * tile_bytes;
        } else if (mode == OZ_LAUUM) {          // targets (i, j), j <= i <= p = k, from row p
            int ii, jj;
            tri_decode(tsk, ii, jj);
            Ct = C + tile_offset(ii, jj, T, 128);
            sa = slA + (size_t)ii * tile_bytes;
            sb = slA + (size_t)jj * tile_bytes;
        } else if (mode == OZ_SINGLE) {         // one tile: C points at it
            Ct = C;
            sa = slA;
            sb = slB;
        } else {                                // OZ_ROWSOLVE, m = k: targets (m, kk), kk < m
            Ct = C + tile_offset(k, (int)tsk, T, 128);
            sa = slA;
            sb = slB + (size_t)tsk * tile_bytes;
        }
    }
};

// ---- partial-sum slot layout (doubles) ----
struct Slots {
    double* logdet;     // [T]               sum_j log L_jj of diagonal tile k
    double* qform;      // [ntiles * 2]      w_i^T Sigma_a,b(i,j) w_j per tile (x2 off-diagonal)
    double* diag;       // [T * strips * 5]  tr B_a, tr B_n, <B_a,B_a>, <B_a,B_n>, <B_n,B_n>
    double* offd;       // [ntiles * strips * 3]  <.,.> of off-diagonal tiles (not yet doubled)
};

// Raise a kernel's dynamic shared-memory limit to at least `bytes`, calling the runtime only when
// the limit grows (host-side state, kept out of captured launch sequences; thread safe).
void ensure_smem(const void* kernel, int bytes);

// ---- launch bookkeeping: launch counter and optional CUDA-event timing per kernel family ----
struct Profiler;
struct Launcher {
    cudaStream_t stream = nullptr;
    Profiler* prof = nullptr;        // non-null while profiling is enabled
    long long* launches = nullptr;   // running count of this library's kernel launches
    long long spin = 0;              // iteration limit of the tensor-core kernel's waits (0: default)
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
// the same from device memory th[4] = (sigma^2, alpha, nu, jitter)
int launch_prep_theta_dev(Launcher& L, const double* th, ThetaConsts* tc, QuadTables* qt);
int launch_generate(Launcher& L, const Geom& g, const double* X, const double* Y,
                    const ThetaConsts* tc, const QuadTables* qt, double* S, double* SA,
                    double* SN, bool deriv, int* status);

int launch_ozaki_slice(Launcher& L, const Geom& g, const SliceJob& job, int ntiles, bool rows,
                       unsigned char* dst,
                       const char* family = "ozaki_slice");
// the same tiles of two jobs (ntiles each) in one launch
int launch_ozaki_slice2(Launcher& L, const Geom& g, const SliceJob& job0, unsigned char* dst0,
                        const SliceJob& job1, unsigned char* dst1, int ntiles, bool rows);
int launch_ozaki_gemm(Launcher& L, const OzGemmJob& job, long long ctas, double flops, int* status,
                      const char* family);
// up to 4 jobs (tasks[j] tasks each, targets that do not overlap) in one persistent launch
int launch_ozaki_gemm_multi(Launcher& L, const OzGemmJob* job, const long long* tasks, int njobs, double flops,
                            int* status, const char* family, int reserve_sms = 0);

// tiled Cholesky of the S slab in place (lower tiles), log-det partials per diagonal tile;
// precision PREC_FP64_OZAKI runs the trailing updates on tensor cores (needs `slices`), and with
// `wtiles` / `wslices` (T FP64 tiles, T sliced tiles of scratch) the panel solves as well
// side / ev[2] (optional, tensor path): a second stream and two events for the lookahead, in
// which the next diagonal tile is factored on one SM while the rest of the trailing update runs
// on the others
int launch_potrf(Launcher& L, const Geom& g, double* S, double* logdet_slots, int* status,
                 int precision = PREC_FP64, unsigned char* slices = nullptr,
                 const MixedPolicy& pol = MixedPolicy(), double* wtiles = nullptr,
                 unsigned char* wslices = nullptr, cudaStream_t side = nullptr,
                 cudaEvent_t* ev = nullptr);
// two-sided transform B = L^-1 M L^-T of both derivative slabs in place, with the trace and
// Frobenius-product partials of the result
// precision PREC_FP64_OZAKI: L_slices holds the digit planes of every strictly-lower tile of L
// (written by launch_potrf); scratch: room for 2 (T - 1) + 6 more sliced tiles; Winv: T FP64 tiles
// (inverses of the diagonal factor tiles), Wsl: their digit planes, Y: 2 FP64 scratch tiles
int launch_sygst(Launcher& L, const Geom& g, const double* S, double* M0, double* M1,
                 double* diag_slots, double* offd_slots, int* status, int precision = PREC_FP64,
                 const unsigned char* L_slices = nullptr, unsigned char* scratch = nullptr,
                 double* Winv = nullptr, unsigned char* Wsl = nullptr, double* Y = nullptr,
                 const MixedPolicy& pol = MixedPolicy());
int strips_per_tile(int nb);

// Sigma^-1 = L^-T L^-1 from the factor in S (emulated FP64 on tensor cores): W = L^-1 into the W
// slab (tile forward substitution with the inverted diagonal tiles), then X = W^T W (lower tiles)
// into the X slab.  Needs the digit planes of L (L_slices), scratch for 2 (T - 1) + 6 sliced
// tiles, Winv (T FP64 tiles), Wsl and Wcs (T sliced tiles each).
int launch_inverse_from_factor(Launcher& L, const Geom& g, const double* S, double* W, double* X,
                               int* status, const unsigned char* L_slices, unsigned char* scratch,
                               double* Winv, unsigned char* Wsl, unsigned char* Wcs,
                               const MixedPolicy& pol);
// per-tile partials f sum_(r,c) (w_r w_c - X_rc) dSigma/dtheta_i (r,c) for i = alpha, nu with the
// partials regenerated on the fly (f = 2 off the diagonal): slots[2 t + i - 1]
int launch_adjoint_reduce(Launcher& L, const Geom& g, const double* Xs, const double* Yc,
                          const double* X, const double* w, const ThetaConsts* tc,
                          const QuadTables* qt, double* slots, int* status);

// v <- L^-1 v (trans = false) or v <- L^-T v (trans = true), tile by tile
// winv (optional): the inverted diagonal factor tiles; the diagonal steps then multiply by them,
// writing each solved block to vx (nb doubles of scratch, required with winv) first
int launch_trsv(Launcher& L, const Geom& g, const double* S, double* v, bool trans, const double* winv = nullptr,
                double* vx = nullptr);
// per-tile partials of w^T M0 w and w^T M1 w over the lower tiles (off-diagonal tiles doubled)
int launch_qform(Launcher& L, const Geom& g, const double* M0, const double* M1, const double* w,
                 double* qform_slots);
int launch_assemble(Launcher& L, const Geom& g, const double* y, const Slots& s, bool deriv,
                    const ThetaConsts* tc, const int* status, EvalOut* out);

}  // namespace fbt
