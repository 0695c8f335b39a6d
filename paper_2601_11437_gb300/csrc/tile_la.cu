// Steps a2, a3, a7, a8: tiled FP64 Cholesky with log-det partials, and the two-sided transform
// B_i = L^-1 Sigma_i L^-T of both derivative matrices with fused trace / Frobenius partials.
//
// On GB300 the FP64 rate is set by the DFMA pipe (measured 1.19 TFLOP/s over 152 SMs, i.e. two
// FP64 FMAs per clock per SM; the FP64 mma.sync path measured 1.05 TFLOP/s), so these kernels
// are plain DFMA register-blocked tiles: every SM must simply be kept issuing DFMAs.
//
// Cholesky (Algorithm 2/3 step "Cholesky factorization"), right-looking over tile steps k:
//   L_kk = chol(S_kk); L_ik = S_ik L_kk^-T (i > k); S_ij -= L_ik L_jk^T (k < j <= i).
// Two-sided transform (replaces the paper's A_i = Sigma^-1 Sigma_i, whose traces Eq. 3 needs:
// tr(Sigma^-1 S_a Sigma^-1 S_b) = <B_a, B_b>_F and tr(Sigma^-1 S_a) = tr B_a), by the tile
// recursion of the blocked LAPACK-style algorithm, step k:
//   B_kk = L_kk^-1 M_kk L_kk^-T
//   C_ik = M_ik L_kk^-T,  E_ik = C_ik - 1/2 L_ik B_kk                       (i > k)
//   M_ij -= L_ik E_jk^T + E_ik L_jk^T                                       (k < j <= i)
//   P_ik = E_ik - 1/2 L_ik B_kk
// and finally B_(k+1:,k) = L_(k+1:,k+1:)^-1 P_(k+1:,k), done for all columns at once as a
// left-looking tile forward substitution over rows m (TRSM with L_mm, then GEMM updates).
#include <math.h>

#include "fbt_kernels.cuh"

namespace fbt {

// ------------------------------------------------------------------------------------------
// Diagonal tile Cholesky (one CTA, tile resident in shared memory)
// ------------------------------------------------------------------------------------------
template <int NB>
__global__ void __launch_bounds__(512) k_potrf_diag(double* __restrict__ S, int T, int k,
                                                    double* __restrict__ logdet_slots,
                                                    int* status) {
    extern __shared__ double A[];
    constexpr int LD = NB + 1;
    __shared__ double s_inv;
    __shared__ int s_bad;
    double* tile = S + tile_offset(k, k, T, NB);
    {
        const double2* __restrict__ t2 = (const double2*)tile;
#pragma unroll 16
        for (int e2 = threadIdx.x; e2 < NB * NB / 2; e2 += blockDim.x) {
            const double2 w = t2[e2];
            const int r = (2 * e2) % NB, c = (2 * e2) / NB;
            A[r + c * LD] = r >= c ? w.x : 0.0;
            A[r + 1 + c * LD] = r + 1 >= c ? w.y : 0.0;
        }
    }
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int j = 0; j < NB; ++j) {
        if (threadIdx.x == 0) {
            double d = A[j + j * LD];
            if (!(d > 0.0) || !isfinite(d)) { s_bad = 1; d = 1.0; }
            const double inv = rsqrt(d);             // one long-latency FP64 operation on the
            A[j + j * LD] = d * inv;                 // sequential chain instead of sqrt and 1 / l
            s_inv = inv;
        }
        __syncthreads();
        for (int r = j + 1 + threadIdx.x; r < NB; r += blockDim.x) A[r + j * LD] *= s_inv;
        __syncthreads();
        // trailing update of the lower triangle: warp w takes columns j + 1 + w, + nwarps, ...,
        // its lanes the rows c, c + 1, ... of each (no index division, no idle upper half)
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int c = j + 1 + warp; c < NB; c += nw) {
            const double lc = A[c + j * LD];
            for (int r = c + lane; r < NB; r += 32) A[r + c * LD] -= A[r + j * LD] * lc;
        }
        __syncthreads();
    }
    {
        double2* t2 = (double2*)tile;
#pragma unroll 16
        for (int e2 = threadIdx.x; e2 < NB * NB / 2; e2 += blockDim.x) {
            const int r = (2 * e2) % NB, c = (2 * e2) / NB;
            t2[e2] = make_double2(r >= c ? A[r + c * LD] : 0.0, r + 1 >= c ? A[r + 1 + c * LD] : 0.0);
        }
    }
    // sum of log L_jj: one logarithm per thread, then a fixed-order tree
    __shared__ double s_log[NB];
    for (int j = threadIdx.x; j < NB; j += blockDim.x) s_log[j] = log(A[j + j * LD]);
    __syncthreads();
    for (int w = NB / 2; w > 0; w >>= 1) {
        for (int j = threadIdx.x; j < w; j += blockDim.x) s_log[j] += s_log[j + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        logdet_slots[k] = s_log[0];
        if (s_bad) atomicOr(status, ST_NOT_PD);
    }
}

// ------------------------------------------------------------------------------------------
// Strip triangular solves.  A strip is 32 rows (RIGHT: X = A L^-T) or 32 columns (LEFT:
// X = L^-1 A) of a target tile; each of the 32 strip vectors v obeys the same forward
// substitution v_d /= L_dd, v_d' -= L_d'd v_d (d' > d).  Up to two target tiles share L.
// ------------------------------------------------------------------------------------------
enum TrsmMode : int {
    TRSM_POTRF_PANEL = 0,   // targets S(i,k), i > k;            RIGHT, 1 matrix
    TRSM_SYGST_DIAG_R = 1,  // targets M(k,k);                   RIGHT, 2 matrices
    TRSM_SYGST_DIAG_L = 2,  // targets M(k,k);                   LEFT,  2 matrices, diag epilogue
    TRSM_SYGST_PANEL = 3,   // targets M(i,k), i > k;            RIGHT, 2 matrices
    TRSM_SYGST_ROW = 4      // targets M(m,kk), kk < m, L=S(m,m); LEFT, 2 matrices, off-diag epilogue
};

struct TrsmParams {
    int mode, k, T;
    const double* S;
    double* M0;
    double* M1;
    double* slots;
};

constexpr int STRIP = 32;

int strips_per_tile(int nb) { return nb / STRIP; }

template <int NB, bool LEFT, int NMAT, int EPI>
__global__ void __launch_bounds__(256) k_trsm_strip(TrsmParams p) {
    extern __shared__ double V[];                      // [NMAT][STRIP][NB + 1], then L [NB][NB + 1]
    constexpr int LDV = NB + 1;
    double* Ls = V + NMAT * STRIP * LDV;               // the triangular factor, staged once
    constexpr int NSTRIPS = NB / STRIP;
    __shared__ double s_inv[NB];
    __shared__ double s_red[STRIP][8];
    const int task = blockIdx.x / NSTRIPS, strip = blockIdx.x % NSTRIPS;
    const int T = p.T;
    int li, ti, tj;   // L tile (li, li); target tile (ti, tj)
    switch (p.mode) {
        case TRSM_POTRF_PANEL: li = p.k; ti = p.k + 1 + task; tj = p.k; break;
        case TRSM_SYGST_DIAG_R:
        case TRSM_SYGST_DIAG_L: li = p.k; ti = p.k; tj = p.k; break;
        case TRSM_SYGST_PANEL: li = p.k; ti = p.k + 1 + task; tj = p.k; break;
        default: li = p.k; ti = p.k; tj = task; break;   // TRSM_SYGST_ROW, m = p.k
    }
    const double* __restrict__ Lt = p.S + tile_offset(li, li, T, NB);
    const long long toff = tile_offset(ti, tj, T, NB);
    double* tgt[2];
    tgt[0] = (NMAT == 1 ? const_cast<double*>(p.S) : p.M0) + toff;
    tgt[1] = NMAT == 2 ? p.M1 + toff : nullptr;
    const int o = strip * STRIP;
    for (int m = 0; m < NMAT; ++m) {
        double* src = tgt[m];
        for (int e = threadIdx.x; e < STRIP * NB; e += blockDim.x) {
            int lane, d;
            double val;
            if (LEFT) { d = e % NB; lane = e / NB; val = src[d + (long long)(o + lane) * NB]; }
            else { lane = e % STRIP; d = e / STRIP; val = src[(o + lane) + (long long)d * NB]; }
            V[(m * STRIP + lane) * LDV + d] = val;
        }
    }
    {
        const double2* __restrict__ L2 = (const double2*)Lt;
#pragma unroll 16
        for (int e2 = threadIdx.x; e2 < NB * NB / 2; e2 += blockDim.x) {
            const double2 w = L2[e2];
            const int r = (2 * e2) % NB, c = (2 * e2) / NB;
            if (r > c) Ls[r + c * LDV] = w.x;
            if (r + 1 > c) Ls[r + 1 + c * LDV] = w.y;
        }
    }
    for (int d = threadIdx.x; d < NB; d += blockDim.x) s_inv[d] = 1.0 / Lt[d + (long long)d * NB];
    __syncthreads();
    const int lane = threadIdx.x % STRIP, grp = threadIdx.x / STRIP;   // 8 groups of 32
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int d = 0; d < NB; ++d) {
        const double* __restrict__ Lcol = Ls + d * LDV;
        double vv[NMAT];
#pragma unroll
        for (int m = 0; m < NMAT; ++m) vv[m] = V[(m * STRIP + lane) * LDV + d] * s_inv[d];
        if (grp == 0) {
#pragma unroll
            for (int m = 0; m < NMAT; ++m) {
                if (LEFT) tgt[m][d + (long long)(o + lane) * NB] = vv[m];
                else tgt[m][(o + lane) + (long long)d * NB] = vv[m];
            }
            if (EPI == 1) {                       // diagonal tile: traces and Frobenius products
                if (d == o + lane) { acc[0] += vv[0]; acc[1] += vv[NMAT - 1]; }
                acc[2] += vv[0] * vv[0];
                acc[3] += vv[0] * vv[NMAT - 1];
                acc[4] += vv[NMAT - 1] * vv[NMAT - 1];
            } else if (EPI == 2) {                // off-diagonal tile: Frobenius products
                acc[2] += vv[0] * vv[0];
                acc[3] += vv[0] * vv[NMAT - 1];
                acc[4] += vv[NMAT - 1] * vv[NMAT - 1];
            }
        }
        for (int dp = d + 1 + grp; dp < NB; dp += 8) {
            const double l = Lcol[dp];
#pragma unroll
            for (int m = 0; m < NMAT; ++m) V[(m * STRIP + lane) * LDV + dp] -= vv[m] * l;
        }
        __syncthreads();
    }
    if (EPI != 0 && grp == 0) {
        // fixed-order reduction over the 32 lanes of warp 0
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            double v = acc[q];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            acc[q] = v;
        }
        if (lane == 0) {
            if (EPI == 1) {
                double* out = p.slots + ((long long)p.k * NSTRIPS + strip) * 5;
                for (int q = 0; q < 5; ++q) out[q] = acc[q];
            } else {
                double* out = p.slots + (tile_index(ti, tj, T) * NSTRIPS + strip) * 3;
                out[0] = acc[2]; out[1] = acc[3]; out[2] = acc[4];
            }
        }
    }
    (void)s_red;
}

// ------------------------------------------------------------------------------------------
// Tile GEMM: one CTA computes a 64 x 64 block of a target tile,
//   C -= scale * sum_terms op(A) op(B),  NT: C[r][c] -= A[r][p] B[c][p];  NN: A[r][p] B[p][c]
// 256 threads as 16 x 16, each a 4 x 4 register block (rows tx + 16a, columns ty + 16b).
// ------------------------------------------------------------------------------------------
enum GemmMode : int {
    GEMM_POTRF_UPD = 0,      // S(i,j) -= S(i,k) S(j,k)^T,  k < j <= i, lower 64-blocks of diagonal tiles
    GEMM_SYGST_UPD = 1,      // M(i,j) -= S(i,k) M(j,k)^T + M(i,k) S(j,k)^T, k < j <= i, full tiles
    GEMM_SYGST_FIX = 2,      // M(i,k) -= 1/2 S(i,k) M(k,k),  i > k      (M(k,k) symmetric: NT)
    GEMM_SYGST_ROWUPD = 3    // M(i,kk) -= S(i,m) M(m,kk),   i > m > kk  (NN)
};

struct GemmParams {
    int mode, k, T;
    const double* S;
    double* M0;
    double* M1;
};

constexpr int GB = 64, GK = 32;

template <int NB, bool NN, int NTERMS>
__global__ void __launch_bounds__(256) k_gemm_tile(GemmParams p) {
    constexpr int SB = NB / GB;            // 64-blocks per tile side
    __shared__ double As[GK][GB];
    __shared__ double Bs[GK][GB + 1];
    const int T = p.T, k = p.k;
    const long long bid = blockIdx.x;
    const int sub = (int)(bid % (SB * SB));
    const long long task = bid / (SB * SB);
    const int sr = sub % SB, sc = sub / SB;
    double* M = blockIdx.y == 0 ? p.M0 : p.M1;
    int ci, cj;
    const double *A1, *B1, *A2 = nullptr, *B2 = nullptr;
    double scale = 1.0;
    if (p.mode == GEMM_POTRF_UPD || p.mode == GEMM_SYGST_UPD) {
        int ii, jj;
        tri_decode(task, ii, jj);
        ci = k + 1 + ii;
        cj = k + 1 + jj;
        if (p.mode == GEMM_POTRF_UPD) {
            if (ci == cj && sr < sc) return;           // only the lower triangle of S is used
            M = const_cast<double*>(p.S);
            A1 = p.S + tile_offset(ci, k, T, NB);
            B1 = p.S + tile_offset(cj, k, T, NB);
        } else {
            A1 = p.S + tile_offset(ci, k, T, NB);
            B1 = M + tile_offset(cj, k, T, NB);
            A2 = M + tile_offset(ci, k, T, NB);
            B2 = p.S + tile_offset(cj, k, T, NB);
        }
    } else if (p.mode == GEMM_SYGST_FIX) {
        ci = k + 1 + (int)task;
        cj = k;
        A1 = p.S + tile_offset(ci, k, T, NB);
        B1 = M + tile_offset(k, k, T, NB);
        scale = 0.5;
    } else {   // GEMM_SYGST_ROWUPD, m = k: tasks (ci, cj) with ci in (m, T), cj in [0, m)
        const int m = k;
        cj = (int)(task % m);
        ci = m + 1 + (int)(task / m);
        A1 = p.S + tile_offset(ci, m, T, NB);
        B1 = M + tile_offset(m, cj, T, NB);
    }
    double* C = M + tile_offset(ci, cj, T, NB);
    const int r0 = sr * GB, c0 = sc * GB;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
#pragma unroll
    for (int term = 0; term < NTERMS; ++term) {
        const double* __restrict__ A = term == 0 ? A1 : A2;
        const double* __restrict__ B = term == 0 ? B1 : B2;
        for (int k0 = 0; k0 < NB; k0 += GK) {
            for (int e = threadIdx.x; e < GK * GB; e += 256) {
                const int rr = e % GB, kk = e / GB;
                As[kk][rr] = A[(r0 + rr) + (long long)(k0 + kk) * NB];
            }
            if (NN) {
                for (int e = threadIdx.x; e < GK * GB; e += 256) {
                    const int kk = e % GK, cc = e / GK;
                    Bs[kk][cc] = B[(k0 + kk) + (long long)(c0 + cc) * NB];
                }
            } else {
                for (int e = threadIdx.x; e < GK * GB; e += 256) {
                    const int cc = e % GB, kk = e / GB;
                    Bs[kk][cc] = B[(c0 + cc) + (long long)(k0 + kk) * NB];
                }
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < GK; ++kk) {
                double av[4], bv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
                for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            double* cp = C + (r0 + tx + 16 * a) + (long long)(c0 + ty + 16 * b) * NB;
            *cp -= scale * acc[a][b];
        }
}

// ------------------------------------------------------------------------------------------
// host orchestration
// ------------------------------------------------------------------------------------------
static inline OzGemmJob with_policy(OzGemmJob j, const MixedPolicy& pol) {
    j.mixed = pol.on;
    j.e_fp64 = pol.e_fp64;
    j.e_fp32 = pol.e_fp32;
    j.e_skip = pol.e_skip;
    j.counts = pol.counts;
    j.task_list = pol.task_list;
    j.task_count = pol.task_count;
    j.task_cap = pol.task_cap;
    return j;
}
// W = L_kk^-1 by columns: warp c of the launch solves L w = e_c by forward substitution with the
// vector in registers (as the diagonal TRSV does), so one tile's inverse spreads over NB / 8
// CTAs instead of running column after column in one.  The factor tile is staged in shared memory.
template <int NB>
__global__ void __launch_bounds__(256) k_trtri_cols(const double* __restrict__ S, int T, int k0,
                                                   double* __restrict__ Wbase) {
    // tile k = k0 + blockIdx.y, its inverse at Wbase + k nb^2
    const int k = k0 + (int)blockIdx.y;
    double* __restrict__ W = Wbase + (long long)k * NB * NB;
    extern __shared__ double A[];
    constexpr int LD = NB + 1;
    constexpr int NBLK = NB / 32;
    double* rinv = A + NB * LD;
    const double* __restrict__ Lt = S + tile_offset(k, k, T, NB);
    {
        const double2* __restrict__ L2 = (const double2*)Lt;
#pragma unroll 16
        for (int e2 = threadIdx.x; e2 < NB * NB / 2; e2 += blockDim.x) {
            const double2 w = L2[e2];
            const int r = (2 * e2) % NB, c = (2 * e2) / NB;
            if (r >= c) A[r + c * LD] = w.x;
            if (r + 1 >= c) A[r + 1 + c * LD] = w.y;
        }
    }
    for (int d = threadIdx.x; d < NB; d += blockDim.x) rinv[d] = 1.0 / Lt[d + (long long)d * NB];
    __syncthreads();
    const int lane = threadIdx.x & 31, c = blockIdx.x * 8 + (threadIdx.x >> 5);
    double x[NBLK];
#pragma unroll
    for (int s = 0; s < NBLK; ++s) x[s] = lane + 32 * s == c ? 1.0 : 0.0;
#pragma unroll
    for (int s = 0; s < NBLK; ++s) {
        for (int dd = 0; dd < 32; ++dd) {
            const int d = 32 * s + dd;
            if (d < c) continue;                        // warp-uniform
            double xd = 0.0;
            if (lane == dd) { xd = x[s] * rinv[d]; x[s] = xd; }
            xd = __shfl_sync(0xffffffffu, xd, dd);
#pragma unroll
            for (int t = 0; t < NBLK; ++t) {
                const int r = lane + 32 * t;
                if (t >= s && r > d) x[t] -= A[r + d * LD] * xd;
            }
        }
    }
    double* Wc = W + (long long)c * NB;
#pragma unroll
    for (int s = 0; s < NBLK; ++s) {
        const int r = lane + 32 * s;
        Wc[r] = r >= c ? x[s] : 0.0;
    }
}

// Tensor-core Cholesky with lookahead.  Per step k: the panel L_ik = A_ik W_k^T (tensor cores),
// its digit planes, the first column of the trailing update, then the rest of the update as a
// persistent launch on all SMs but one while the side stream factors and inverts diagonal tile
// k + 1 on the free SM (its inputs are final once the first column is updated).
template <int NB>
static int potrf_tensor(Launcher& L, const Geom& g, double* S, double* logdet_slots, int* status,
                        unsigned char* slices, const MixedPolicy& pol, double* wtiles, unsigned char* wslices,
                        cudaStream_t side, cudaEvent_t* ev) {
    const int T = g.T;
    const size_t tb = ozaki_tile_bytes();
    const double nb3 = (double)NB * NB * NB, nb2 = (double)NB * NB;
    const size_t smem_potrf = (size_t)NB * (NB + 1) * sizeof(double);
    const size_t smem_tc = (size_t)NB * (NB + 2) * sizeof(double);
    ensure_smem((const void*)k_potrf_diag<NB>, (int)smem_potrf);
    ensure_smem((const void*)k_trtri_cols<NB>, (int)smem_tc);
    Launcher LS = L;
    LS.stream = side;
    auto diag = [&](Launcher& X, int k) -> int {
        X.begin("potrf_diag");
        k_potrf_diag<NB><<<1, 512, smem_potrf, X.stream>>>(S, T, k, logdet_slots, status);
        X.count();
        int r = X.end(nb3 / 3.0, 16.0 * nb2);
        if (r) return r;
        X.begin("trtri_panel");
        k_trtri_cols<NB><<<dim3(NB / 8, 1), 256, smem_tc, X.stream>>>(S, T, k, wtiles);
        X.count();
        return X.end(nb3 / 3.0, 16.0 * nb2);
    };
    int rc = diag(L, 0);
    if (rc) return rc;
    for (int k = 0; k + 1 < T; ++k) {
        const int m = T - k - 1;
        unsigned char* Wks = wslices + (size_t)k * tb;
        unsigned char* panel = slices + strict_lower_pos(k + 1, k, T) * tb;
        SliceJob wj{wtiles + (size_t)k * NB * NB, SLICE_PTR, 0, T};
        if ((rc = launch_ozaki_slice(L, g, wj, 1, true, Wks, "cholesky_slice"))) return rc;
        SliceJob aj{S, SLICE_PANEL, k, T};
        if ((rc = launch_ozaki_slice(L, g, aj, m, true, panel, "cholesky_slice"))) return rc;   // digits of A_ik
        OzGemmJob pj{OZ_SYGST_FIX, k, T, S, panel, Wks, tb, -1.0, 1};
        if ((rc = launch_ozaki_gemm(L, pj, (long long)m * 2, m * 2.0 * nb3, status, "ozaki_potrf_panel"))) return rc;
        // digit planes of panel k, kept for the two-sided transforms
        if ((rc = launch_ozaki_slice(L, g, aj, m, true, panel, "cholesky_slice"))) return rc;
        OzGemmJob cj = with_policy({OZ_POTRF_COL, k, T, S, panel, panel, tb, 1.0, 0}, pol);
        const double fl_col = (m - 1) * 2.0 * nb3 + nb3 + nb2;
        if ((rc = launch_ozaki_gemm(L, cj, (long long)m * 2, fl_col, status, "ozaki_potrf_update"))) return rc;
        if (m == 1) {
            if ((rc = diag(L, k + 1))) return rc;
            continue;
        }
        OzGemmJob rj = with_policy({OZ_POTRF_REST, k, T, S, panel, panel, tb, 1.0, 0}, pol);
        const long long rest = (long long)(m - 1) * m;      // (m - 1) m / 2 tiles, two tasks each
        const double fl_rest = (double)(m - 1) * (m - 2) / 2 * 2.0 * nb3 + (m - 1) * (nb3 + nb2);
        if (side) {
            if (cudaEventRecord(ev[0], L.stream) != cudaSuccess || cudaStreamWaitEvent(side, ev[0], 0) != cudaSuccess)
                return cudaGetLastError();
            if ((rc = diag(LS, k + 1))) return rc;
            if (cudaEventRecord(ev[1], side) != cudaSuccess) return cudaGetLastError();
            if ((rc = launch_ozaki_gemm_multi(L, &rj, &rest, 1, fl_rest, status, "ozaki_potrf_update", 1))) return rc;
            if (cudaStreamWaitEvent(L.stream, ev[1], 0) != cudaSuccess) return cudaGetLastError();
        } else {
            if ((rc = launch_ozaki_gemm_multi(L, &rj, &rest, 1, fl_rest, status, "ozaki_potrf_update"))) return rc;
            if ((rc = diag(L, k + 1))) return rc;
        }
    }
    return rc;
}

template <int NB>
static int potrf_impl(Launcher& L, const Geom& g, double* S, double* logdet_slots, int* status,
                      int precision, unsigned char* slices, const MixedPolicy& pol, double* wtiles,
                      unsigned char* wslices) {
    const int T = g.T;
    const size_t smem_potrf = (size_t)NB * (NB + 1) * sizeof(double);
    const size_t smem_trsm1 = (size_t)(STRIP + NB) * (NB + 1) * sizeof(double);
    ensure_smem((const void*)k_potrf_diag<NB>, (int)smem_potrf);
    ensure_smem((const void*)k_trsm_strip<NB, false, 1, 0>, (int)smem_trsm1);
    constexpr int NS = NB / STRIP;
    constexpr int SB = NB / GB;
    const double nb3 = (double)NB * NB * NB;
    int rc = 0;
    for (int k = 0; k < T; ++k) {
        L.begin("potrf_diag");
        k_potrf_diag<NB><<<1, 512, smem_potrf, L.stream>>>(S, T, k, logdet_slots, status);
        L.count();
        if ((rc = L.end(nb3 / 3.0, 16.0 * NB * NB))) return rc;
        const int m = T - k - 1;
        const bool tensor = NB == 128 && (precision == PREC_FP64_OZAKI || precision == PREC_MIXED);
        if (tensor && wtiles && wslices) {
            // W_k = L_kk^-1 (column-parallel) for every diagonal tile, the last one included: the
            // panel below uses it, and so do the field's triangular solves
            const size_t smem_tc = (size_t)NB * (NB + 2) * sizeof(double);
            ensure_smem((const void*)k_trtri_cols<NB>, (int)smem_tc);
            L.begin("trtri_panel");
            k_trtri_cols<NB><<<dim3(NB / 8, 1), 256, smem_tc, L.stream>>>(S, T, k, wtiles);
            L.count();
            if ((rc = L.end(nb3 / 3.0, 16.0 * NB * NB))) return rc;
        }
        if (m == 0) break;
        if (tensor && wtiles && wslices) {
            // panel on tensor cores: L_ik = A_ik W_k^T as an FP64-accurate tile product (all digit
            // planes), instead of FP64 strip solves
            const size_t tb = ozaki_tile_bytes();
            double* Wk = wtiles + (size_t)k * NB * NB;
            unsigned char* Wks = wslices + (size_t)k * tb;
            unsigned char* panel = slices + strict_lower_pos(k + 1, k, T) * tb;
            SliceJob wj{Wk, SLICE_PTR, 0, T};
            if ((rc = launch_ozaki_slice(L, g, wj, 1, true, Wks))) return rc;
            SliceJob aj{S, SLICE_PANEL, k, T};
            if ((rc = launch_ozaki_slice(L, g, aj, m, true, panel))) return rc;   // digits of A_ik
            OzGemmJob pj{OZ_SYGST_FIX, k, T, S, panel, Wks, tb, -1.0, 1};
            if ((rc = launch_ozaki_gemm(L, pj, (long long)m * 2, m * 2.0 * nb3, status, "ozaki_potrf_panel"))) return rc;
        } else {
            TrsmParams tp{TRSM_POTRF_PANEL, k, T, S, nullptr, nullptr, nullptr};
            L.begin("trsm_panel");
            k_trsm_strip<NB, false, 1, 0><<<m * NS, 256, smem_trsm1, L.stream>>>(tp);
            L.count();
            if ((rc = L.end((double)m * nb3, 16.0 * m * NB * NB))) return rc;
        }
        const long long tasks = (long long)m * (m + 1) / 2;
        // algorithmic flops: 2 nb^3 per off-diagonal tile, nb^3 + nb^2 for a diagonal (SYRK) tile
        const double fl = (double)m * (m - 1) / 2 * 2.0 * nb3 + m * (nb3 + (double)NB * NB);
        if (tensor) {
            // digit planes of panel k, kept for the two-sided transforms
            unsigned char* panel = slices + strict_lower_pos(k + 1, k, T) * ozaki_tile_bytes();
            SliceJob sj{S, SLICE_PANEL, k, T};
            if ((rc = launch_ozaki_slice(L, g, sj, m, true, panel))) return rc;
            OzGemmJob oj = with_policy({OZ_POTRF_UPD, k, T, S, panel, panel, ozaki_tile_bytes(), 1.0, 0}, pol);
            if ((rc = launch_ozaki_gemm(L, oj, tasks * 2, fl, status, "ozaki_potrf_update"))) return rc;
            continue;
        }
        GemmParams gp{GEMM_POTRF_UPD, k, T, S, nullptr, nullptr};
        L.begin("gemm_potrf_update");
        k_gemm_tile<NB, false, 1><<<dim3((unsigned)(tasks * SB * SB), 1), 256, 0, L.stream>>>(gp);
        L.count();
        if ((rc = L.end(fl, 8.0 * NB * NB * (3.0 * tasks)))) return rc;
    }
    return rc;
}

int launch_potrf(Launcher& L, const Geom& g, double* S, double* logdet_slots, int* status,
                 int precision, unsigned char* slices, const MixedPolicy& pol, double* wtiles,
                 unsigned char* wslices, cudaStream_t side, cudaEvent_t* ev) {
    if (g.nb == 128 && (precision == PREC_FP64_OZAKI || precision == PREC_MIXED) && wtiles && wslices && slices)
        return potrf_tensor<128>(L, g, S, logdet_slots, status, slices, pol, wtiles, wslices, side, side ? ev : nullptr);
    if (g.nb == 128) return potrf_impl<128>(L, g, S, logdet_slots, status, precision, slices, pol, wtiles, wslices);
    if (g.nb == 64) return potrf_impl<64>(L, g, S, logdet_slots, status, precision, slices, pol, wtiles, wslices);
    return cudaErrorInvalidValue;
}

// Trace and Frobenius-product partials of the final transformed tiles (one CTA per lower tile,
// fixed-order reduction): diagonal tile k -> diag slots [k][strip 0] = (tr B0, tr B1, <B0,B0>,
// <B0,B1>, <B1,B1>), off-diagonal tile -> offd slots [tile][strip 0] = (<B0,B0>, <B0,B1>, <B1,B1>);
// the other strip slots are zeroed.
__global__ void __launch_bounds__(256) k_frob_tiles(Geom g, const double* __restrict__ B0,
                                                    const double* __restrict__ B1, int nstrips,
                                                    double* __restrict__ diag_slots,
                                                    double* __restrict__ offd_slots) {
    __shared__ double red[5][256];
    const int T = g.T, nb = g.nb;
    const long long t = blockIdx.x;
    int j = (int)(((2.0 * T + 1.0) - sqrt((2.0 * T + 1.0) * (2.0 * T + 1.0) - 8.0 * (double)t)) * 0.5);
    if (j < 0) j = 0;
    while (j > 0 && tile_index(j, j, T) > t) --j;
    while (j + 1 < T && tile_index(j + 1, j + 1, T) <= t) ++j;
    const int i = j + (int)(t - tile_index(j, j, T));
    const long long base = t * (long long)nb * nb;
    double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const double x = B0[base + e], y = B1[base + e];
        if (i == j && (e % nb) == (e / nb)) { a[0] += x; a[1] += y; }
        a[2] = fma(x, x, a[2]);
        a[3] = fma(x, y, a[3]);
        a[4] = fma(y, y, a[4]);
    }
    for (int q = 0; q < 5; ++q) red[q][threadIdx.x] = a[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 5; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < nstrips) {
        const bool first = threadIdx.x == 0;
        if (i == j) {
            double* o = diag_slots + ((long long)i * nstrips + threadIdx.x) * 5;
            for (int q = 0; q < 5; ++q) o[q] = first ? red[q][0] : 0.0;
        } else {
            double* o = offd_slots + (t * nstrips + threadIdx.x) * 3;
            for (int q = 0; q < 3; ++q) o[q] = first ? red[q + 2][0] : 0.0;
        }
    }
}

// Two-sided transform with every GEMM-shaped step on tensor cores (emulated FP64): the
// triangular solves use the inverted diagonal factor tiles W_k, so they are tile products too.
static int sygst_ozaki(Launcher& L, const Geom& g, const double* S, double* M0, double* M1,
                       double* diag_slots, double* offd_slots, int* status,
                       const unsigned char* LS, unsigned char* scratch, double* Winv,
                       unsigned char* Wsl, double* Y, const MixedPolicy& pol) {
    constexpr int NB = 128;
    const int T = g.T;
    const size_t tb = ozaki_tile_bytes();
    const double nb3 = (double)NB * NB * NB;
    const long long span = T > 1 ? T - 1 : 1;
    unsigned char* Xs[2] = {scratch, scratch + (size_t)span * tb};       // panels / rows
    unsigned char* Ds[2] = {scratch + (size_t)2 * span * tb, scratch + (size_t)(2 * span + 1) * tb};
    unsigned char* Zs[2] = {scratch + (size_t)(2 * span + 2) * tb, scratch + (size_t)(2 * span + 3) * tb};
    double* M[2] = {M0, M1};
    double* Ys[2] = {Y, Y + NB * NB};
    int rc = 0;
    {
        // the same column-parallel kernel as the Cholesky's panels: bitwise the same inverses
        const size_t smem_tc = (size_t)NB * (NB + 2) * sizeof(double);
        ensure_smem((const void*)k_trtri_cols<NB>, (int)smem_tc);
        L.begin("trtri");
        k_trtri_cols<NB><<<dim3(NB / 8, T), 256, smem_tc, L.stream>>>(S, T, 0, Winv);
        L.count();
        if ((rc = L.end(T * nb3 / 3.0, 16.0 * T * NB * NB))) return rc;
        SliceJob wj{Winv, SLICE_PTR, 0, T};
        if ((rc = launch_ozaki_slice(L, g, wj, T, true, Wsl))) return rc;
    }
    const double tile_fl = 2.0 * nb3;
    // the two matrices' products of each step share one launch (their targets are disjoint)
    auto both = [&](const OzGemmJob& j0, const OzGemmJob& j1, long long tasks, double fl, const char* fam) {
        const OzGemmJob js[2] = {with_policy(j0, pol), with_policy(j1, pol)};
        const long long ts[2] = {tasks, tasks};
        return launch_ozaki_gemm_multi(L, js, ts, 2, 2.0 * fl, status, fam);
    };
    for (int k = 0; k < T; ++k) {
        const unsigned char* Wk = Wsl + (size_t)k * tb;
        // B_kk = W_k M_kk W_k^T: Y = M_kk W_k^T, then B_kk = W_k Y
        if ((rc = launch_ozaki_slice2(L, g, SliceJob{M[0], SLICE_DIAG, k, T}, Ds[0],
                                      SliceJob{M[1], SLICE_DIAG, k, T}, Ds[1], 1, true))) return rc;
        if ((rc = both({OZ_SINGLE, k, T, Ys[0], Ds[0], Wk, tb, -1.0, 1}, {OZ_SINGLE, k, T, Ys[1], Ds[1], Wk, tb, -1.0, 1},
                       2, tile_fl, "ozaki_sygst_solve"))) return rc;
        if ((rc = launch_ozaki_slice2(L, g, SliceJob{Ys[0], SLICE_PTR, 0, T}, Zs[0],
                                      SliceJob{Ys[1], SLICE_PTR, 0, T}, Zs[1], 1, false))) return rc;
        if ((rc = both({OZ_SINGLE, k, T, M[0] + tile_offset(k, k, T, NB), Wk, Zs[0], tb, -1.0, 1},
                       {OZ_SINGLE, k, T, M[1] + tile_offset(k, k, T, NB), Wk, Zs[1], tb, -1.0, 1},
                       2, tile_fl, "ozaki_sygst_solve"))) return rc;
        const int m = T - k - 1;
        if (m == 0) break;
        const unsigned char* Lp = LS + strict_lower_pos(k + 1, k, T) * tb;
        // C_ik = M_ik W_k^T, then the digit planes of B_kk
        if ((rc = launch_ozaki_slice2(L, g, SliceJob{M[0], SLICE_PANEL, k, T}, Xs[0],
                                      SliceJob{M[1], SLICE_PANEL, k, T}, Xs[1], m, true))) return rc;
        if ((rc = both({OZ_SYGST_FIX, k, T, M[0], Xs[0], Wk, tb, -1.0, 1}, {OZ_SYGST_FIX, k, T, M[1], Xs[1], Wk, tb, -1.0, 1},
                       (long long)m * 2, m * tile_fl, "ozaki_sygst_solve"))) return rc;
        if ((rc = launch_ozaki_slice2(L, g, SliceJob{M[0], SLICE_DIAG, k, T}, Ds[0],
                                      SliceJob{M[1], SLICE_DIAG, k, T}, Ds[1], 1, true))) return rc;
        // E_ik = C_ik - 1/2 L_ik B_kk
        if ((rc = both({OZ_SYGST_FIX, k, T, M[0], Lp, Ds[0], tb, 0.5, 0}, {OZ_SYGST_FIX, k, T, M[1], Lp, Ds[1], tb, 0.5, 0},
                       (long long)m * 2, m * tile_fl, "ozaki_sygst_fix"))) return rc;
        if ((rc = launch_ozaki_slice2(L, g, SliceJob{M[0], SLICE_PANEL, k, T}, Xs[0],
                                      SliceJob{M[1], SLICE_PANEL, k, T}, Xs[1], m, true))) return rc;
        const long long tasks = (long long)m * (m + 1) / 2;
        // M_ij -= L_ik E_jk^T + E_ik L_jk^T (the two terms of one target in separate launches)
        if ((rc = both({OZ_SYGST_UPD, k, T, M[0], Lp, Xs[0], tb, 1.0, 0}, {OZ_SYGST_UPD, k, T, M[1], Lp, Xs[1], tb, 1.0, 0},
                       tasks * 2, tasks * tile_fl, "ozaki_sygst_update"))) return rc;
        if ((rc = both({OZ_SYGST_UPD, k, T, M[0], Xs[0], Lp, tb, 1.0, 0}, {OZ_SYGST_UPD, k, T, M[1], Xs[1], Lp, tb, 1.0, 0},
                       tasks * 2, tasks * tile_fl, "ozaki_sygst_update"))) return rc;
        // P_ik = E_ik - 1/2 L_ik B_kk
        if ((rc = both({OZ_SYGST_FIX, k, T, M[0], Lp, Ds[0], tb, 0.5, 0}, {OZ_SYGST_FIX, k, T, M[1], Lp, Ds[1], tb, 0.5, 0},
                       (long long)m * 2, m * tile_fl, "ozaki_sygst_fix"))) return rc;
    }
    // B_(m,kk) = W_m (P_(m,kk) - sum_(kk<p<m) L_mp B_(p,kk)), row by row
    for (int m = 1; m < T; ++m) {
        const unsigned char* Wm = Wsl + (size_t)m * tb;
        if ((rc = launch_ozaki_slice2(L, g, SliceJob{M[0], SLICE_ROW, m, T}, Xs[0],
                                      SliceJob{M[1], SLICE_ROW, m, T}, Xs[1], m, false))) return rc;
        if ((rc = both({OZ_ROWSOLVE, m, T, M[0], Wm, Xs[0], tb, -1.0, 1}, {OZ_ROWSOLVE, m, T, M[1], Wm, Xs[1], tb, -1.0, 1},
                       (long long)m * 2, m * tile_fl, "ozaki_sygst_solve"))) return rc;
        const int below = T - m - 1;
        if (below == 0) continue;
        const unsigned char* Lp = LS + strict_lower_pos(m + 1, m, T) * tb;
        if ((rc = launch_ozaki_slice2(L, g, SliceJob{M[0], SLICE_ROW, m, T}, Xs[0],
                                      SliceJob{M[1], SLICE_ROW, m, T}, Xs[1], m, false))) return rc;
        const long long tasks = (long long)below * m;
        // M_(i,kk) -= L_(i,m) M_(m,kk)
        if ((rc = both({OZ_SYGST_ROWUPD, m, T, M[0], Lp, Xs[0], tb, 1.0, 0}, {OZ_SYGST_ROWUPD, m, T, M[1], Lp, Xs[1], tb, 1.0, 0},
                       tasks * 2, tasks * tile_fl, "ozaki_sygst_rowupd"))) return rc;
    }
    L.begin("frob_epilogue");
    k_frob_tiles<<<(unsigned)num_tiles(T), 256, 0, L.stream>>>(g, M0, M1, strips_per_tile(NB), diag_slots, offd_slots);
    L.count();
    return L.end(6.0 * num_tiles(T) * NB * NB, 16.0 * num_tiles(T) * NB * NB);
}

__global__ void k_copy_diag_tiles(const double* __restrict__ Winv, int T, int nb, double* __restrict__ W) {
    const int k = blockIdx.x;
    const double* src = Winv + (long long)k * nb * nb;
    double* dst = W + tile_offset(k, k, T, nb);
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) dst[e] = src[e];
}

int launch_inverse_from_factor(Launcher& L, const Geom& g, const double* S, double* W, double* X,
                               int* status, const unsigned char* LS, unsigned char* scratch,
                               double* Winv, unsigned char* Wsl, unsigned char* Wcs,
                               const MixedPolicy& pol) {
    constexpr int NB = 128;
    if (g.nb != NB) return cudaErrorInvalidValue;
    const int T = g.T;
    const size_t tb = ozaki_tile_bytes();
    const double nb3 = (double)NB * NB * NB, tile_fl = 2.0 * nb3;
    unsigned char* Xs = scratch;                                   // up to T sliced tiles
    int rc = 0;
    const size_t smem_tc = (size_t)NB * (NB + 2) * sizeof(double);
    ensure_smem((const void*)k_trtri_cols<NB>, (int)smem_tc);
    L.begin("trtri");
    k_trtri_cols<NB><<<dim3(NB / 8, T), 256, smem_tc, L.stream>>>(S, T, 0, Winv);
    L.count();
    if ((rc = L.end(T * nb3 / 3.0, 16.0 * T * NB * NB))) return rc;
    SliceJob wr{Winv, SLICE_PTR, 0, T};
    if ((rc = launch_ozaki_slice(L, g, wr, T, true, Wsl))) return rc;
    if ((rc = launch_ozaki_slice(L, g, wr, T, false, Wcs))) return rc;
    // W: diagonal tiles W_kk; below them A_ik = -L_ik W_kk, then row by row
    // W_mk = W_mm A_mk and A_ik -= L_im W_mk (i > m) -- the forward substitution L W = I
    L.begin("copy_tiles");
    k_copy_diag_tiles<<<T, 256, 0, L.stream>>>(Winv, T, NB, W);
    L.count();
    if ((rc = L.end(0.0, 16.0 * T * NB * NB))) return rc;
    for (int k = 0; k + 1 < T; ++k) {
        const int m = T - k - 1;
        const unsigned char* Lp = LS + strict_lower_pos(k + 1, k, T) * tb;
        OzGemmJob a = with_policy({OZ_SYGST_FIX, k, T, W, Lp, Wcs + (size_t)k * tb, tb, 1.0, 1}, pol);
        if ((rc = launch_ozaki_gemm(L, a, (long long)m * 2, m * tile_fl, status, "ozaki_trtri"))) return rc;
    }
    for (int m = 1; m < T; ++m) {
        SliceJob rj{W, SLICE_ROW, m, T};
        if ((rc = launch_ozaki_slice(L, g, rj, m, false, Xs))) return rc;
        OzGemmJob r = with_policy({OZ_ROWSOLVE, m, T, W, Wsl + (size_t)m * tb, Xs, tb, -1.0, 1}, pol);
        if ((rc = launch_ozaki_gemm(L, r, (long long)m * 2, m * tile_fl, status, "ozaki_trtri"))) return rc;
        const int below = T - m - 1;
        if (below == 0) continue;
        if ((rc = launch_ozaki_slice(L, g, rj, m, false, Xs))) return rc;
        const unsigned char* Lp = LS + strict_lower_pos(m + 1, m, T) * tb;
        OzGemmJob u = with_policy({OZ_SYGST_ROWUPD, m, T, W, Lp, Xs, tb, 1.0, 0}, pol);
        if ((rc = launch_ozaki_gemm(L, u, (long long)below * m * 2, below * m * tile_fl, status, "ozaki_trtri"))) return rc;
    }
    // X = W^T W: row p of W contributes W_pi^T W_pj to every (i, j), j <= i <= p
    const size_t slab = (size_t)num_tiles(T) * NB * NB * sizeof(double);
    if (cudaMemsetAsync(X, 0, slab, L.stream) != cudaSuccess) return cudaGetLastError();
    for (int p = 0; p < T; ++p) {
        SliceJob rj{W, SLICE_ROW, p, T};
        if ((rc = launch_ozaki_slice(L, g, rj, p + 1, false, Xs))) return rc;
        const long long tasks = (long long)(p + 1) * (p + 2) / 2;
        OzGemmJob l = with_policy({OZ_LAUUM, p, T, X, Xs, Xs, tb, -1.0, 0}, pol);
        if ((rc = launch_ozaki_gemm(L, l, tasks * 2, tasks * tile_fl, status, "ozaki_lauum"))) return rc;
    }
    return rc;
}

template <int NB>
static int sygst_impl(Launcher& L, const Geom& g, const double* S, double* M0, double* M1,
                      double* diag_slots, double* offd_slots) {
    const int T = g.T;
    constexpr int NS = NB / STRIP;
    constexpr int SB = NB / GB;
    const size_t smem2 = (size_t)(2 * STRIP + NB) * (NB + 1) * sizeof(double);
    ensure_smem((const void*)k_trsm_strip<NB, false, 2, 0>, (int)smem2);
    ensure_smem((const void*)k_trsm_strip<NB, true, 2, 1>, (int)smem2);
    ensure_smem((const void*)k_trsm_strip<NB, true, 2, 2>, (int)smem2);
    const double nb3 = (double)NB * NB * NB;
    const double tb = 8.0 * NB * NB;
    int rc = 0;
    for (int k = 0; k < T; ++k) {
        TrsmParams tp{TRSM_SYGST_DIAG_R, k, T, S, M0, M1, diag_slots};
        L.begin("trsm_sygst");
        k_trsm_strip<NB, false, 2, 0><<<NS, 256, smem2, L.stream>>>(tp);
        L.count();
        tp.mode = TRSM_SYGST_DIAG_L;
        k_trsm_strip<NB, true, 2, 1><<<NS, 256, smem2, L.stream>>>(tp);
        L.count();
        if ((rc = L.end(4.0 * nb3, 6.0 * tb))) return rc;
        const int m = T - k - 1;
        if (m == 0) break;
        tp.mode = TRSM_SYGST_PANEL;
        L.begin("trsm_sygst");
        k_trsm_strip<NB, false, 2, 0><<<m * NS, 256, smem2, L.stream>>>(tp);
        L.count();
        if ((rc = L.end(2.0 * m * nb3, 4.0 * m * tb))) return rc;
        GemmParams gp{GEMM_SYGST_FIX, k, T, S, M0, M1};
        L.begin("gemm_sygst_fix");
        k_gemm_tile<NB, false, 1><<<dim3((unsigned)(m * SB * SB), 2), 256, 0, L.stream>>>(gp);
        L.count();
        if ((rc = L.end(2.0 * m * 2.0 * nb3, 2.0 * m * 4.0 * tb))) return rc;
        const long long tasks = (long long)m * (m + 1) / 2;
        gp.mode = GEMM_SYGST_UPD;
        L.begin("gemm_sygst_update");
        k_gemm_tile<NB, false, 2><<<dim3((unsigned)(tasks * SB * SB), 2), 256, 0, L.stream>>>(gp);
        L.count();
        if ((rc = L.end(2.0 * tasks * 4.0 * nb3, 2.0 * tasks * 5.0 * tb))) return rc;
        gp.mode = GEMM_SYGST_FIX;
        L.begin("gemm_sygst_fix");
        k_gemm_tile<NB, false, 1><<<dim3((unsigned)(m * SB * SB), 2), 256, 0, L.stream>>>(gp);
        L.count();
        if ((rc = L.end(2.0 * m * 2.0 * nb3, 2.0 * m * 4.0 * tb))) return rc;
    }
    // B_(m, kk) = L_mm^-1 (P_(m,kk) - sum_(kk<p<m) L_mp B_(p,kk)), row by row
    for (int m = 1; m < T; ++m) {
        TrsmParams tp{TRSM_SYGST_ROW, m, T, S, M0, M1, offd_slots};
        L.begin("trsm_sygst");
        k_trsm_strip<NB, true, 2, 2><<<m * NS, 256, smem2, L.stream>>>(tp);
        L.count();
        if ((rc = L.end(2.0 * m * nb3, 4.0 * m * tb))) return rc;
        const int below = T - m - 1;
        if (below == 0) continue;
        GemmParams gp{GEMM_SYGST_ROWUPD, m, T, S, M0, M1};
        const long long tasks = (long long)below * m;
        L.begin("gemm_sygst_rowupd");
        k_gemm_tile<NB, true, 1><<<dim3((unsigned)(tasks * SB * SB), 2), 256, 0, L.stream>>>(gp);
        L.count();
        if ((rc = L.end(2.0 * tasks * 2.0 * nb3, 2.0 * tasks * 4.0 * tb))) return rc;
    }
    return rc;
}

int launch_sygst(Launcher& L, const Geom& g, const double* S, double* M0, double* M1,
                 double* diag_slots, double* offd_slots, int* status, int precision,
                 const unsigned char* L_slices, unsigned char* scratch, double* Winv,
                 unsigned char* Wsl, double* Y, const MixedPolicy& pol) {
    if (g.nb == 128 && (precision == PREC_FP64_OZAKI || precision == PREC_MIXED))
        return sygst_ozaki(L, g, S, M0, M1, diag_slots, offd_slots, status, L_slices, scratch, Winv,
                           Wsl, Y, pol);
    if (g.nb == 128) return sygst_impl<128>(L, g, S, M0, M1, diag_slots, offd_slots);
    if (g.nb == 64) return sygst_impl<64>(L, g, S, M0, M1, diag_slots, offd_slots);
    return cudaErrorInvalidValue;
}

}  // namespace fbt
