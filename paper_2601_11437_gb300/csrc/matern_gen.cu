// Steps a1 and a6: Matern covariance Sigma and its partials Sigma_alpha, Sigma_nu, generated
// straight into the lower-tile layout.
//
// Sec. 2.1 / 2.2 of the paper: with x = h / alpha, R = x^nu K_nu(x) / (2^(nu-1) Gamma(nu)),
//   C = sigma^2 R,  dC/dalpha = sigma^2 / (2^(nu-1) Gamma(nu) alpha) x^(nu+1) K_(nu-1)(x),
//   dC/dnu = sigma^2 (d/dnu[x^nu K_nu(x)] - (log 2 + psi(nu)) x^nu K_nu(x)) / (2^(nu-1) Gamma(nu)),
// and at x = 0: C = sigma^2, both partials 0 (Supp. A, case 1).  Diagonal: sigma^2 (1 + delta).
//
// K_nu, K_(nu-1) and dK_nu/dnu all come from one trapezoid sum over the integral representation
//   K_mu(x) = int_0^inf exp(-x cosh t) cosh(mu t) dt,   dK_nu/dnu = int_0^inf t sinh(nu t) exp(-x cosh t) dt
// written as exp(-x) * sum_j w_j exp(-x * 2 sinh^2(t_j/2)) f(t_j): one exponential per node
// serves all three sums (the paper's five-way case split of Supp. A is replaced by this single
// branch-uniform rule; its truncated series agree with it to their truncation error).  The node
// weights w_j f(t_j) depend only on theta and are tabulated once per evaluation; the step h of
// a level bounds the discretisation error (about exp(-2 pi^2 / (h^2 x)) for large x and
// exp(-2 pi d / h) for small x) below 1e-17 relative: h = 0.15 for x <= 20, halved each time
// the range grows 4x.  Each sum stops once its term drops below 1e-17 of its running value.
#include <math.h>

#include "fbt_kernels.cuh"

namespace fbt {

__constant__ double c_level_h[QUAD_LEVELS] = {0.15, 0.075, 0.0375, 0.01875};
__constant__ double c_level_xmax[QUAD_LEVELS] = {20.0, 80.0, 320.0, 1280.0};
constexpr double X_ZERO_BELOW = 2.5e-15;   // x smaller than this: coincident points, R = 1
constexpr double X_UNDERFLOW = 720.0;      // x larger than this: R and partials underflow to 0
constexpr double STOP_REL = 1e-17;

// psi(x) for x > 0: recurrence psi(x) = psi(x + 1) - 1/x up to x >= 10, then the asymptotic
// series ln x - 1/(2x) - sum_k B_2k / (2k x^2k) with B_2 .. B_14 (DLMF 5.11.2).
__device__ double digamma_pos(double x) {
    double acc = 0.0;
    while (x < 10.0) { acc -= 1.0 / x; x += 1.0; }
    const double b[7] = {1.0 / 6.0, -1.0 / 30.0, 1.0 / 42.0, -1.0 / 30.0, 5.0 / 66.0,
                         -691.0 / 2730.0, 7.0 / 6.0};
    double inv2 = 1.0 / (x * x), p = inv2, s = 0.0;
    for (int k = 0; k < 7; ++k) { s += b[k] / (2.0 * (k + 1)) * p; p *= inv2; }
    return acc + log(x) - 0.5 / x - s;
}

__device__ inline double clamp_finite(double v) { return v > 1.0e308 ? 1.0e308 : v; }

// e^a for a <= 0 by table-driven argument reduction (P. T. P. Tang, "Table-driven implementation
// of the exponential function in IEEE floating-point arithmetic", ACM TOMS 15, 1989):
// a = (64 m + j) ln2/64 + r with |r| <= ln2/128, e^a = 2^m 2^(j/64) e^r, e^r - 1 by its degree-5
// Taylor polynomial (truncation < 4e-17 relative), ln2/64 split into a 36-bit head (n * head is
// exact for |n| < 2^17) and a tail, 2^m applied to the exponent field.  Error ~2 ulp.
__device__ __forceinline__ double exp_nonpos(double a, const double* __restrict__ tab) {
    if (a < -700.0) return 0.0;                                 // keeps 2^m y a normal number
    const double n = rint(a * 92.33248261689366);               // 64 / ln 2
    double r = fma(-n, 0x1.62e42fefa0000p-7, a);               // ln 2 / 64, head
    r = fma(-n, 0x1.cf79abc9e3b3ap-46, r);                      // ln 2 / 64, tail
    const int ni = (int)n;
    const int j = ni & (EXP_TABLE - 1), m = ni >> 6;
    const double p = r * fma(r, fma(r, fma(r, fma(r, 1.0 / 120.0, 1.0 / 24.0), 1.0 / 6.0), 0.5), 1.0);
    const double y = fma(tab[j], p, tab[j]);                    // 2^(j/64) e^r in [1, 2)
    return __longlong_as_double(__double_as_longlong(y) + ((long long)m << 52));
}

__global__ void k_prep_theta(double sigma2, double alpha, double nu, double jitter,
                             ThetaConsts* __restrict__ tc, QuadTables* __restrict__ qt) {
    const int j = threadIdx.x;
    if (j < EXP_TABLE) qt->exp2tab[j] = exp2(j / (double)EXP_TABLE);
    for (int l = 0; l < QUAD_LEVELS; ++l) {
        const double h = c_level_h[l];
        const double t = j * h;
        const double w = j == 0 ? 0.5 * h : h;   // trapezoid on [0, inf) of an even integrand
        const double sh = sinh(0.5 * t);
        qt->st2[l][j] = 2.0 * sh * sh;
        qt->wa[l][j] = clamp_finite(w * cosh(nu * t));
        qt->wb[l][j] = clamp_finite(w * cosh((nu - 1.0) * t));
        qt->wd[l][j] = clamp_finite(w * t * sinh(nu * t));
    }
    if (j == 0) {
        tc->sigma2 = sigma2;
        tc->alpha = alpha;
        tc->nu = nu;
        tc->inv_alpha = 1.0 / alpha;
        tc->norm = exp(-(nu - 1.0) * 0.69314718055994530942 - lgamma(nu));
        tc->c_nu = 0.69314718055994530942 + digamma_pos(nu);
        tc->jitter = jitter;
    }
}

int launch_prep_theta(Launcher& L, const double theta[3], double jitter, ThetaConsts* tc,
                      QuadTables* qt) {
    L.begin("prep_theta");
    k_prep_theta<<<1, QUAD_NODES, 0, L.stream>>>(theta[0], theta[1], theta[2], jitter, tc, qt);
    L.count();
    return L.end(0.0, 0.0);
}

struct MaternVals { double r, da, dn; };

// R(x), dR/dalpha, dR/dnu for x > 0 with tables in shared memory.
template <bool DERIV>
__device__ __forceinline__ MaternVals matern_corr(double x, const ThetaConsts& tc,
                                                  const double* __restrict__ st2,
                                                  const double* __restrict__ wa,
                                                  const double* __restrict__ wb,
                                                  const double* __restrict__ wd,
                                                  const double* __restrict__ etab) {
    MaternVals v{0.0, 0.0, 0.0};
    if (x < X_ZERO_BELOW) { v.r = 1.0; return v; }
    if (x > X_UNDERFLOW) return v;
    int l = x <= c_level_xmax[0] ? 0 : x <= c_level_xmax[1] ? 1 : x <= c_level_xmax[2] ? 2 : 3;
    const int base = l * QUAD_NODES;
    double sa = 0.0, sb = 0.0, sd = 0.0;
    // four nodes per round; the stopping test (last terms below STOP_REL of the sums, which
    // can only happen past the integrand's peak) is evaluated once per round
    for (int j = 0; j < QUAD_NODES; j += 4) {
        double ta = 0.0, tb = 0.0, td = 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double e = exp_nonpos(-x * st2[base + j + u], etab);
            ta = e * wa[base + j + u];
            sa += ta;
            if (DERIV) {
                tb = e * wb[base + j + u];
                td = e * wd[base + j + u];
                sb += tb;
                sd += td;
            }
        }
        bool done = ta <= STOP_REL * sa;
        if (DERIV) done = done && tb <= STOP_REL * sb && td <= STOP_REL * sd;
        if (done) break;
    }
    const double lx = log(x);
    const double P = tc.norm * exp(tc.nu * lx - x);      // x^nu e^-x / (2^(nu-1) Gamma(nu))
    v.r = P * sa;
    if (DERIV) {
        v.da = P * x * sb * tc.inv_alpha;
        v.dn = P * ((lx - tc.c_nu) * sa + sd);
    }
    return v;
}

// One block per lower tile (column-major tile order), the whole nb x nb tile (diagonal tiles
// in full, both triangles), written column-major with consecutive threads on consecutive rows.
template <bool DERIV>
__global__ void __launch_bounds__(256) k_generate(Geom g, const double* __restrict__ X,
                                                  const double* __restrict__ Y,
                                                  const ThetaConsts* __restrict__ tcp,
                                                  const QuadTables* __restrict__ qt,
                                                  double* __restrict__ S, double* __restrict__ SA,
                                                  double* __restrict__ SN, int* status) {
    extern __shared__ double sm[];
    constexpr int NTAB = QUAD_LEVELS * QUAD_NODES;
    double* s_st2 = sm;
    double* s_wa = sm + NTAB;
    double* s_wb = sm + 2 * NTAB;
    double* s_wd = sm + 3 * NTAB;
    double* s_xy = sm + (DERIV ? 4 : 2) * NTAB;
    double* s_etab = s_xy + 4 * g.nb;
    const int nb = g.nb, T = g.T;
    for (int q = threadIdx.x; q < EXP_TABLE; q += blockDim.x) s_etab[q] = qt->exp2tab[q];
    for (int q = threadIdx.x; q < NTAB; q += blockDim.x) {
        s_st2[q] = (&qt->st2[0][0])[q];
        s_wa[q] = (&qt->wa[0][0])[q];
        if (DERIV) {
            s_wb[q] = (&qt->wb[0][0])[q];
            s_wd[q] = (&qt->wd[0][0])[q];
        }
    }
    // tile (i, j) from the linear column-major lower-tile index
    const long long t = blockIdx.x;
    int j = (int)(((2.0 * T + 1.0) - sqrt((2.0 * T + 1.0) * (2.0 * T + 1.0) - 8.0 * (double)t)) * 0.5);
    if (j < 0) j = 0;
    while (j > 0 && tile_index(j, j, T) > t) --j;
    while (j + 1 < T && tile_index(j + 1, j + 1, T) <= t) ++j;
    const int i = j + (int)(t - tile_index(j, j, T));
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
        s_xy[q] = X[(long long)i * nb + q];
        s_xy[nb + q] = Y[(long long)i * nb + q];
        s_xy[2 * nb + q] = X[(long long)j * nb + q];
        s_xy[3 * nb + q] = Y[(long long)j * nb + q];
    }
    __syncthreads();
    const ThetaConsts tc = *tcp;
    const long long base = t * (long long)nb * nb;
    bool bad = false;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int r = e % nb, c = e / nb;
        const long long gr = (long long)i * nb + r, gc = (long long)j * nb + c;
        double s, sa = 0.0, sn = 0.0;
        if (gr >= g.n || gc >= g.n) {
            s = gr == gc ? 1.0 : 0.0;
        } else if (gr == gc) {
            s = tc.sigma2 * (1.0 + tc.jitter);
        } else {
            const double dx = s_xy[r] - s_xy[2 * nb + c];
            const double dy = s_xy[nb + r] - s_xy[3 * nb + c];
            const double x = sqrt(dx * dx + dy * dy) * tc.inv_alpha;
            const MaternVals v = matern_corr<DERIV>(x, tc, s_st2, s_wa, s_wb, s_wd, s_etab);
            s = tc.sigma2 * v.r;
            sa = tc.sigma2 * v.da;
            sn = tc.sigma2 * v.dn;
        }
        bad |= !isfinite(s) || (DERIV && (!isfinite(sa) || !isfinite(sn)));
        if (S) S[base + e] = s;            // S == nullptr: Sigma's factor is kept, partials only
        if (DERIV) {
            SA[base + e] = sa;
            SN[base + e] = sn;
        }
    }
    if (bad) atomicOr(status, ST_BESSEL);
}

int launch_generate(Launcher& L, const Geom& g, const double* X, const double* Y,
                    const ThetaConsts* tc, const QuadTables* qt, double* S, double* SA,
                    double* SN, bool deriv, int* status) {
    const long long tiles = num_tiles(g.T);
    const size_t smem = (size_t)((deriv ? 4 : 2) * QUAD_LEVELS * QUAD_NODES + 4 * g.nb + EXP_TABLE) * sizeof(double);
    const double entries = (double)tiles * g.nb * g.nb;
    L.begin(deriv ? "generate_deriv" : "generate");
    if (deriv) {
        cudaFuncSetAttribute(k_generate<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_generate<true><<<(unsigned)tiles, 256, smem, L.stream>>>(g, X, Y, tc, qt, S, SA, SN, status);
    } else {
        cudaFuncSetAttribute(k_generate<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_generate<false><<<(unsigned)tiles, 256, smem, L.stream>>>(g, X, Y, tc, qt, S, SA, SN, status);
    }
    L.count();
    // algorithmic bytes: the tile slabs written once
    return L.end(0.0, entries * 8.0 * (deriv ? 3.0 : 1.0));
}

}  // namespace fbt
