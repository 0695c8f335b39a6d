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
// exp(-2 pi d / h) for small x) below 1e-17 relative: h = 0.2 for x <= 11, 0.15 for x <= 20,
// then halved each time the range grows 4x.  Each sum stops once its term drops below 1e-17 of
// its running value.
#include <math.h>

#include "fbt_kernels.cuh"
#include "fbt_matern.cuh"

namespace fbt {

__device__ inline double clamp_finite(double v) { return v > 1.0e308 ? 1.0e308 : v; }

__device__ void prep_theta_body(double sigma2, double alpha, double nu, double jitter,
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

__global__ void k_prep_theta(double sigma2, double alpha, double nu, double jitter,
                             ThetaConsts* __restrict__ tc, QuadTables* __restrict__ qt) {
    prep_theta_body(sigma2, alpha, nu, jitter, tc, qt);
}

// theta and the jitter read from device memory (sigma^2, alpha, nu, jitter), so that a captured
// launch sequence serves every theta
__global__ void k_prep_theta_dev(const double* __restrict__ th, ThetaConsts* __restrict__ tc,
                                 QuadTables* __restrict__ qt) {
    prep_theta_body(th[0], th[1], th[2], th[3], tc, qt);
}

// ------------------------------------------------------------------------------------------
// Piecewise polynomials of the three sums for 1 <= x < 1024 (QuadTables::ipoly).
//
// The sums g(x) = e^x K_nu(x), e^x K_(nu-1)(x), e^x dK_nu/dnu(x) are smooth and vary slowly (like
// x^-1/2); their only singularity is at x = 0.  On each interval [a, a + H], H = 2^s / 8 in the
// octave [2^s, 2^(s+1)), the polynomial of degree 11 interpolating g at the 12 Chebyshev points
// errs by about rho^-12 relative with rho ~ 4 a / H >= 32 (Bernstein ellipse clear of 0): about
// 1e-18, below FP64 rounding.  The node values come from the trapezoid sums; the Chebyshev
// coefficients c_k = (2/12) sum_j g(x_j) cos(pi k (j + 1/2) / 12) (c_0 halved) and their
// conversion to powers of t are accumulated in double-double arithmetic (cosines of multiples of
// pi / 24 as double-double constants) and rounded once, so that the evaluation by Horner's rule
// in t in [-1, 1] (terms decreasing) errs by about one rounding.  Each entry then costs one
// polynomial per sum instead of a quadrature.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void dd_two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// (hi, lo) += a * (ch, cl), with the product's rounding error carried
__device__ __forceinline__ void dd_mac(double& hi, double& lo, double a, double ch, double cl) {
    const double p = a * ch;
    const double pe = fma(a, ch, -p);
    double s, e;
    dd_two_sum(hi, p, s, e);
    lo += e + pe + a * cl;
    dd_two_sum(s, lo, hi, lo);
}

// cos(m pi / 24) for m = 0 .. 12 as double-double (head, tail)
static __constant__ double c_cos24[13][2] = {
    {1.0, 0.0},
    {0.9914448613738104, 2.898989874454537e-17},
    {0.9659258262890683, -2.5463971562308955e-17},
    {0.9238795325112867, 1.7645047084336677e-17},
    {0.8660254037844386, 5.0175421109034514e-17},
    {0.7933533402912352, -5.028625073907125e-19},
    {0.7071067811865476, -4.833646656726457e-17},
    {0.6087614290087207, -1.647047979025087e-17},
    {0.5, 0.0},
    {0.3826834323650898, -1.0050772696461588e-17},
    {0.25881904510252074, 2.287249500495561e-17},
    {0.1305261922200516, -9.607666023901524e-18},
    {0.0, 0.0}};

__device__ inline void cos24(int m, double& h, double& l) {
    m %= 48;                                   // cos(m pi / 24), period 48
    if (m > 24) m = 48 - m;                    // even
    const bool neg = m > 12;                   // cos(pi - y) = -cos(y)
    if (neg) m = 24 - m;
    h = neg ? -c_cos24[m][0] : c_cos24[m][0];
    l = neg ? -c_cos24[m][1] : c_cos24[m][1];
}

// one warp (one block) per interval: each lane's quadrature is a long FP64 chain, so the
// intervals are spread over as many SMs as there are intervals
__global__ void __launch_bounds__(32) k_interp_build(const ThetaConsts* __restrict__ tcp, QuadTables* __restrict__ qt) {
    __shared__ double s_g[1][3][IP_DEG];
    __shared__ double s_ch[1][3][IP_DEG], s_cl[1][3][IP_DEG];
    __shared__ int s_B[IP_DEG][IP_DEG];       // coefficient of t^i in T_k: s_B[k][i]
    if (threadIdx.x == 0) {
        for (int k = 0; k < IP_DEG; ++k)
            for (int i = 0; i < IP_DEG; ++i) s_B[k][i] = 0;
        s_B[0][0] = 1;
        s_B[1][1] = 1;
        for (int k = 2; k < IP_DEG; ++k)
            for (int i = 0; i < IP_DEG; ++i) s_B[k][i] = (i > 0 ? 2 * s_B[k - 1][i - 1] : 0) - s_B[k - 2][i];
    }
    __syncthreads();
    const int w = 0, lane = threadIdx.x & 31;
    const int iv = blockIdx.x;
    if (iv >= IP_INTERVALS) return;
    const int s = iv / IP_SUB, k = iv % IP_SUB;
    const double a = ldexp(1.0 + k / (double)IP_SUB, s), H = ldexp(1.0 / IP_SUB, s);
    if (lane < IP_DEG) {
        double ch, cl;
        cos24(2 * lane + 1, ch, cl);           // Chebyshev point t_j = cos(pi (2 j + 1) / 24)
        const double x = a + 0.5 * H * (1.0 + ch);
        double sa, sb, sd;
        quad_sums<true>(x, &qt->st2[0][0], &qt->wa[0][0], &qt->wb[0][0], &qt->wd[0][0], qt->exp2tab, sa, sb, sd);
        s_g[w][0][lane] = sa;
        s_g[w][1][lane] = sb;
        s_g[w][2][lane] = sd;
    }
    __syncwarp();
    if (lane < IP_DEG) {                       // Chebyshev coefficient c_lane of each sum
        for (int q = 0; q < 3; ++q) {
            double hi = 0.0, lo = 0.0;
            for (int j = 0; j < IP_DEG; ++j) {
                double ch, cl;
                cos24(lane * (2 * j + 1), ch, cl);
                dd_mac(hi, lo, s_g[w][q][j], ch, cl);
            }
            // (hi + lo) / 12 in double-double: the head's quotient, its exact remainder
            const double qh = hi / IP_DEG;
            const double r = fma(-qh, (double)IP_DEG, hi);
            double h2, l2;
            dd_two_sum(qh, (r + lo) / IP_DEG, h2, l2);
            if (lane > 0) { h2 *= 2.0; l2 *= 2.0; }
            s_ch[w][q][lane] = h2;
            s_cl[w][q][lane] = l2;
        }
    }
    __syncwarp();
    if (lane < IP_DEG) {                       // power-of-t coefficient a_lane = sum_k c_k B[k][lane]
        for (int q = 0; q < 3; ++q) {
            double hi = 0.0, lo = 0.0;
            for (int kk = 0; kk < IP_DEG; ++kk) {
                const int bk = s_B[kk][lane];
                if (bk == 0) continue;
                dd_mac(hi, lo, (double)bk, s_ch[w][q][kk], s_cl[w][q][kk]);
            }
            qt->ipoly[iv][q][lane] = hi + lo;
        }
    }
}

static int launch_interp_build(Launcher& L, const ThetaConsts* tc, QuadTables* qt) {
    L.begin("prep_theta");
    k_interp_build<<<IP_INTERVALS, 32, 0, L.stream>>>(tc, qt);
    L.count();
    return L.end(0.0, 0.0);
}

int launch_prep_theta_dev(Launcher& L, const double* th, ThetaConsts* tc, QuadTables* qt) {
    L.begin("prep_theta");
    k_prep_theta_dev<<<1, QUAD_NODES, 0, L.stream>>>(th, tc, qt);
    L.count();
    const int rc = L.end(0.0, 0.0);
    return rc ? rc : launch_interp_build(L, tc, qt);
}

int launch_prep_theta(Launcher& L, const double theta[3], double jitter, ThetaConsts* tc,
                      QuadTables* qt) {
    L.begin("prep_theta");
    k_prep_theta<<<1, QUAD_NODES, 0, L.stream>>>(theta[0], theta[1], theta[2], jitter, tc, qt);
    L.count();
    const int rc = L.end(0.0, 0.0);
    return rc ? rc : launch_interp_build(L, tc, qt);
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
            const MaternVals v = matern_corr<DERIV>(x, tc, s_st2, s_wa, s_wb, s_wd, s_etab, &qt->ipoly[0][0][0]);
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
        ensure_smem((const void*)k_generate<true>, (int)smem);
        k_generate<true><<<(unsigned)tiles, 256, smem, L.stream>>>(g, X, Y, tc, qt, S, SA, SN, status);
    } else {
        ensure_smem((const void*)k_generate<false>, (int)smem);
        k_generate<false><<<(unsigned)tiles, 256, smem, L.stream>>>(g, X, Y, tc, qt, S, SA, SN, status);
    }
    L.count();
    // algorithmic bytes: the tile slabs written once
    return L.end(0.0, entries * 8.0 * (deriv ? 3.0 : 1.0));
}

}  // namespace fbt
