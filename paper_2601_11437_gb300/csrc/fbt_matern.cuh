// Per-entry Matern correlation and its partials (trapezoid quadrature of K_nu, K_(nu-1) and
// dK_nu/dnu with one exponential per node), shared by the tile generator and the adjoint
// reduction.  See matern_gen.cu for the derivation.
#pragma once

#include <math.h>

#include "fbt_kernels.cuh"

namespace fbt {

// Step h of each level and the largest x it serves.  For large x the discretisation error is
// about exp(-2 pi^2 / (h^2 x)) (the integrand is close to a Gaussian of variance 1 / x), below
// 1e-18 while h^2 x <= 0.476; for small x it is about exp(-2 pi d / h) with d just below pi / 2,
// the half-width of the strip where the integrand stays analytic and decaying: below 1e-18 for
// h <= 0.2 (the level h = 0.2 serves x <= 11).
static __constant__ double c_level_h[QUAD_LEVELS] = {0.2, 0.15, 0.075, 0.0375, 0.01875};
static __constant__ double c_level_xmax[QUAD_LEVELS] = {11.0, 20.0, 80.0, 320.0, 1280.0};
constexpr double X_ZERO_BELOW = 2.5e-15;   // x smaller than this: coincident points, R = 1
constexpr double X_UNDERFLOW = 720.0;      // x larger than this: R and partials underflow to 0
constexpr double STOP_REL = 1e-17;

// psi(x) for x > 0: recurrence psi(x) = psi(x + 1) - 1/x up to x >= 10, then the asymptotic
// series ln x - 1/(2x) - sum_k B_2k / (2k x^2k) with B_2 .. B_14 (DLMF 5.11.2).
static __device__ double digamma_pos(double x) {
    double acc = 0.0;
    while (x < 10.0) { acc -= 1.0 / x; x += 1.0; }
    const double b[7] = {1.0 / 6.0, -1.0 / 30.0, 1.0 / 42.0, -1.0 / 30.0, 5.0 / 66.0,
                         -691.0 / 2730.0, 7.0 / 6.0};
    double inv2 = 1.0 / (x * x), p = inv2, s = 0.0;
    for (int k = 0; k < 7; ++k) { s += b[k] / (2.0 * (k + 1)) * p; p *= inv2; }
    return acc + log(x) - 0.5 / x - s;
}

// e^a for a <= 700 by table-driven argument reduction (P. T. P. Tang, "Table-driven implementation
// of the exponential function in IEEE floating-point arithmetic", ACM TOMS 15, 1989):
// a = (256 m + j) ln2/256 + r with |r| <= ln2/512, e^a = 2^m 2^(j/256) e^r, e^r - 1 by its
// degree-4 Taylor polynomial (truncation below 4e-17 relative, odd in r), ln2/256 split into a
// 35-bit head (n * head is exact for |n| < 2^18) and a tail, 2^m applied to the exponent field.
__device__ __forceinline__ double exp_nonpos(double a, const double* __restrict__ tab) {
    if (a < -700.0) return 0.0;                                 // keeps 2^m y a normal number
                                                                // (a <= 700: no overflow either)
    const double n = rint(a * 369.3299304675746);              // 256 / ln 2
    double r = fma(-n, 0x1.62e42fefc0000p-9, a);               // ln 2 / 256, head
    r = fma(-n, -0x1.c610ca86c3899p-45, r);                     // ln 2 / 256, tail
    const int ni = (int)n;
    const int j = ni & (EXP_TABLE - 1), m = ni >> 8;
    const double p = r * fma(r, fma(r, fma(r, 1.0 / 24.0, 1.0 / 6.0), 0.5), 1.0);
    const double y = fma(tab[j], p, tab[j]);                    // 2^(j/256) e^r in [1, 2)
    return __longlong_as_double(__double_as_longlong(y) + ((long long)m << 52));
}

struct MaternVals { double r, da, dn; };

// The trapezoid sums e^x K_nu(x), e^x K_(nu-1)(x), e^x dK_nu/dnu(x) (sa, sb, sd) at x > 0 with
// tables in shared (or global) memory.
template <bool DERIV>
__device__ __forceinline__ void quad_sums(double x, const double* __restrict__ st2, const double* __restrict__ wa,
                                          const double* __restrict__ wb, const double* __restrict__ wd,
                                          const double* __restrict__ etab, double& sa, double& sb, double& sd) {
    int l = x <= c_level_xmax[0] ? 0 : x <= c_level_xmax[1] ? 1 : x <= c_level_xmax[2] ? 2 : x <= c_level_xmax[3] ? 3 : 4;
    const int base = l * QUAD_NODES;
    sa = 0.0;
    sb = 0.0;
    sd = 0.0;
    // four nodes per round; the stopping test (last terms below STOP_REL of the sums, which
    // can only happen past the integrand's peak) is evaluated once per round
    for (int j = 0; j < QUAD_NODES; j += 4) {
        double e = 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            e = exp_nonpos(-x * st2[base + j + u], etab);
            sa = fma(e, wa[base + j + u], sa);
            if (DERIV) {
                sb = fma(e, wb[base + j + u], sb);
                sd = fma(e, wd[base + j + u], sd);
            }
        }
        // the round's last terms against the sums (the terms decrease past the peak)
        bool done = e * wa[base + j + 3] <= STOP_REL * sa;
        if (DERIV) done = done && e * wb[base + j + 3] <= STOP_REL * sb && e * wd[base + j + 3] <= STOP_REL * sd;
        if (done) break;
    }
}

// The same sums from the piecewise polynomials (ip = QuadTables::ipoly) for 1 <= x < 1024.  The
// octave s and the position f in it, x = 2^s (1 + f), come from the bits of x; interval
// k = floor(8 f) and t = 16 f - 2 k - 1 in [-1, 1] are exact.
template <bool DERIV>
__device__ __forceinline__ void interp_sums(double x, const double* __restrict__ ip, double& sa, double& sb,
                                            double& sd) {
    const long long b = __double_as_longlong(x);
    const int s = (int)(b >> 52) - 1023;
    const double f = __longlong_as_double((b & 0xFFFFFFFFFFFFFll) | 0x3FF0000000000000ll) - 1.0;
    const int k = (int)(f * IP_SUB);
    const double t = f * (2 * IP_SUB) - (2 * k + 1);
    const double* __restrict__ a = ip + (size_t)((s * IP_SUB + k) * 3) * IP_DEG;
    double pa = __ldg(a + IP_DEG - 1), pb = 0.0, pd = 0.0;
    if (DERIV) {
        pb = __ldg(a + 2 * IP_DEG - 1);
        pd = __ldg(a + 3 * IP_DEG - 1);
    }
#pragma unroll
    for (int i = IP_DEG - 2; i >= 0; --i) {
        pa = fma(pa, t, __ldg(a + i));
        if (DERIV) {
            pb = fma(pb, t, __ldg(a + IP_DEG + i));
            pd = fma(pd, t, __ldg(a + 2 * IP_DEG + i));
        }
    }
    sa = pa;
    sb = pb;
    sd = pd;
}

// R(x), dR/dalpha, dR/dnu for x > 0 with tables in shared memory; ip (optional): the piecewise
// polynomials of the sums, used for 1 <= x < 1024 (ip == nullptr: the quadrature everywhere).
template <bool DERIV>
__device__ __forceinline__ MaternVals matern_corr(double x, const ThetaConsts& tc,
                                                  const double* __restrict__ st2,
                                                  const double* __restrict__ wa,
                                                  const double* __restrict__ wb,
                                                  const double* __restrict__ wd,
                                                  const double* __restrict__ etab,
                                                  const double* __restrict__ ip = nullptr) {
    MaternVals v{0.0, 0.0, 0.0};
    if (x < X_ZERO_BELOW) { v.r = 1.0; return v; }
    if (x > X_UNDERFLOW) return v;
    double sa, sb, sd;
    if (ip && x >= 1.0) interp_sums<DERIV>(x, ip, sa, sb, sd);
    else quad_sums<DERIV>(x, st2, wa, wb, wd, etab, sa, sb, sd);
    const double lx = log(x);
    // x^nu e^-x / (2^(nu-1) Gamma(nu)); nu log x - x <= nu (log nu - 1) stays far below 700
    const double P = tc.norm * exp_nonpos(tc.nu * lx - x, etab);
    v.r = P * sa;
    if (DERIV) {
        v.da = P * x * sb * tc.inv_alpha;
        v.dn = P * ((lx - tc.c_nu) * sa + sd);
    }
    return v;
}


}  // namespace fbt
