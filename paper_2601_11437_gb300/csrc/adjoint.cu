// Adjoint of the log-likelihood with respect to theta (Eq. 2 in trace form):
//   dl/dtheta_i = 1/2 sum_(r,c) (w_r w_c - (Sigma^-1)_rc) (Sigma_i)_rc,   w = Sigma^-1 z,
// with Sigma_alpha and Sigma_nu regenerated entry by entry inside the reduction and never
// stored.  Sigma^-1 comes from the factor (launch_inverse_from_factor).  For sigma^2 the
// closed form of Algorithm 3, Step 2 applies.
#include <math.h>

#include "fbt_kernels.cuh"
#include "fbt_matern.cuh"

namespace fbt {

__global__ void __launch_bounds__(256) k_adjoint_reduce(Geom g, const double* __restrict__ Xc,
                                                        const double* __restrict__ Yc,
                                                        const double* __restrict__ Xinv,
                                                        const double* __restrict__ w,
                                                        const ThetaConsts* __restrict__ tcp,
                                                        const QuadTables* __restrict__ qt,
                                                        double* __restrict__ slots) {
    extern __shared__ double sm[];
    constexpr int NTAB = QUAD_LEVELS * QUAD_NODES;
    double* s_st2 = sm;
    double* s_wa = sm + NTAB;
    double* s_wb = sm + 2 * NTAB;
    double* s_wd = sm + 3 * NTAB;
    double* s_xy = sm + 4 * NTAB;
    double* s_w = s_xy + 4 * g.nb;
    double* s_etab = s_w + 2 * g.nb;
    __shared__ double red[2][256];
    const int nb = g.nb, T = g.T;
    for (int q = threadIdx.x; q < EXP_TABLE; q += blockDim.x) s_etab[q] = qt->exp2tab[q];
    for (int q = threadIdx.x; q < NTAB; q += blockDim.x) {
        s_st2[q] = (&qt->st2[0][0])[q];
        s_wa[q] = (&qt->wa[0][0])[q];
        s_wb[q] = (&qt->wb[0][0])[q];
        s_wd[q] = (&qt->wd[0][0])[q];
    }
    const long long t = blockIdx.x;
    int j = (int)(((2.0 * T + 1.0) - sqrt((2.0 * T + 1.0) * (2.0 * T + 1.0) - 8.0 * (double)t)) * 0.5);
    if (j < 0) j = 0;
    while (j > 0 && tile_index(j, j, T) > t) --j;
    while (j + 1 < T && tile_index(j + 1, j + 1, T) <= t) ++j;
    const int i = j + (int)(t - tile_index(j, j, T));
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
        s_xy[q] = Xc[(long long)i * nb + q];
        s_xy[nb + q] = Yc[(long long)i * nb + q];
        s_xy[2 * nb + q] = Xc[(long long)j * nb + q];
        s_xy[3 * nb + q] = Yc[(long long)j * nb + q];
        s_w[q] = w[(long long)i * nb + q];
        s_w[nb + q] = w[(long long)j * nb + q];
    }
    __syncthreads();
    const ThetaConsts tc = *tcp;
    const long long base = t * (long long)nb * nb;
    double ga = 0.0, gn = 0.0;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int r = e % nb, c = e / nb;
        const long long gr = (long long)i * nb + r, gc = (long long)j * nb + c;
        if (gr >= g.n || gc >= g.n || gr == gc) continue;      // padding; the partials vanish at h = 0
        const double dx = s_xy[r] - s_xy[2 * nb + c];
        const double dy = s_xy[nb + r] - s_xy[3 * nb + c];
        const double x = sqrt(dx * dx + dy * dy) * tc.inv_alpha;
        const MaternVals v = matern_corr<true>(x, tc, s_st2, s_wa, s_wb, s_wd, s_etab, &qt->ipoly[0][0][0]);
        const double wt = fma(s_w[r], s_w[nb + c], -Xinv[base + e]);
        ga = fma(wt, v.da, ga);
        gn = fma(wt, v.dn, gn);
    }
    red[0][threadIdx.x] = ga;
    red[1][threadIdx.x] = gn;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double f = (i == j ? 1.0 : 2.0) * tc.sigma2;      // upper tiles mirror the lower ones
        slots[2 * t] = f * red[0][0];
        slots[2 * t + 1] = f * red[1][0];
    }
}

int launch_adjoint_reduce(Launcher& L, const Geom& g, const double* Xs, const double* Yc,
                          const double* X, const double* w, const ThetaConsts* tc,
                          const QuadTables* qt, double* slots, int* status) {
    (void)status;
    const long long tiles = num_tiles(g.T);
    const size_t smem = (size_t)(4 * QUAD_LEVELS * QUAD_NODES + 6 * g.nb + EXP_TABLE) * sizeof(double);
    ensure_smem((const void*)k_adjoint_reduce, (int)smem);
    L.begin("adjoint_reduce");
    k_adjoint_reduce<<<(unsigned)tiles, 256, smem, L.stream>>>(g, Xs, Yc, X, w, tc, qt, slots);
    L.count();
    return L.end(0.0, 8.0 * (double)tiles * g.nb * g.nb);
}

}  // namespace fbt
