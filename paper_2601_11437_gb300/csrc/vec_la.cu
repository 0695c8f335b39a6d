// Steps a4, a5, a9, a10: triangular solves y = L^-1 z and w = L^-T y (Algorithm 2/3), the
// quadratic forms w^T Sigma_i w (Algorithm 3, Steps 3-4), and the assembly of l, score and
// Fisher information (Eq. 1-3, Algorithm 3 Step 2's closed forms for sigma^2).
//
// All reductions sum per-tile / per-thread partials in a fixed order, so every result is
// bitwise reproducible from run to run.
#include <math.h>

#include "fbt_kernels.cuh"

namespace fbt {

// v_m <- L_mm^-1 v_m (trans = false) or L_mm^-T v_m (trans = true), one CTA.
template <bool TRANS>
__global__ void __launch_bounds__(256) k_trsv_diag(const double* __restrict__ S, int T, int nb,
                                                   int m, double* __restrict__ v) {
    // the tile's lower triangle is staged in shared memory (leading dimension nb + 1: column and
    // row walks are both free of bank conflicts), then one warp runs the substitution with the
    // vector in registers, lane l holding entries l, l + 32, l + 64, l + 96: no block barrier
    // inside the sequential loop
    extern __shared__ double A[];
    const int LD = nb + 1;
    double* rinv = A + nb * LD;                // 1 / L_dd, computed in parallel before the
    const double* __restrict__ Lt = S + tile_offset(m, m, T, nb);   // sequential loop
    // 16-byte loads, many in flight per thread: one CTA must pull the whole tile
    const double2* __restrict__ L2 = (const double2*)Lt;
#pragma unroll 16
    for (int e2 = threadIdx.x; e2 < nb * nb / 2; e2 += blockDim.x) {
        const double2 w = L2[e2];
        const int r = (2 * e2) % nb, c = (2 * e2) / nb;
        if (r >= c) A[r + c * LD] = w.x;
        if (r + 1 >= c) A[r + 1 + c * LD] = w.y;
    }
    for (int d = threadIdx.x; d < nb; d += blockDim.x) rinv[d] = 1.0 / Lt[d + (long long)d * nb];
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    double* vm = v + (long long)m * nb;
    const int nblk = nb / 32;
    double x[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) x[s] = s < nblk ? vm[lane + 32 * s] : 0.0;
    if (!TRANS) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (s >= nblk) break;
            for (int dd = 0; dd < 32; ++dd) {
                const int d = 32 * s + dd;
                double xd = 0.0;
                if (lane == dd) { xd = x[s] * rinv[d]; x[s] = xd; }
                xd = __shfl_sync(0xffffffffu, xd, dd);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int r = lane + 32 * t;
                    if (t >= s && t < nblk && r > d) x[t] -= A[r + d * LD] * xd;
                }
            }
        }
    } else {
#pragma unroll
        for (int s = 3; s >= 0; --s) {
            if (s >= nblk) continue;
            for (int dd = 31; dd >= 0; --dd) {
                const int d = 32 * s + dd;
                double xd = 0.0;
                if (lane == dd) { xd = x[s] * rinv[d]; x[s] = xd; }
                xd = __shfl_sync(0xffffffffu, xd, dd);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int r = lane + 32 * t;
                    if (t <= s && r < d) x[t] -= A[d + r * LD] * xd;     // L[d][r], r < d
                }
            }
        }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
        if (s < nblk) vm[lane + 32 * s] = x[s];
}

// One 32-entry chunk q of A x (TRANS = false) or A^T x (TRANS = true) for a column-major
// nb x nb tile A and the vector x staged in shared memory; 256 threads, nb in {64, 128}. Each
// output entry is owned by one CTA and summed in a fixed order, so results are reproducible.
// The value is returned in threads 0..31 (entry 32 q + threadIdx.x).
template <bool TRANS>
__device__ __forceinline__ double chunk_matvec(const double* __restrict__ A, int nb, const double* sx,
                                               double* part, int q) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (!TRANS) {
        // rows 32 q + lane; warp w takes columns [w nb / 8, (w + 1) nb / 8): every load of a warp
        // is 32 consecutive doubles of one column, all nb / 8 of them in flight at once
        const int cw = nb >> 3, c0 = warp * cw;
        const double* __restrict__ a = A + 32 * q + lane + (long long)c0 * nb;
        double acc = 0.0;
#pragma unroll 16
        for (int c = 0; c < cw; ++c) acc = fma(a[(long long)c * nb], sx[c0 + c], acc);
        part[warp * 32 + lane] = acc;
    } else {
        // entries 32 q + 4 w + j are dots of whole (contiguous) columns with x, lanes over rows
        const int nr = nb >> 5;
        double acc[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const double* __restrict__ col = A + (long long)(32 * q + 4 * warp + j) * nb;
            acc[j] = 0.0;
#pragma unroll
            for (int s = 0; s < 4; ++s)
                if (s < nr) acc[j] = fma(col[lane + 32 * s], sx[lane + 32 * s], acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            for (int off = 16; off > 0; off >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], off);
            if (lane == 0) part[4 * warp + j] = acc[j];
        }
    }
    __syncthreads();
    double y = 0.0;
    if (threadIdx.x < 32) {
        if (!TRANS) {
#pragma unroll
            for (int w = 0; w < 8; ++w) y += part[w * 32 + threadIdx.x];
        } else {
            y = part[threadIdx.x];
        }
    }
    return y;
}

// The diagonal step as a product with the inverted diagonal tile W_m = L_mm^-1 (when the
// emulated path has it): x = W_m v_m (forward) or W_m^T v_m (backward), written to x (nb
// doubles) rather than in place, because the nb / 32 CTAs of the launch all read v_m.
template <bool TRANS>
__global__ void __launch_bounds__(256) k_trsv_diag_inv(const double* __restrict__ Winv, int nb, int m,
                                                       const double* __restrict__ v, double* __restrict__ x) {
    __shared__ double sb[128];
    __shared__ double part[256];
    const double* vm = v + (long long)m * nb;
    for (int d = threadIdx.x; d < nb; d += blockDim.x) sb[d] = vm[d];
    __syncthreads();
    const double y = chunk_matvec<TRANS>(Winv + (long long)m * nb * nb, nb, sb, part, blockIdx.x);
    if (threadIdx.x < 32) x[32 * blockIdx.x + threadIdx.x] = y;
}

// forward: v_i -= L(i, m) x for i > m; backward: v_p -= L(m, p)^T x for p < m, where x is
// the solved block m. Grid (nb / 32, tiles): CTA (q, t) owns entries 32 q .. 32 q + 31 of one
// updated block, so a step reads its column (row) of tiles with nb / 32 times as many CTAs as
// tiles. When copy_x is set, x came from k_trsv_diag_inv and the first tile's CTAs also store
// it into v_m (nothing else in the launch touches v_m).
template <bool TRANS>
__global__ void __launch_bounds__(256) k_trsv_update(const double* __restrict__ S, int T, int nb, int m,
                                                     const double* x, double* v, int copy_x) {
    __shared__ double sx[128];
    __shared__ double part[256];
    for (int d = threadIdx.x; d < nb; d += blockDim.x) sx[d] = x[d];
    __syncthreads();
    const int q = blockIdx.x;
    if (copy_x && blockIdx.y == 0 && threadIdx.x < 32)
        v[(long long)m * nb + 32 * q + threadIdx.x] = sx[32 * q + threadIdx.x];
    const int t = TRANS ? (int)blockIdx.y : m + 1 + (int)blockIdx.y;
    const double* __restrict__ A = S + (TRANS ? tile_offset(m, t, T, nb) : tile_offset(t, m, T, nb));
    const double y = chunk_matvec<TRANS>(A, nb, sx, part, q);
    if (threadIdx.x < 32) v[(long long)t * nb + 32 * q + threadIdx.x] -= y;
}

int launch_trsv(Launcher& L, const Geom& g, const double* S, double* v, bool trans, const double* winv,
                double* vx) {
    const int T = g.T, nb = g.nb;
    if (winv && !vx) return (int)cudaErrorInvalidValue;
    const size_t smem_diag = (size_t)nb * (nb + 2) * sizeof(double);
    ensure_smem((const void*)k_trsv_diag<false>, (int)smem_diag);
    ensure_smem((const void*)k_trsv_diag<true>, (int)smem_diag);
    const double tb = 8.0 * nb * nb;
    const int chunks = nb / 32;
    int rc = 0;
    L.begin(trans ? "trsv_backward" : "trsv_forward");
    for (int k = 0; k < T; ++k) {
        const int m = trans ? T - 1 - k : k;
        const int rest = trans ? m : T - 1 - m;          // tiles updated by this step
        if (winv) {
            if (trans) k_trsv_diag_inv<true><<<chunks, 256, 0, L.stream>>>(winv, nb, m, v, vx);
            else k_trsv_diag_inv<false><<<chunks, 256, 0, L.stream>>>(winv, nb, m, v, vx);
        } else {
            if (trans) k_trsv_diag<true><<<1, 256, smem_diag, L.stream>>>(S, T, nb, m, v);
            else k_trsv_diag<false><<<1, 256, smem_diag, L.stream>>>(S, T, nb, m, v);
        }
        L.count();
        const double* x = winv ? vx : v + (long long)m * nb;
        if (rest > 0) {
            const dim3 grid(chunks, rest);
            if (trans) k_trsv_update<true><<<grid, 256, 0, L.stream>>>(S, T, nb, m, x, v, winv ? 1 : 0);
            else k_trsv_update<false><<<grid, 256, 0, L.stream>>>(S, T, nb, m, x, v, winv ? 1 : 0);
            L.count();
        } else if (winv) {
            const cudaError_t e = cudaMemcpyAsync(v + (long long)m * nb, vx, (size_t)nb * sizeof(double),
                                                  cudaMemcpyDeviceToDevice, L.stream);
            if (e != cudaSuccess) return (int)e;
        }
    }
    // algorithmic: n_pad^2 flops (one multiply-add per stored lower entry), the lower triangle read once
    const double ntri = (double)num_tiles(T);
    rc = L.end((double)g.npad * g.npad, ntri * tb);
    return rc;
}

// Per-tile partial of w^T M w over the lower tiles for M0 and M1 (off-diagonal tiles doubled,
// since the upper tiles are their transposes); diagonal tiles are stored in full.
__global__ void __launch_bounds__(256) k_qform(Geom g, const double* __restrict__ M0,
                                               const double* __restrict__ M1,
                                               const double* __restrict__ w,
                                               double* __restrict__ slots) {
    __shared__ double red[2][8];
    const int T = g.T, nb = g.nb;
    const long long t = blockIdx.x;
    int j = (int)(((2.0 * T + 1.0) - sqrt((2.0 * T + 1.0) * (2.0 * T + 1.0) - 8.0 * (double)t)) * 0.5);
    if (j < 0) j = 0;
    while (j > 0 && tile_index(j, j, T) > t) --j;
    while (j + 1 < T && tile_index(j + 1, j + 1, T) <= t) ++j;
    const int i = j + (int)(t - tile_index(j, j, T));
    const double* wi = w + (long long)i * nb;
    const double* wj = w + (long long)j * nb;
    const long long base = t * (long long)nb * nb;
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    double a0 = 0.0, a1 = 0.0;
    for (int c = warp; c < nb; c += 8) {
        double s0 = 0.0, s1 = 0.0;
        for (int r = lane; r < nb; r += 32) {
            const long long e = base + r + (long long)c * nb;
            s0 = fma(M0[e], wi[r], s0);
            s1 = fma(M1[e], wi[r], s1);
        }
        a0 = fma(s0, wj[c], a0);
        a1 = fma(s1, wj[c], a1);
    }
    for (int off = 16; off > 0; off >>= 1) {
        a0 += __shfl_down_sync(0xffffffffu, a0, off);
        a1 += __shfl_down_sync(0xffffffffu, a1, off);
    }
    if (lane == 0) { red[0][warp] = a0; red[1][warp] = a1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int q = 0; q < 8; ++q) { s0 += red[0][q]; s1 += red[1][q]; }
        const double f = i == j ? 1.0 : 2.0;
        slots[2 * t] = f * s0;
        slots[2 * t + 1] = f * s1;
    }
}

int launch_qform(Launcher& L, const Geom& g, const double* M0, const double* M1, const double* w,
                 double* qform_slots) {
    const long long tiles = num_tiles(g.T);
    L.begin("qform");
    k_qform<<<(unsigned)tiles, 256, 0, L.stream>>>(g, M0, M1, w, qform_slots);
    L.count();
    const double e = (double)tiles * g.nb * g.nb;
    return L.end(4.0 * e, 16.0 * e);
}

// fixed-order block sum of src[0..count) with stride `stride` starting at `first`
__device__ double block_sum(const double* __restrict__ src, long long count, int stride, int first,
                            double* red) {
    double s = 0.0;
    for (long long q = threadIdx.x; q < count; q += blockDim.x) s += src[q * stride + first];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(1024) k_assemble(Geom g, const double* __restrict__ y,
                                                   Slots s, int nstrips, int deriv,
                                                   const ThetaConsts* __restrict__ tc,
                                                   const int* __restrict__ status,
                                                   EvalOut* __restrict__ out) {
    __shared__ double red[1024];
    __shared__ double sq[1024];
    // y^T y (padding entries of y are zero)
    double a = 0.0;
    for (long long q = threadIdx.x; q < g.npad; q += blockDim.x) a = fma(y[q], y[q], a);
    sq[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sq[threadIdx.x] += sq[threadIdx.x + w];
        __syncthreads();
    }
    const double quad = sq[0];
    const double logdet = 2.0 * block_sum(s.logdet, g.T, 1, 0, red);
    const double n = (double)g.n;
    const double s2 = tc->sigma2;
    double qa = 0, qn = 0, ta = 0, tn = 0, faa = 0, fan = 0, fnn = 0;
    if (deriv) {
        const long long tiles = num_tiles(g.T);
        qa = block_sum(s.qform, tiles, 2, 0, red);
        qn = block_sum(s.qform, tiles, 2, 1, red);
        const long long nd = (long long)g.T * nstrips, no = tiles * nstrips;
        ta = block_sum(s.diag, nd, 5, 0, red);
        tn = block_sum(s.diag, nd, 5, 1, red);
        faa = block_sum(s.diag, nd, 5, 2, red) + 2.0 * block_sum(s.offd, no, 3, 0, red);
        fan = block_sum(s.diag, nd, 5, 3, red) + 2.0 * block_sum(s.offd, no, 3, 1, red);
        fnn = block_sum(s.diag, nd, 5, 4, red) + 2.0 * block_sum(s.offd, no, 3, 2, red);
    }
    if (threadIdx.x == 0) {
        out->logdet = logdet;
        out->quad = quad;
        out->loglik = -0.5 * n * 1.83787706640934548356 - 0.5 * logdet - 0.5 * quad;   // log(2 pi)
        out->status = *status;
        if (deriv) {
            out->q_alpha = qa; out->q_nu = qn; out->t_alpha = ta; out->t_nu = tn;
            out->f_aa = faa; out->f_an = fan; out->f_nn = fnn;
            // Eq. 2 with Step 2's closed form for sigma^2
            out->score[0] = (quad - n) / (2.0 * s2);
            out->score[1] = -0.5 * ta + 0.5 * qa;
            out->score[2] = -0.5 * tn + 0.5 * qn;
            // Eq. 3: I_11 = n / (2 sigma^4), I_1j = tr(Sigma^-1 Sigma_j) / (2 sigma^2),
            // I_ij = <B_i, B_j> / 2 for i, j in {alpha, nu}
            double* F = out->fisher;
            F[0] = n / (2.0 * s2 * s2);
            F[1] = F[3] = ta / (2.0 * s2);
            F[2] = F[6] = tn / (2.0 * s2);
            F[4] = 0.5 * faa;
            F[5] = F[7] = 0.5 * fan;
            F[8] = 0.5 * fnn;
        }
    }
}

int launch_assemble(Launcher& L, const Geom& g, const double* y, const Slots& s, bool deriv,
                    const ThetaConsts* tc, const int* status, EvalOut* out) {
    L.begin("assemble");
    k_assemble<<<1, 1024, 0, L.stream>>>(g, y, s, strips_per_tile(g.nb), deriv ? 1 : 0, tc, status, out);
    L.count();
    return L.end(0.0, 0.0);
}

}  // namespace fbt
