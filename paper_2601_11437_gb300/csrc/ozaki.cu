// FP64-accurate tile updates on the BF16 tensor cores (tcgen05), by error-free slicing.
//
// A tile update C -= op(A) op(B) with K = nb = 128 is computed as follows (the splitting scheme
// of Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 2012, carried out on tensor cores):
//  1. Slicing.  Every row r of an operand (the dimension that survives into C) is scaled by
//     s_r = 2^E_r with |x| < s_r for all its entries; the scaled magnitude, as the integer
//     F = floor(|x| 2^(55 - E_r)) < 2^55, is written in S = 7 balanced 8-bit digits,
//     F = sum_p d_p 2^(48 - 8p) with |d_p| <= 128, and the sign of x is applied to every digit:
//     x = s_r sum_p d_p 2^(-8(p+1) + 1) up to the truncation below 2^-55 s_r.  Digits are exact
//     in BF16 (at most 8 significant bits); the cut is exact integer arithmetic on the FP64 bits.
//  2. Products.  For digit planes A_p, B_q the product A_p B_q^T over K = 128 is a sum of
//     integers bounded by 128 * 128^2 = 2^21, so FP32 accumulation in TMEM is exact; all products
//     of one "weight" g = p + q (at most 7 of them) share one accumulator and stay exact
//     (7 * 2^21 < 2^24).  The 28 products with g <= 6 are kept; the dropped ones are below
//     2^-55 relative per element product, i.e. at FP64 rounding of the K-term dot product.
//  3. Recombination.  The 7 exact group sums are combined in 64-bit fixed point, converted to
//     FP64 (one rounding), scaled by s_r s_c and subtracted from the FP64 C.
// The MMA is tcgen05.mma kind::f16 (BF16 in, FP32 out), M = 128, N = 64 .. 256, K = 16,
// operands in shared memory (canonical K-major core-matrix layout, no swizzle) filled by bulk
// copies (cp.async.bulk, 1-D) from a pre-sliced panel buffer; accumulators live in tensor memory.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include "fbt_kernels.cuh"
#include "fbt_fx.h"

namespace fbt {

constexpr int OZ_S = 7;                      // digit planes per operand
constexpr int OZ_G = 7;                      // accumulated weights g = 0..6
constexpr int OZ_N = 64;                     // output columns per task (TMEM: 7 groups x 64 columns)
constexpr int OZ_TMEM_COLS = 512;            // allocation (a power of two >= 7 x 64)
constexpr int OZ_KC = 16;                    // K per pipeline stage (one MMA K-step)
constexpr int OZ_NKC = 128 / OZ_KC;          // stages per K = 128
constexpr int OZ_CHUNK = 128 * OZ_KC * 2;    // bytes of one plane chunk: 128 rows x 16 K bf16
constexpr int OZ_PLANE = OZ_NKC * OZ_CHUNK;  // 32 KB: one plane of a 128 x 128 tile
constexpr size_t OZ_TILE_BYTES = (size_t)OZ_S * OZ_PLANE;   // 224 KB of digits per tile
constexpr int OZ_STAGE_A = OZ_S * OZ_CHUNK;                  // 28 KB
constexpr int OZ_STAGE_B = OZ_S * (OZ_N * OZ_KC * 2);        // 14 KB
constexpr int OZ_STAGES = 4;
constexpr int OZ_SMEM = OZ_STAGES * (OZ_STAGE_A + OZ_STAGE_B) + 1024;   // 169 KB
constexpr long long OZ_SPIN_LIMIT = 1ll << 26;               // bounded mbarrier waits (default)
// After a wait has run out, the roles wait (with this budget) for the bulk copies and MMAs they
// already issued before the CTA frees its tensor memory and exits.
constexpr long long OZ_DRAIN_LIMIT = 1ll << 26;

size_t ozaki_tile_bytes() { return OZ_TILE_BYTES + 128 * sizeof(double); }   // digits + row exponents

// byte offset of digit (row, k) of plane p inside a sliced tile: K chunk k/16 (all 7 planes of a
// chunk are contiguous, so one bulk copy fetches an A stage), plane p, then the canonical K-major
// core-matrix layout of a 128 x 16 block (LBO = 128 B, SBO = 256 B)
__host__ __device__ inline uint32_t oz_off(int p, int row, int k) {
    return (uint32_t)((k >> 4) * (OZ_S * OZ_CHUNK) + p * OZ_CHUNK + (row & 7) * 16 + (row >> 3) * 256 +
                      ((k >> 3) & 1) * 128 + (k & 7) * 2);
}

// ------------------------------------------------------------------------------------------
// slicing: 4 CTAs per tile (32 operand rows each), thread t handles (row, 8-wide k group) pairs
//   ROWS = true : operand rows = tile rows, K = tile columns  (A = X, or B = X in C -= A X^T)
//   ROWS = false: operand rows = tile columns, K = tile rows  (B = X in C -= A X)
// ------------------------------------------------------------------------------------------
template <bool ROWS>
__global__ void __launch_bounds__(256) k_ozaki_slice(int nb, SliceJob job0, unsigned char* __restrict__ dst0,
                                                     SliceJob job1, unsigned char* __restrict__ dst1, int n0) {
    // 4 CTAs per tile, 32 operand rows each; the digits are taken from the FP64 bit fields:
    // F = floor(|x| 2^(55 - E_r)) < 2^55 (exact), cut into 8-bit chunks from the least
    // significant up; a chunk of 128 or more becomes chunk - 256 with a carry into the next, so
    // every digit lies in [-128, 127] (the top one in [0, 128], as F < 2^55); then the sign of x.
    __shared__ int s_exp[32];
    __shared__ unsigned long long s_part[8][32];
    // tiles [0, n0) of the launch come from job0, the rest from job1 (two matrices in one launch)
    const bool second = (int)(blockIdx.x >> 2) >= n0;
    const SliceJob& job = second ? job1 : job0;
    unsigned char* __restrict__ dst = second ? dst1 : dst0;
    const int t = (int)(blockIdx.x >> 2) - (second ? n0 : 0), rq = (blockIdx.x & 3) * 32;
    const double* X = job.tile_ptr(t, nb);
    unsigned char* out = dst + (size_t)t * (OZ_TILE_BYTES + 128 * sizeof(double));
    int* exp_out = (int*)(out + OZ_TILE_BYTES);
    {   // row maxima: the 8 warps take 16 entries of each of the 32 rows
        const int rl = threadIdx.x & 31, kq = threadIdx.x >> 5, r = rq + rl;
        unsigned long long mbits = 0;
#pragma unroll
        for (int k = kq * 16; k < kq * 16 + 16; ++k) {
            const double v = ROWS ? X[r + k * 128] : X[k + r * 128];
            const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
            mbits = b > mbits ? b : mbits;          // |x| order = integer order of the bits
        }
        s_part[kq][rl] = mbits;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int r = rq + threadIdx.x;
        unsigned long long mbits = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) mbits = s_part[q][threadIdx.x] > mbits ? s_part[q][threadIdx.x] : mbits;
        const int E = (int)(mbits >> 52);
        const int e = E == 0 ? 0 : E - 1022;        // 2^(e-1) <= max |x| < 2^e (zero row: e = 0)
        s_exp[threadIdx.x] = e;
        exp_out[r] = e;
        // largest exponent of a non-zero row among these 32 rows (-10000: all rows zero), for the
        // per-task precision choice of the mixed path
        int em = E == 0 ? -10000 : e;
        for (int off = 16; off > 0; off >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, off));
        if (threadIdx.x == 0) exp_out[128 + (rq >> 5)] = em;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < 32 * 16; w += blockDim.x) {
        const int rl = w & 31, r = rq + rl, k8 = (w >> 5) * 8;
        const int e = s_exp[rl];
        uint32_t packed[OZ_S][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const double v = ROWS ? X[r + (k8 + j) * 128] : X[(k8 + j) + r * 128];
            const unsigned long long b = (unsigned long long)__double_as_longlong(v);
            const int E = (int)((b >> 52) & 0x7FF);
            const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
            const int sh = 1020 + e - E;            // F = M * 2^(E - 1075 - e + 55)
            unsigned long long F = 0;
            if (E != 0) F = sh < 0 ? (M << (-sh)) : (sh < 64 ? (M >> sh) : 0ull);
            const bool neg = (b >> 63) != 0;
            int carry = 0;
#pragma unroll
            for (int p = OZ_S - 1; p >= 0; --p) {
                int d = (int)((F >> (48 - 8 * p)) & 255ull) + carry;
                carry = (p > 0 && d >= 128) ? 1 : 0;
                d -= carry * 256;
                d = neg ? -d : d;
                const uint32_t h = __float_as_uint((float)d) >> 16;    // exact: |d| <= 128
                if (j & 1) packed[p][j >> 1] |= h << 16;
                else packed[p][j >> 1] = h;
            }
        }
#pragma unroll
        for (int p = 0; p < OZ_S; ++p) {
            uint4 v = make_uint4(packed[p][0], packed[p][1], packed[p][2], packed[p][3]);
            *(uint4*)(out + oz_off(p, r, k8)) = v;
        }
    }
}

// ------------------------------------------------------------------------------------------
// PTX helpers
// ------------------------------------------------------------------------------------------
__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline uint64_t oz_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;         // LBO: next 8-element K group
    d |= (uint64_t)(256 >> 4) << 32;         // SBO: next 8-row group
    d |= (uint64_t)1 << 46;                  // descriptor version
    return d;
}

__device__ inline void mbar_init(uint64_t* b, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ inline bool mbar_wait(uint64_t* b, uint32_t parity, long long limit) {
    uint32_t done = 0;
    for (long long it = 0; it < limit; ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(smem_u32(b)), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}
__device__ inline void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ inline void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ inline void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}
__device__ inline void tmem_ld8(uint32_t taddr, float v[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------------------------------
// the tile-update kernel and its epilogue helpers
// ------------------------------------------------------------------------------------------
__device__ inline void tmem_ld8x(uint32_t taddr, uint32_t r[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// Persistent (one CTA per SM), warp-specialised: warp 0 issues the MMAs, warp 1 streams digit
// stages with bulk copies (4-stage ring), warps 2..17 drain the TMEM accumulators (warp w reads
// TMEM lanes 32 (w % 4) .. +31, columns 16 ((w - 2) / 4) .. +15).  The accumulators are released
// once they are in registers (the FP64-accurate kernel: after the last TMEM load; the mixed
// kernel: after the fold into 64-bit fixed point), so the next task's MMAs run while the epilogue
// converts and updates C; the drain is on the critical path between tasks, hence 16 epilogue
// warps.  N = 64 per task because TMEM holds the 7 groups x 64 columns.  The task period is the
// MMAs (fed by a 42 KB operand stage per K = 16 from L2) plus the drain up to the hand-back of
// TMEM; the rest of the epilogue (fold, int64-to-FP64 conversion with integer instructions, one
// FP64 subtraction per output, 64 KB of C read and written) fits inside the next task's MMAs.
constexpr int OZ_EPI_WARPS = 16;                        // 4 per TMEM lane quarter
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;
constexpr int OZ_EPI_COLS = OZ_N * 4 / OZ_EPI_WARPS;   // accumulator columns per epilogue warp

// Digit planes used for a task: 7 (FP64-accurate); in the mixed path 3, 1 or 0 (skipped) when
// the operand tiles' largest entries, 2^ea over the task's 128 A rows and 2^eb over its 64 B rows
// (output columns c0 .. c0 + 63), make the product small against the thresholds.
__device__ inline int task_planes(const OzGemmJob& job, const unsigned char* sa, const unsigned char* sb, int c0) {
    if (!job.mixed) return OZ_S;
    const int* ha = (const int*)(sa + OZ_TILE_BYTES) + 128;
    const int* hb = (const int*)(sb + OZ_TILE_BYTES) + 128 + (c0 >> 5);
    const int ea = max(max(ha[0], ha[1]), max(ha[2], ha[3]));
    const int eb = max(hb[0], hb[1]);
    const int e = ea + eb;
    return e >= job.e_fp64 ? OZ_S : (e >= job.e_fp32 ? 3 : (e >= job.e_skip ? 1 : 0));
}

// The MMAs of one K stage for NP digit planes: the products A_p B_q with p + q < NP, stacked
// as (p, q0 .. q0 + 3) into one MMA of N = 64 (q1 - q0 + 1) (see the MMA warp below).
template <int NP>
__device__ inline void issue_stage(uint32_t tmem, uint32_t a0, uint32_t b0, int kc, uint32_t idesc0) {
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int q0 = 0; p + q0 < NP; q0 += 4) {
            const int nq = min(4, NP - p - q0);
            const uint32_t acc = (kc > 0 || p > 0) ? 1u : 0u;
            const uint32_t idesc = idesc0 | ((uint32_t)(nq * OZ_N >> 3) << 17);
            mma_bf16(tmem + (p + q0) * OZ_N, oz_desc(a0 + p * OZ_CHUNK), oz_desc(b0 + q0 * (OZ_N * OZ_KC * 2)),
                     idesc, acc);
        }
}

// Up to four jobs run as one task list (their targets must not overlap): task t belongs to the
// first job whose cumulative end exceeds t.
struct OzJobList {
    OzGemmJob job[4];
    long long end[4];
    long long spin;                // iteration limit of every mbarrier wait
    const long long* list;         // mixed path: classified tasks, (task << 3) | tier
    const unsigned* count;         //   and their number (null: every task, all planes)
    int n;
    __device__ const OzGemmJob& pick(long long t, long long& local) const {
        int j = 0;
        while (j + 1 < n && t >= end[j]) ++j;
        local = t - (j ? end[j - 1] : 0);
        return job[j];
    }
};

// Mixed path: the classification that precedes every launch.  One thread per task takes its
// tier from the operand tiles' largest entries (task_planes) and appends every task that is
// not skipped, or that must write zeros, to the list as (task << 3) | tier, tier 0..3 for 0, 1,
// 3 and 7 planes; the tile-update kernel then walks the list, so a skipped task costs nothing
// there.  The list's order varies from run to run, the results do not: the tasks of one launch
// write disjoint targets, each the same values whichever CTA computes it.
__device__ inline int tier_planes(int tier) { return tier == 0 ? 0 : (tier == 1 ? 1 : (tier == 2 ? 3 : OZ_S)); }

__global__ void __launch_bounds__(256) k_mixed_classify(OzJobList jobs, long long ntasks, long long* __restrict__ list,
                                                        unsigned* __restrict__ count) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int tier = -1;
    bool keep = false;
    if (t < ntasks) {
        const unsigned char *sa, *sb;
        double* C;
        int c0;
        double mult;
        long long lt;
        const OzGemmJob& job = jobs.pick(t, lt);
        job.task(lt, sa, sb, C, c0, mult);
        const int np = task_planes(job, sa, sb, c0);
        tier = np == 0 ? 0 : (np == 1 ? 1 : (np == 3 ? 2 : 3));
        keep = np != 0 || job.assign != 0;
    }
    unsigned long long* tiers = jobs.job[0].counts;
    if (tiers) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const unsigned m = __ballot_sync(0xffffffffu, tier == q);
            if (lane == 0 && m) atomicAdd(&tiers[q], (unsigned long long)__popc(m));
        }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, keep);
    if (mask) {
        const int leader = __ffs(mask) - 1;
        unsigned base = 0;
        if (lane == leader) base = atomicAdd(count, (unsigned)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (keep) list[base + __popc(mask & ((1u << lane) - 1u))] = (t << 3) | tier;
    }
}

// MIXED: the job list may use fewer digit planes per task (compiled separately, so that the
// FP64-accurate path carries no plane-count logic)
// Work item i of a launch: task i with all planes, or entry i of the mixed path's classified
// list (its task and its plane count).  Without MIXED the plane count is a compile-time constant.
template <bool MIXED>
__device__ inline long long work_item(const OzJobList& jobs, long long i, int& np) {
    if (!MIXED || !jobs.list) { np = OZ_S; return i; }
    const long long e = jobs.list[i];
    np = tier_planes((int)(e & 7));
    return e >> 3;
}

template <bool MIXED>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_ozaki_gemm(OzJobList jobs, long long ntasks, int* status) {
    extern __shared__ __align__(1024) unsigned char oz_smem[];
    unsigned char* stA = oz_smem;                                    // [4][28 KB]
    unsigned char* stB = oz_smem + OZ_STAGES * OZ_STAGE_A;           // [4][14 KB]
    uint64_t* bars = (uint64_t*)(oz_smem + OZ_STAGES * (OZ_STAGE_A + OZ_STAGE_B));
    uint64_t* full = bars;                   // [4] stage loaded
    uint64_t* empty = bars + OZ_STAGES;      // [4] stage consumed by the MMAs
    uint64_t* tfull = bars + 2 * OZ_STAGES;  // accumulators complete
    uint64_t* tempty = tfull + 1;            // accumulators drained into registers
    uint32_t* tmem_slot = (uint32_t*)(tempty + 1);
    int* fail = (int*)(tempty + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(OZ_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < OZ_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(tfull, 1);
        mbar_init(tempty, OZ_EPI_WARPS);
        *fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // work items: every task, or the mixed path's classified list (written by the preceding
    // launch on this stream)
    const long long nwork = (MIXED && jobs.list) ? (long long)*jobs.count : ntasks;

    if (warp == 1) {
        if (lane == 0) {
            // producer: stages (task, kc) in order through the ring, stage s = it % OZ_STAGES
            long long it = 0;                        // stage iterations issued so far
            for (long long i = blockIdx.x; i < nwork && !*(volatile int*)fail; i += gridDim.x) {
                const unsigned char *sa, *sb;
                double* C;
                int c0;
                double mult;
                long long lt;
                int np;
                const long long t = work_item<MIXED>(jobs, i, np);
                const OzGemmJob& job = jobs.pick(t, lt);
                job.task(lt, sa, sb, C, c0, mult);
                if (MIXED && np == 0) continue;          // writes zeros only: no stages, no MMAs
                // the task's 64 columns of C (64 KB, contiguous in the column-major tile) into
                // L2 now, so that the epilogue's loads of them, a task later, do not wait on DRAM
                if (!job.assign)
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(C + (size_t)c0 * 128),
                                 "r"(128u * 64u * 8u) : "memory");
                for (int kc = 0; kc < OZ_NKC; ++kc, ++it) {
                    const int s = (int)(it % OZ_STAGES);
                    if (it >= OZ_STAGES && !mbar_wait(&empty[s], (uint32_t)(((it / OZ_STAGES) - 1) & 1), jobs.spin)) {
                        atomicOr(fail, 1);
                        break;
                    }
                    mbar_expect_tx(&full[s], (uint32_t)np * (OZ_CHUNK + OZ_N * OZ_KC * 2));
                    const size_t chunk = (size_t)kc * OZ_S * OZ_CHUNK;
                    bulk_g2s(stA + s * OZ_STAGE_A, sa + chunk, (uint32_t)np * OZ_CHUNK, &full[s]);
                    for (int p = 0; p < np; ++p)
                        bulk_g2s(stB + s * OZ_STAGE_B + p * (OZ_N * OZ_KC * 2),
                                 sb + chunk + p * OZ_CHUNK + (c0 >> 3) * 256, OZ_N * OZ_KC * 2, &full[s]);
                }
            }
            if (*(volatile int*)fail) {
                // a wait ran out somewhere: let the copies already issued land before the CTA
                // exits.  Stages are issued round robin, so the last iteration issued on stage q
                // is it - 1 - ((it - 1 - q) mod OZ_STAGES); no later phase of it was started, so
                // that phase's parity is unambiguous.
#pragma unroll
                for (int q = 0; q < OZ_STAGES; ++q) {
                    if (it <= q) continue;
                    const long long last = it - 1 - ((it - 1 - q) % OZ_STAGES);
                    if (!mbar_wait(&full[q], (uint32_t)((last / OZ_STAGES) & 1), OZ_DRAIN_LIMIT)) atomicOr(fail, 16);
                }
            }
        }
    } else if (warp == 0) {
        if (lane == 0) {
            // MMA issuer: per stage the 28 digit products with p + q <= 6 into group g = p + q.
            // The groups occupy consecutive 64-column ranges of TMEM and the B planes consecutive
            // 64-row blocks of the stage, so the products (p, q0 .. q1) are one MMA with
            // N = 64 (q1 - q0 + 1) <= 256 into the columns of groups p + q0 .. p + q1: 10 MMAs
            // per stage instead of 28, and A_p is read from shared memory once per MMA.
            const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 4) << 24);
            long long it = 0, nt = 0, commits = 0;
            for (long long i = blockIdx.x; i < nwork; i += gridDim.x, ++nt) {
                int np;
                work_item<MIXED>(jobs, i, np);
                if (MIXED && np == 0) { --nt; continue; }   // zero-writing task: not counted in nt
                if (nt > 0 && !mbar_wait(tempty, (uint32_t)((nt - 1) & 1), jobs.spin)) { atomicOr(fail, 4); break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                bool bad = false;
                for (int kc = 0; kc < OZ_NKC; ++kc, ++it) {
                    const int s = (int)(it % OZ_STAGES);
                    if (!mbar_wait(&full[s], (uint32_t)((it / OZ_STAGES) & 1), jobs.spin)) { atomicOr(fail, 2); bad = true; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(stA + s * OZ_STAGE_A), b0 = smem_u32(stB + s * OZ_STAGE_B);
                    if (!MIXED || np == OZ_S) issue_stage<OZ_S>(tmem, a0, b0, kc, idesc0);
                    else if (np == 3) issue_stage<3>(tmem, a0, b0, kc, idesc0);
                    else issue_stage<1>(tmem, a0, b0, kc, idesc0);
                    mma_commit(&empty[s]);
                }
                mma_commit(tfull);
                ++commits;
                if (bad) break;
            }
            if (*(volatile int*)fail && commits > 0) {
                // the last commit tracks every MMA this thread issued: wait for it before the
                // tensor memory is freed
                if (!mbar_wait(tfull, (uint32_t)((commits - 1) & 1), OZ_DRAIN_LIMIT)) atomicOr(fail, 32);
            }
        }
    } else {
        // epilogue warps 2..: rows of TMEM lane quarter w % 4, columns OZ_EPI_COLS ((w - 2) / 4) ..
        const int quarter = warp & 3;
        const int r = quarter * 32 + lane;
        const int chalf = ((warp - 2) >> 2) * OZ_EPI_COLS;
        long long nt = 0;
        for (long long i = blockIdx.x; i < nwork; i += gridDim.x, ++nt) {
            const unsigned char *sa, *sb;
            double* C;
            int c0;
            double mult;
            long long lt;
            int np;
            const long long t = work_item<MIXED>(jobs, i, np);
            const OzGemmJob& job = jobs.pick(t, lt);
            job.task(lt, sa, sb, C, c0, mult);
            if (MIXED && np == 0) {
                // an assigning task whose entries are all below the tolerance writes zeros
                --nt;
                if (job.assign) {
                    double* __restrict__ Cz = C + r + (long long)(c0 + chalf) * 128;
#pragma unroll
                    for (int h = 0; h < OZ_EPI_COLS; ++h) Cz[(long long)h * 128] = 0.0;
                }
                continue;
            }
            // one decision per warp: the TMEM loads below are warp-collective
            const bool ready = mbar_wait(tfull, (uint32_t)(nt & 1), jobs.spin) && !*(volatile int*)fail;
            if (!__all_sync(0xffffffffu, ready)) { atomicOr(fail, 8); break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            long long fx[OZ_EPI_COLS];
#pragma unroll
            for (int cb = 0; cb < OZ_EPI_COLS; cb += 8) {
                uint32_t v[OZ_G][8];
                // groups this task did not accumulate hold an earlier task's data: they are not
                // read and count as 0 (np is the same for every thread of the warp)
#pragma unroll
                for (int g = 0; g < OZ_G; ++g) {
                    if (g < np) {
                        tmem_ld8x(tmem + ((uint32_t)(quarter * 32) << 16) + g * OZ_N + chalf + cb, v[g]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j) v[g][j] = 0u;
                    }
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (!MIXED && cb + 8 == OZ_EPI_COLS) {
                    // the last accumulator columns are in registers: hand TMEM back to the MMA
                    // warp before folding them, so the fold leaves the MMAs' critical path (the
                    // mixed kernel, short of registers for it, releases after the fold)
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tempty)) : "memory");
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    // exact group sums -> fixed point with unit 2^-46 of s_r s_c.  Group g (at
                    // most g + 1 products of digits <= 2^7 over K = 128) is below (g + 1) 2^21 and
                    // carries weight 2^(32 - 8 g) units.  Group 0 (<= 2^21) converts exactly by
                    // adding 1.5 2^23 in FP32, groups 1..4 with F2I.  Groups 5, 6 only enter below
                    // the unit: t56 = v_5 + v_6 / 256 in one FMA (|t56| < 2^24, error <= 1/2 ulp),
                    // then t56 / 256 + 1.5 2^23 in another rounds their sum to the unit, to
                    // nearest: at most 1/2 + 2^-9 unit off, without bias.  P = v_g 2^8 + v_(g+1)
                    // for g = 0, 2 is exact in 32-bit integers (|P23| <= 3 2^29 + 2^23 < 2^31).
                    const int iv0 = __float_as_int(__uint_as_float(v[0][j]) + 12582912.0f) - 0x4B400000;
                    const int iv1 = __float2int_rn(__uint_as_float(v[1][j]));
                    const int iv2 = __float2int_rn(__uint_as_float(v[2][j]));
                    const int iv3 = __float2int_rn(__uint_as_float(v[3][j]));
                    const int iv4 = __float2int_rn(__uint_as_float(v[4][j]));
                    const float t56 = fmaf(__uint_as_float(v[6][j]), 0.00390625f, __uint_as_float(v[5][j]));
                    const int r56 = __float_as_int(fmaf(t56, 0.00390625f, 12582912.0f)) - 0x4B400000;
                    const int p01 = iv0 * 256 + iv1, p23 = iv2 * 256 + iv3;
                    fx[cb + j] = (long long)p01 * (1ll << 24) + (long long)p23 * (1ll << 8) + (iv4 + r56);
                }
            }
            if (MIXED) {
                // accumulators are in registers: hand TMEM back to the MMA warp
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tempty)) : "memory");
            }
            const int* __restrict__ exp_a = (const int*)(sa + OZ_TILE_BYTES);
            const int* __restrict__ exp_b = (const int*)(sb + OZ_TILE_BYTES);
            // |mult| is a power of two: its exponent is read from the bits (ilogb costs a dozen
            // instructions on the narrow FP64 pipe, per thread and task)
            const int er = exp_a[r] - 46 + (int)((__double_as_longlong(mult) >> 52) & 0x7FF) - 1023;
            const bool assign = job.assign != 0;
            const bool negm = mult < 0.0;
            double* __restrict__ Cr = C + r + (long long)(c0 + chalf) * 128;
            // C values are loaded 8 at a time before any is stored, so their latencies overlap
#pragma unroll
            for (int h = 0; h < OZ_EPI_COLS; h += 8) {
                double cv[8];
                int eb[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    cv[j] = assign ? 0.0 : Cr[(long long)(h + j) * 128];
                    eb[j] = exp_b[c0 + chalf + h + j];
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    // converted with integer instructions: the FP64 pipe, two lanes per clock
                    // per SM, is left the subtraction alone
                    const double y = fx_to_double_int(fx[h + j], er + eb[j], negm);
                    Cr[(long long)(h + j) * 128] = cv[j] - y;
                }
            }
        }
    }
    __syncthreads();
    if (*fail && tid == 0) atomicOr(status, ST_TIMEOUT);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS));
    }
}

int launch_ozaki_slice(Launcher& L, const Geom& g, const SliceJob& job, int ntiles, bool rows,
                       unsigned char* dst, const char* family) {
    if (ntiles <= 0) return 0;
    L.begin(family);
    if (rows) k_ozaki_slice<true><<<ntiles * 4, 256, 0, L.stream>>>(g.nb, job, dst, job, dst, ntiles);
    else k_ozaki_slice<false><<<ntiles * 4, 256, 0, L.stream>>>(g.nb, job, dst, job, dst, ntiles);
    L.count();
    return L.end(0.0, (double)ntiles * (128.0 * 128 * 8 + OZ_TILE_BYTES));
}

int launch_ozaki_slice2(Launcher& L, const Geom& g, const SliceJob& job0, unsigned char* dst0,
                        const SliceJob& job1, unsigned char* dst1, int ntiles, bool rows) {
    if (ntiles <= 0) return 0;
    L.begin("ozaki_slice");
    if (rows) k_ozaki_slice<true><<<ntiles * 8, 256, 0, L.stream>>>(g.nb, job0, dst0, job1, dst1, ntiles);
    else k_ozaki_slice<false><<<ntiles * 8, 256, 0, L.stream>>>(g.nb, job0, dst0, job1, dst1, ntiles);
    L.count();
    return L.end(0.0, 2.0 * ntiles * (128.0 * 128 * 8 + OZ_TILE_BYTES));
}

int launch_ozaki_gemm(Launcher& L, const OzGemmJob& job, long long ctas, double flops, int* status,
                      const char* family) {
    return launch_ozaki_gemm_multi(L, &job, &ctas, 1, flops, status, family);
}

int launch_ozaki_gemm_multi(Launcher& L, const OzGemmJob* job, const long long* tasks, int njobs, double flops,
                            int* status, const char* family, int reserve_sms) {
    if (njobs < 1 || njobs > 4) return cudaErrorInvalidValue;
    OzJobList jl{};
    long long ctas = 0;
    for (int j = 0; j < njobs; ++j) {
        jl.job[j] = job[j];
        ctas += tasks[j];
        jl.end[j] = ctas;
    }
    jl.n = njobs;
    jl.spin = L.spin > 0 ? L.spin : OZ_SPIN_LIMIT;
    if (ctas <= 0) return 0;
    static const int sms = [] {          // initialised once, also when several host threads launch
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 152;
    }();
    bool mixed = false;
    for (int j = 0; j < njobs; ++j) mixed = mixed || job[j].mixed != 0;
    ensure_smem((const void*)k_ozaki_gemm<false>, OZ_SMEM);
    ensure_smem((const void*)k_ozaki_gemm<true>, OZ_SMEM);
    // persistent: one CTA per SM, reserve_sms of them left to concurrent work
    const long long avail = (long long)sms - reserve_sms > 1 ? (long long)sms - reserve_sms : 1;
    const long long grid = ctas < avail ? ctas : avail;
    L.begin(family);
    jl.list = nullptr;
    jl.count = nullptr;
    if (mixed && !(job[0].task_list && job[0].task_count && ctas <= job[0].task_cap))
        return cudaErrorInvalidValue;          // the mixed path needs room for its task list
    if (mixed) {
        // classify the tasks, then walk the list of those not skipped (persistent grid: the
        // list's length is only known on the device)
        if (cudaMemsetAsync(job[0].task_count, 0, sizeof(unsigned), L.stream) != cudaSuccess) return cudaGetLastError();
        k_mixed_classify<<<(unsigned)((ctas + 255) / 256), 256, 0, L.stream>>>(jl, ctas, job[0].task_list,
                                                                               job[0].task_count);
        L.count();
        jl.list = job[0].task_list;
        jl.count = job[0].task_count;
        k_ozaki_gemm<true><<<(unsigned)avail, OZ_THREADS, OZ_SMEM, L.stream>>>(jl, ctas, status);
    } else {
        k_ozaki_gemm<false><<<(unsigned)grid, OZ_THREADS, OZ_SMEM, L.stream>>>(jl, ctas, status);
    }
    L.count();
    return L.end(flops, 0.0);
}

}  // namespace fbt
