// Mixed-precision evaluation of the dual of the entropy closure [Sec. 3.1, Eq. entropyOCP].
//
// The Hessian <m m^T e> of the dual needs the moments V_c = sum_q w_q e_q m~_c(q) of the ansatz
// against the degree-2N basis (H_ab = sum_c G_abc V_c, Gaunt coefficients G). Its first n
// moments are the gradient's <m e> and stay in FP64; the remaining n2 - n moments enter only the
// Hessian and are a batched dense contraction
//     V_hi[cells x (n2-n)] = E[cells x Q'] . (w M_hi)[Q' x (n2-n)],   E = exp(alpha.m)
// that runs on the 5th-generation tensor cores: tcgen05.mma with TF32 (kind::tf32) or BF16
// (kind::f16) operands and FP32 accumulation in tensor memory (the quadrature weights are folded
// into the basis table). Exponents, exp and the gradient moments run in FP64 in the
// sum-factorised form of sweep.cuh (pairs of mirrored azimuths, coefficients per ring); the
// objective, the Cholesky factorisation and the line search stay in FP64 (newton_post).
//
// One CTA (256 threads) owns a tile of 128 listed cells (the MMA's M = 128 rows, row = cell).
// The quadrature runs in chunks of 16 pairs (32 points): every thread evaluates 8 pairs of one
// row in FP64, accumulates its FP64 gradient moments, and stores E rounded to TF32/BF16 into
// shared memory in the canonical K-major core-matrix layout (8 rows x 16 bytes per core matrix,
// no swizzle); the threads also stage the matching 32 columns of the weighted M_hi. One elected
// thread issues the MMAs of the chunk and commits them to an mbarrier; chunks alternate between
// two buffers so that the next chunk's FP64 work overlaps the tensor-core work of the previous
// one. Every wait is bounded: on expiry the kernel records KITRT_ETIMEOUT, drains what it issued
// (bounded) and frees its tensor memory.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include "kitrt_internal.cuh"
#include "kexp.cuh"
#include "newton_common.cuh"
#include "async_copy.cuh"
#include "sweep.cuh"

namespace {

using namespace kitrt_dev;
using namespace kitrt_async;

constexpr int kTileM = 128;   // cells per tile (MMA M)
constexpr int kChunk = 32;    // quadrature points per chunk (MMA K per chunk)
constexpr int kThreads = 256;
constexpr int kWarpsM = kThreads / 32;
// ----- tcgen05 wrappers (mbarrier helpers: async_copy.cuh) -------------------------------------
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

template <bool BF16>
__device__ __forceinline__ void mma_issue(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    if (BF16) {
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "setp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
            "}\n" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "setp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
            "}\n" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, K-major, no swizzle: start address, leading-dimension byte
// offset (between core matrices adjacent in K), stride byte offset (between 8-row groups), and
// the descriptor version bits of the 5th-generation tensor cores.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: D FP32, A/B format (TF32 = 2 under kind::tf32, BF16 = 1 under
// kind::f16), both K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, uint32_t ab)
{
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int NN>
struct MixedDims {
    static constexpr int n = Dims<NN>::n, n2 = Dims<NN>::n2;
    static constexpr int nhi = n2 - n;
    static constexpr int NP = ((nhi + 15) / 16) * 16;          // MMA N
    static constexpr int tcols = NP <= 32 ? 32 : (NP <= 64 ? 64 : 128);
};

// Byte layout of the dynamic shared memory of the mixed kernel. Each of the two chunk buffers
// holds the operands split into a high and a low part (x = x_hi + x_lo, both representable in
// the tensor-core input format), so that E.M ~ E_hi.M_hi + E_hi.M_lo + E_lo.M_hi is accurate to
// about FP32 rounding instead of the input format's.
template <int NN, bool BF16>
struct MixedSmem {
    static constexpr int esz = BF16 ? 2 : 4;
    static constexpr int T = 16 / esz;                           // elements per core-matrix row
    static constexpr int LBO = 128;                              // K-adjacent core matrices
    static constexpr int SBO = (kChunk / T) * 128;               // 8-row groups
    static constexpr int A_bytes = kTileM * kChunk * esz;
    static constexpr int B_bytes = MixedDims<NN>::NP * kChunk * esz;
    static constexpr int buf_bytes = 2 * A_bytes + 2 * B_bytes;  // A_hi, A_lo, B_hi, B_lo
    static __host__ __device__ constexpr int off_Ahi(int b) { return b * buf_bytes; }
    static __host__ __device__ constexpr int off_Alo(int b) { return b * buf_bytes + A_bytes; }
    static __host__ __device__ constexpr int off_Bhi(int b) { return b * buf_bytes + 2 * A_bytes; }
    static __host__ __device__ constexpr int off_Blo(int b) { return b * buf_bytes + 2 * A_bytes + B_bytes; }
    static constexpr int off_V = (2 * buf_bytes + 1023) / 1024 * 1024;
    static constexpr int V_bytes = kTileM * Dims<NN>::n * 8;      // second half's gradient sums
    static constexpr int off_bar = off_V + V_bytes;
    static constexpr int total = off_bar + 64;
    static constexpr int kmma = BF16 ? 16 : 8;                   // MMA K
    // byte offset of element (row r, k) inside an operand chunk
    static __device__ __forceinline__ int elem_off(int r, int k)
    {
        return (r >> 3) * SBO + (k / T) * LBO + (r & 7) * 16 + (k % T) * esz;
    }
};

// E rounded to the tensor-core input format, split into a high and a low part, at (row r, k) of
// the chunk's operand tiles.
template <bool BF16, typename L>
__device__ __forceinline__ void store_operand(unsigned char *Ahi, unsigned char *Alo, int r, int kk, float e)
{
    if (BF16) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(e);
        const __nv_bfloat16 lo = __float2bfloat16_rn(e - __bfloat162float(hi));
        *(__nv_bfloat16 *)(Ahi + L::elem_off(r, kk)) = hi;
        *(__nv_bfloat16 *)(Alo + L::elem_off(r, kk)) = lo;
    } else {
        uint32_t hi, lo;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(e));
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(e - __uint_as_float(hi)));
        *(uint32_t *)(Ahi + L::elem_off(r, kk)) = hi;
        *(uint32_t *)(Alo + L::elem_off(r, kk)) = lo;
    }
}

// Work item = (tile of 128 listed cells, range of quadrature chunks). When few cells are listed
// (the later sweeps of a closure), each tile's quadrature range is split over several CTAs
// (sweep_split) so that every SM gets work; each work item stores its partial moments with plain
// stores into its own column block of Vacc (entry c of list slot j, part p at
// Vacc[c vs_c + (p cnt + j) vs_s]; [n2 x vs] columns for the Newton sweeps, [C x n2] rows and one
// part for the moments of given alphas), and the Newton kernel adds the parts in order.
template <int NN, bool BF16, bool MOMENTS_ONLY>
__global__ void __launch_bounds__(kThreads, NN <= 3 ? 2 : 1)
eval_mixed_kernel(Tables T, NewtonState S, int k, const void *__restrict__ Mhi,
                  const double *__restrict__ alpha_in, double *__restrict__ Vacc, int vs_c, int vs_s,
                  int C, int target_items, float *__restrict__ psi32)
{
    using D = MixedDims<NN>;
    using L = MixedSmem<NN, BF16>;
    constexpr int n = D::n, n2 = D::n2, NP = D::NP, NA = 2 * NN + 1;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = (uint64_t *)(smem + L::off_bar);
    uint32_t *tmem_slot = (uint32_t *)(smem + L::off_bar + 16);
    int *abort_flag = (int *)(smem + L::off_bar + 24);
    double *sU = (double *)(smem + L::off_V);  // [n][128]: the second half's gradient moments
    const int tid = threadIdx.x, warp = tid >> 5;
    const int Qp = T.Qp, nchunks = Qp / kChunk;
    constexpr int TW = 4 * NN + 1;  // ptrig row width

    int cnt_in;
    const int32_t *list_in = nullptr;
    if (MOMENTS_ONLY) {
        cnt_in = C;
    } else {
        list_in = S.list[k & 1];
        cnt_in = S.cnt[k % 3];
        if (blockIdx.x == 0 && tid == 0) S.cnt[(k + 2) % 3] = 0;
    }
    const SweepSplit sp = sweep_split(cnt_in, target_items, nchunks);
    const int ks = sp.parts, cpp = sp.units_per_part;
    const int items = sp.tiles * ks;
    if ((int)blockIdx.x >= items) return;  // no work item for this CTA (uniform per CTA)

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tmem_slot, D::tcols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t idesc = instr_desc(kTileM, NP, BF16 ? 1u : 2u);
    uint32_t commits[2] = {0, 0}, waited[2] = {0, 0};
    const int r = tid & (kTileM - 1), h = tid >> 7;  // row of this thread, half of each chunk

    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int tile = item / ks, part = item % ks;
        const int c_begin = part * cpp, c_end = min(nchunks, c_begin + cpp);
        const int base = tile * kTileM;
        const int rows = min(kTileM, cnt_in - base);
        int cell = -1;
        if (r < rows) cell = MOMENTS_ONLY ? base + r : list_in[base + r];
        bool active = cell >= 0;
        if (!MOMENTS_ONLY && active && S.h64[cell]) active = false;  // done by the FP64 sweep
        double at[n], U[n], A[NA], B[NA];
#pragma unroll
        for (int a = 0; a < n; ++a) {
            U[a] = 0.0;
            at[a] = 0.0;
        }
#pragma unroll
        for (int j = 0; j < NA; ++j) A[j] = B[j] = 0.0;
        if (active) {
            if (MOMENTS_ONLY) {
#pragma unroll
                for (int a = 0; a < n; ++a) at[a] = alpha_in[(size_t)cell * n + a];
            } else {
                const int ph = S.phase[cell];
                const double lam = ph == PH_NEWTON ? S.lam[cell] : 0.0;
#pragma unroll
                for (int a = 0; a < n; ++a) {
                    const double al = S.alpha[(size_t)cell * n + a];
                    at[a] = ph == PH_NEWTON ? fma(lam, S.dir[(size_t)cell * n + a], al) : al;
                }
            }
            // the pairs take the exponent in units of ln2/2048 (kexp_scaled)
#pragma unroll
            for (int a = 0; a < n; ++a) at[a] *= 2954.639443740597;  // 2048 / ln2
        }
        int ring = -1;  // ring whose azimuthal sums B holds (uniform within a warp)
        for (int c = c_begin; c < c_end; ++c) {
            const int b = c & 1;
            unsigned char *Ahi = smem + L::off_Ahi(b), *Alo = smem + L::off_Alo(b);
            unsigned char *Bhi = smem + L::off_Bhi(b), *Blo = smem + L::off_Blo(b);
            if (commits[b] > waited[b]) {
                // the MMAs that read this buffer must have finished before it is overwritten:
                // one thread waits on the buffer's mbarrier, the CTA barrier orders the rest
                if (tid == 0 && !mbar_wait_bounded(&bar[b], waited[b] & 1)) *abort_flag = 1;
                ++waited[b];
                __syncthreads();
                if (*abort_flag) break;  // uniform: read after the barrier
            }
            tc_fence_after();
            // FP64 part: 8 pairs of this row (exponents, exp, gradient sums); E to the operand
#pragma unroll 2
            for (int i = 0; i < kChunk / 4; ++i) {
                const int pr = c * (kChunk / 2) + h * (kChunk / 4) + i;
                // padding pairs (w = 0, warp-uniform) add nothing: their operand is 0 and their
                // psi stays at the zeros written at allocation
                const bool real = pr < T.npair;
                if (real) {
                    const int rg = pr / T.P;
                    if (rg != ring) {
                        if (ring >= 0)
                            ring_flush<NN>(T.ringWP + (size_t)ring * n2, B, [&](int cc) -> double & { return U[cc]; });
                        ring_coeffs<NN>(at, T.ringP + (size_t)rg * n2, A);
                        ring = rg;
                    }
                }
                float f1 = 0.0f, f2 = 0.0f;
                if (active && real) {
                    double e1, e2;
                    pair_eval<NN, NN, true>(A, T.ptrig + (size_t)pr * TW, pr % T.P == 0, T.exptab, B, e1, e2);
                    f1 = exp_to_float(e1);
                    f2 = exp_to_float(e2);
                    // ansatz of the trial point (the last accepted trial leaves the solution's)
                    if (psi32) *(float2 *)(psi32 + (size_t)cell * Qp + 2 * pr) = make_float2(f1, f2);
                }
                const int kk = h * (kChunk / 2) + 2 * i;
                store_operand<BF16, L>(Ahi, Alo, r, kk, f1);
                store_operand<BF16, L>(Ahi, Alo, r, kk + 1, f2);
            }
            // stage the chunk of the split table (row-major [2][NP x Qp] in global: high part,
            // then low part), in 16-byte pieces
            constexpr int per16 = L::T;  // elements per 16 bytes
            constexpr int pieces = NP * (kChunk / per16);
            for (int p = tid; p < 2 * pieces; p += kThreads) {
                const int hl = p / pieces, pp = p % pieces;
                const int row = pp / (kChunk / per16), kp = (pp % (kChunk / per16)) * per16;
                const uint4 v = *(const uint4 *)((const unsigned char *)Mhi +
                                                 (((size_t)hl * NP + row) * Qp + c * kChunk + kp) * L::esz);
                *(uint4 *)((hl ? Blo : Bhi) + L::elem_off(row, kp)) = v;
            }
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint64_t ahi = smem_desc(smem_u32(Ahi), L::LBO, L::SBO);
                const uint64_t alo = smem_desc(smem_u32(Alo), L::LBO, L::SBO);
                const uint64_t bhi = smem_desc(smem_u32(Bhi), L::LBO, L::SBO);
                const uint64_t blo = smem_desc(smem_u32(Blo), L::LBO, L::SBO);
#pragma unroll
                for (int j = 0; j < kChunk / L::kmma; ++j) {
                    // each MMA covers 32 bytes of K = two core matrices = 2 * LBO bytes
                    const uint64_t step = (uint64_t)((j * 2 * L::LBO) >> 4);
                    mma_issue<BF16>(tmem, alo + step, bhi + step, idesc, (c > c_begin || j > 0) ? 1u : 0u);
                    mma_issue<BF16>(tmem, ahi + step, blo + step, idesc, 1u);
                    mma_issue<BF16>(tmem, ahi + step, bhi + step, idesc, 1u);
                }
                mma_commit(&bar[b]);
            }
            ++commits[b];
        }
        if (ring >= 0) ring_flush<NN>(T.ringWP + (size_t)ring * n2, B, [&](int cc) -> double & { return U[cc]; });
        // drain: every MMA of this tile has completed once both buffers' last commits have
        if (tid == 0)
            for (int b = 0; b < 2 && !*abort_flag; ++b)
                while (commits[b] > waited[b]) {
                    if (!mbar_wait_bounded(&bar[b], waited[b] & 1)) {
                        *abort_flag = 1;
                        break;
                    }
                    ++waited[b];
                }
        if (tid != 0)
            for (int b = 0; b < 2; ++b) waited[b] = commits[b];
        // the second half hands its gradient moments to the first
        if (h == 1) {
#pragma unroll
            for (int a = 0; a < n; ++a) sU[a * kTileM + r] = U[a];
        }
        __syncthreads();
        tc_fence_after();
        if (*abort_flag) break;
        // partial moments of this work item into its column of the accumulator: the FP64
        // gradient moments of both halves, the tensor-core moments from TMEM (warps 0-3)
        // A row handed to the FP64 Hessian gets its whole sums in part 0 from the FP64 sweep; its
        // other parts are stored as zeros, so that every column the Newton kernel reads was
        // written in this round.
        const bool store = r < rows && (MOMENTS_ONLY || active);
        const bool zero = !MOMENTS_ONLY && r < rows && cell >= 0 && !active && part > 0;
        double *row = Vacc + ((size_t)part * cnt_in + base + r) * vs_s;
        if (h == 0 && store) {
#pragma unroll
            for (int a = 0; a < n; ++a) row[(size_t)a * vs_c] = U[a] + sU[a * kTileM + r];
        }
        if (h == 0) {
            const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
#pragma unroll
            for (int c0 = 0; c0 < NP; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
                if (store) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (c0 + i < n2 - n) row[(size_t)(n + c0 + i) * vs_c] = (double)v[i];
                }
            }
            if (zero) {
#pragma unroll
                for (int c = 0; c < n2; ++c) row[(size_t)c * vs_c] = 0.0;
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    // an aborted tile may still have MMAs in flight: wait for them (bounded) before freeing TMEM
    if (tid == 0 && *abort_flag) {
        if (!MOMENTS_ONLY) atomicExch(&S.cnt[7], KITRT_ETIMEOUT);
        else atomicExch((int *)Vacc + 1, 0x7ff80000);  // poison the first moment (NaN high word)
        for (int b = 0; b < 2; ++b)
            while (commits[b] > waited[b]) {
                if (!mbar_wait_bounded(&bar[b], waited[b] & 1)) break;
                ++waited[b];
            }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, D::tcols);
}

template <int NN, bool BF16, bool MO>
int launch_mixed_impl(kitrt_mn *mn, const Tables &T, const NewtonState &S, const double *u, int k,
                      NewtonParams np, const double *alpha_in, double *Vacc, int C, cudaStream_t s,
                      float *psi32)
{
    using L = MixedSmem<NN, BF16>;
    if (ensure_dyn_smem(eval_mixed_kernel<NN, BF16, MO>, L::total)) return KITRT_ECUDA;
    // persistent grid of the CTAs that fit on the SMs at once; the work is split into about four
    // items per CTA (the moments of given alphas take one part per tile: rows of Vout are written
    // whole)
    eval_mixed_kernel<NN, BF16, MO><<<mn->grid_mixed, kThreads, L::total, s>>>(
        T, S, k, BF16 ? (const void *)mn->d_Mhi16 : (const void *)mn->d_Mhi32, alpha_in, Vacc,
        MO ? 1 : mn->vs, MO ? Dims<NN>::n2 : 1, C, MO ? 0 : mn->target_mixed, psi32);
    if (cudaGetLastError() != cudaSuccess) return KITRT_ECUDA;
    (void)u;
    (void)np;
    return KITRT_OK;
}

template <int NN, bool BF16>
int mixed_grid_impl(const kitrt_mn *mn)
{
    using L = MixedSmem<NN, BF16>;
    if (ensure_dyn_smem(eval_mixed_kernel<NN, BF16, false>, L::total)) return mn->nsm;
    return mn->nsm * resident_ctas(eval_mixed_kernel<NN, BF16, false>, kThreads, L::total, 2);
}

template <bool MO>
int launch_mixed_dispatch(kitrt_mn *mn, const Tables &T, const NewtonState &S, const double *u, int k,
                          NewtonParams np, const double *alpha_in, double *Vacc, int C, bool bf16,
                          cudaStream_t s, float *psi32)
{
#define MIXED_CASE(NNv)                                                                                  \
    case NNv:                                                                                            \
        return bf16 ? launch_mixed_impl<NNv, true, MO>(mn, T, S, u, k, np, alpha_in, Vacc, C, s, psi32) \
                    : launch_mixed_impl<NNv, false, MO>(mn, T, S, u, k, np, alpha_in, Vacc, C, s, psi32);
    switch (mn->N) {
        MIXED_CASE(1)
        MIXED_CASE(2)
        MIXED_CASE(3)
        MIXED_CASE(4)
        MIXED_CASE(5)
    default: return KITRT_EINVAL;
    }
#undef MIXED_CASE
}

}  // namespace

// Grid of the tensor-core sweep of a solver (CTAs resident at once).
int mixed_sweep_grid(const kitrt_mn *mn)
{
    const bool bf16 = mn->p.mode == KITRT_MIXED_BF16;
    switch (mn->N) {
    case 1: return bf16 ? mixed_grid_impl<1, true>(mn) : mixed_grid_impl<1, false>(mn);
    case 2: return bf16 ? mixed_grid_impl<2, true>(mn) : mixed_grid_impl<2, false>(mn);
    case 3: return bf16 ? mixed_grid_impl<3, true>(mn) : mixed_grid_impl<3, false>(mn);
    case 4: return bf16 ? mixed_grid_impl<4, true>(mn) : mixed_grid_impl<4, false>(mn);
    default: return bf16 ? mixed_grid_impl<5, true>(mn) : mixed_grid_impl<5, false>(mn);
    }
}

int launch_eval_mixed(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C, const double *u, int k,
                      NewtonParams np, cudaStream_t s, float *psi32)
{
    LaunchScope ls(mn, PK_EVAL_MIXED, s, 0);
    return launch_mixed_dispatch<false>(mn, T, S, u, k, np, nullptr, mn->d_Vacc, C,
                                        mn->p.mode == KITRT_MIXED_BF16, s, psi32);
}

int launch_moments_mixed(kitrt_mn *mn, const Tables &T, int C, const double *alpha, double *Vout,
                         cudaStream_t s)
{
    LaunchScope ls(mn, PK_OTHER, s, C);
    NewtonState S{};
    NewtonParams np{};
    if (cudaMemsetAsync(Vout, 0, sizeof(double) * (size_t)C * T.n2, s) != cudaSuccess) return KITRT_ECUDA;
    return launch_mixed_dispatch<true>(mn, T, S, nullptr, 0, np, alpha, Vout, C,
                                       mn->p.mode == KITRT_MIXED_BF16, s, nullptr);
}
