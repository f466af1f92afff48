// Device helpers shared by the closure kernels: warp reductions, the warp Cholesky factorisation
// and solves, and the per-cell Newton logic that follows one evaluation of the dual
// [Sec. 3.1, Eq. entropyOCP: dual f(alpha) = <exp(alpha.m)> - alpha.u, gradient <m e> - u,
// Hessian <m m^T e>], with Armijo backtracking.
#pragma once

#include <math.h>

#include "kitrt_internal.cuh"
#include "sweep.cuh"

namespace kitrt_dev {

constexpr unsigned kFull = 0xffffffffu;
// (1e-14)^2: residuals below 1e-14 ||u|| need no further Newton or polish step
constexpr double kRoundoff2 = 1e-28;
// mixed Hessian: a Newton step that does not halve the residual sends the cell to FP64
constexpr double kStallRatio = 0.5;

template <int NN>
struct Dims {
    static constexpr int n = (NN + 1) * (NN + 2) / 2;
    static constexpr int n2 = (2 * NN + 1) * (2 * NN + 2) / 2;
    static constexpr int npairs = n * (n + 1) / 2;
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ void push(int32_t *list, int32_t *cnt, int cell, int lane)
{
    if (lane == 0) {
        int pos = atomicAdd(cnt, 1);
        list[pos] = cell;
    }
}

// A mixed-mode cell goes over to the FP64 Hessian (FP64 sweep) from the next round on; counted
// once per cell and closure (S.cnt[11]).
__device__ __forceinline__ void hand_over(const NewtonState &S, int cell)
{
    if (!S.h64[cell]) {
        S.h64[cell] = 1;
        atomicAdd(&S.cnt[11], 1);
    }
}

__device__ __forceinline__ void fail(const NewtonState &S, int cell, int code, int lane)
{
    if (lane == 0) {
        S.status[cell] = code;
        S.phase[cell] = PH_DONE;
        atomicAdd(&S.cnt[3], 1);
    }
}

// Packed lower-triangle index of (a, b), b <= a.
__device__ __forceinline__ int tri_idx(int a, int b) { return a * (a + 1) / 2 + b; }

// Warp Cholesky of the n x n matrix in sH (row-major). On success the strict lower triangle
// holds L and the diagonal holds 1/L_jj, so the triangular solves multiply instead of divide
// (FP64 division costs many FP64-pipe instructions).
template <int n>
__device__ bool warp_cholesky(double *sH, int lane)
{
    for (int j = 0; j < n; ++j) {
        const double djj = sH[j * n + j];
        if (!(djj > 0.0)) return false;  // warp-uniform: every lane read the same value
        const double rinv = 1.0 / sqrt(djj);
        __syncwarp();
        if (lane > j && lane < n) sH[lane * n + j] *= rinv;
        if (lane == j) sH[j * n + j] = rinv;
        __syncwarp();
        if (lane > j && lane < n) {
            const double lij = sH[lane * n + j];
            for (int k = j + 1; k <= lane; ++k) sH[lane * n + k] = fma(-lij, sH[k * n + j], sH[lane * n + k]);
        }
        __syncwarp();
    }
    return true;
}

// Solve L L^T x = b (factor from warp_cholesky, inverse diagonal) with lane a holding b_a;
// returns x_a in lane a.
template <int n>
__device__ double warp_chol_solve(const double *sH, double b, int lane)
{
    double y = b;
    for (int j = 0; j < n; ++j) {
        const double yj = __shfl_sync(kFull, y, j) * sH[j * n + j];
        if (lane == j) y = yj;
        if (lane > j && lane < n) y = fma(-sH[lane * n + j], yj, y);
    }
    for (int j = n - 1; j >= 0; --j) {
        const double xj = __shfl_sync(kFull, y, j) * sH[j * n + j];
        if (lane == j) y = xj;
        if (lane < j) y = fma(-sH[j * n + lane], xj, y);
    }
    return lane < n ? y : 0.0;
}

// Newton logic of one cell after an evaluation of the dual at the trial point `at` (lane a holds
// component a). Vs holds the n2 degree-2N moments sum_q w_q e_q m~_c(q) (warp-visible), whose
// first n entries are the ansatz moments U. One warp per cell; every branch is warp-uniform.
//   mixed: the moments Vs[n..n2) came from tensor cores; a Cholesky breakdown or a stalled
//          residual sends the cell to the FP64 Hessian (S.h64) instead of failing it.
template <int NN>
__device__ void newton_post(const Tables &T, const NewtonState &S, const NewtonParams &np,
                            int cell, int ph, double lam, double at, double ua, const double *Vs,
                            double *H, int32_t *list_out, int32_t *cnt_out, int lane, bool mixed)
{
    constexpr int n = Dims<NN>::n, n2 = Dims<NN>::n2, npairs = Dims<NN>::npairs;
    const size_t off = (size_t)cell * n;
    bool finite = true;
    for (int c = 0; c < n2; ++c) finite = finite && isfinite(Vs[c]);
    const double fs = Vs[0] / T.m0;
    const double au = warp_sum(at * ua);
    const double ar2 = warp_sum(lane < n && lane >= np.reg0 ? at * at : 0.0);
    const double ft = fma(0.5 * np.gamma, ar2, fs - au);
    if (lane == 0) {
        const int ev = S.evals[cell] + 1;
        S.evals[cell] = ev;
        atomicMax(&S.cnt[4], ev);
        atomicAdd(&S.cnt[6], 1);
    }
    bool accept;
    if (ph == PH_INIT) {
        if (!finite) {
            fail(S, cell, KITRT_ENOTREALIZABLE, lane);
            return;
        }
        accept = true;
    } else {
        const double fs0 = S.fsum[cell], f0 = S.f0[cell];
        const double slack = 64.0 * 2.220446049250313e-16 * (fs0 + fabs(fs0 - f0));
        accept = finite && ft <= f0 + np.c1 * lam * S.gd[cell] + slack;
    }
    if (!accept) {
        const int h = S.halv[cell] + 1;
        if (h > np.max_halvings && mixed && !S.h64[cell]) {
            // as in newton_post_thread: restart from the accepted point with the FP64 Hessian
            if (lane == 0) {
                hand_over(S, cell);
                S.halv[cell] = 0;
                S.phase[cell] = PH_INIT;
            }
            push(list_out, cnt_out, cell, lane);
        } else if (h > np.max_halvings) {
            fail(S, cell, KITRT_ELINESEARCH, lane);
        } else {
            if (lane == 0) {
                S.halv[cell] = h;
                S.lam[cell] = 0.5 * lam;
            }
            push(list_out, cnt_out, cell, lane);
        }
        return;
    }
    // Hessian H_ab = sum_c G_abc V_c from the Gaunt coefficients
    for (int p = lane; p < npairs; p += 32) {
        int a = 0;
        while ((a + 1) * (a + 2) / 2 <= p) ++a;
        const int b = p - a * (a + 1) / 2;
        double h = 0.0;
        for (int t = T.gstart[p]; t < T.gstart[p + 1]; ++t) h = fma(T.gcoef[t], Vs[T.gidx[t]], h);
        if (a == b && a >= np.reg0) h += np.gamma;  // regularized moments
        H[a * n + b] = h;
        H[b * n + a] = h;
    }
    __syncwarp();
    if (!warp_cholesky<n>(H, lane)) {
        __syncwarp();
        if (mixed) {
            // tensor-core rounding broke positive definiteness: redo this point in FP64
            if (lane == 0) hand_over(S, cell);
            push(list_out, cnt_out, cell, lane);
        } else {
            fail(S, cell, KITRT_ECHOL, lane);
        }
        return;
    }
    // accepted: store the point, its moments and the factor of H
    const double Ua = lane < n ? Vs[lane] : 0.0;
    if (lane < n) {
        S.alpha[off + lane] = at;
        S.U[off + lane] = Ua;
    }
    if (lane == 0) {
        S.fsum[cell] = fs;
        S.f0[cell] = ft;
    }
    for (int a = lane; a < n; a += 32)
        for (int b = 0; b <= a; ++b) S.L[(size_t)cell * npairs + tri_idx(a, b)] = H[a * n + b];
    if (lane == 0 && S.lfac) S.lfac[cell] = 1;
    const double g = lane < n ? fma(lane >= np.reg0 ? np.gamma : 0.0, at, Ua - ua) : 0.0;
    const double d = warp_chol_solve<n>(H, -g, lane);
    __syncwarp();
    const double gn2 = warp_sum(g * g), un2 = warp_sum(ua * ua), gd = warp_sum(g * d);
    if (lane < n) S.dir[off + lane] = d;
    int iters = S.iters[cell];
    if (ph == PH_NEWTON) ++iters;
    const double gn = sqrt(gn2);
    if (lane == 0) S.iters[cell] = iters;
    if (gn <= np.tau * sqrt(un2)) {
        if (lane == 0) S.phase[cell] = PH_DONE;
        return;
    }
    if (iters >= np.max_iter) {
        fail(S, cell, KITRT_ENOCONVERGE, lane);
        return;
    }
    if (lane == 0) {
        if (mixed && ph == PH_NEWTON && gn > kStallRatio * S.gnorm[cell]) hand_over(S, cell);
        if (S.gnorm) S.gnorm[cell] = gn;
        S.gd[cell] = gd;
        S.lam[cell] = 1.0;
        S.halv[cell] = 0;
        S.phase[cell] = PH_NEWTON;
    }
    push(list_out, cnt_out, cell, lane);
}

}  // namespace kitrt_dev

namespace kitrt_dev {

// Warp-aggregated append of `cell` to a list when pred holds (all active lanes must call it).
__device__ __forceinline__ void push_agg(int32_t *list, int32_t *cnt, int cell, bool pred)
{
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, pred);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(act, base, leader);
    if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = cell;
}

#define KITRT_PT_NAME newton_post_thread_rolled
#define KITRT_PT_UNROLL _Pragma("unroll 1")
#include "newton_post_thread_body.cuh"
#undef KITRT_PT_NAME
#undef KITRT_PT_UNROLL

// Compact thread-per-cell Newton step (N <= 3), the same logic as newton_post_thread with a
// small instruction footprint: the Hessian assembly, the Cholesky factorisation and the two
// triangular solves run as rolled loops over per-thread slices of shared memory (entry e of a
// thread at e * B + thread), instead of fully unrolled code over registers. With about one warp
// per SM in a typical round, the unrolled body (several thousand instructions, run once) waited
// mostly on instruction fetch (ncu: stalls on no_instruction ~3x those on memory); rolled loops
// run from the instruction cache. R is float (mixed modes, tensor-core cells) or double (FP64
// mode, and mixed-mode cells handed to the FP64 Hessian); dual, gradient, tests and iterate are
// FP64 either way (see the thread body's precision note).
__device__ __forceinline__ float r_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float r_rsqrt(float a) { return rsqrtf(a); }
__device__ __forceinline__ double r_rsqrt(double a) { return rsqrt(a); }
__device__ __forceinline__ bool r_pos(float d) { return d > 0.0f && d < 3.0e38f; }
__device__ __forceinline__ bool r_pos(double d) { return d > 0.0; }

// H (packed lower, + gamma on the regularized diagonal) from the Gaunt terms, its Cholesky factor
// (1/L_jj on the diagonal) in place, then y <- -H^-1 y in place. Vr: the moments in precision R,
// entry c at Vr[c BV]; entry e of L and y at e B.
// Returns false when the factorisation breaks down.
template <int NN, typename R>
__device__ bool hess_factor_solve(const Tables &T, const R *__restrict__ coef, const NewtonParams &np,
                                  const R *Vr, int BV, R *L, R *y, int B)
{
    constexpr int n = Dims<NN>::n, npairs = Dims<NN>::npairs;
#pragma unroll 1
    for (int p = 0; p < npairs; ++p) {
        R h = R(0);
        const int t1 = T.gstart[p + 1];
#pragma unroll 1
        for (int t = T.gstart[p]; t < t1; ++t) h = r_fma(coef[t], Vr[(size_t)T.gidx[t] * BV], h);
        L[(size_t)p * B] = h;
    }
    if (np.gamma != 0.0) {
        const R gam = (R)np.gamma;
#pragma unroll 1
        for (int j = np.reg0; j < n; ++j) L[(size_t)tri_idx(j, j) * B] += gam;
    }
    bool spd = true;
#pragma unroll 1
    for (int j = 0; j < n; ++j) {
        const int jj = j * (j + 1) / 2;
        R d = L[(size_t)(jj + j) * B];
#pragma unroll 1
        for (int k = 0; k < j; ++k) {
            const R l = L[(size_t)(jj + k) * B];
            d = r_fma(-l, l, d);
        }
        spd = spd && r_pos(d);
        const R rinv = r_rsqrt(d > R(0) ? d : R(1));
        L[(size_t)(jj + j) * B] = rinv;
#pragma unroll 1
        for (int i = j + 1; i < n; ++i) {
            const int ii = i * (i + 1) / 2;
            R sacc = L[(size_t)(ii + j) * B];
#pragma unroll 1
            for (int k = 0; k < j; ++k)
                sacc = r_fma(-L[(size_t)(ii + k) * B], L[(size_t)(jj + k) * B], sacc);
            L[(size_t)(ii + j) * B] = sacc * rinv;
        }
    }
    if (!spd) return false;
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        const int ii = i * (i + 1) / 2;
        R sacc = y[(size_t)i * B];
#pragma unroll 1
        for (int k = 0; k < i; ++k) sacc = r_fma(-L[(size_t)(ii + k) * B], y[(size_t)k * B], sacc);
        y[(size_t)i * B] = sacc * L[(size_t)(ii + i) * B];
    }
#pragma unroll 1
    for (int i = n - 1; i >= 0; --i) {
        R sacc = y[(size_t)i * B];
#pragma unroll 1
        for (int k = i + 1; k < n; ++k)
            sacc = r_fma(-L[(size_t)tri_idx(k, i) * B], y[(size_t)k * B], sacc);
        y[(size_t)i * B] = sacc * L[(size_t)tri_idx(i, i) * B];
    }
    return true;
}

// V, Vf: the cell's moments as in newton_post_thread (Vf: FP32 Hessian-only moments of a
// tensor-core cell); Lbase, ybase: shared-memory regions of [npairs x B] and [n x B] doubles, of
// which this thread (tid) owns column tid. The FP32 path keeps its floats in the low half of the
// same 8-byte slots (float stride 2B), so that threads of one block on different paths never
// touch each other's slots.
template <int NN>
__device__ bool newton_cell(const Tables &T, const NewtonState &S, const NewtonParams &np, int cell,
                            const double *__restrict__ V, float *__restrict__ Vf, double *Lbase,
                            double *ybase, int tid, int B, const double *__restrict__ u, bool mixed,
                            int &evals_out)
{
    constexpr int n = Dims<NN>::n, n2 = Dims<NN>::n2, npairs = Dims<NN>::npairs;
    const size_t off = (size_t)cell * n;
    const int ph = S.phase[cell];
    const double lam = ph == PH_NEWTON ? S.lam[cell] : 0.0;
    const bool reg = np.gamma != 0.0;
    const bool h32 = mixed && !S.h64[cell];
    double at[n], ua[n];
    double au = 0.0, ar2 = 0.0;
#pragma unroll
    for (int a = 0; a < n; ++a) {
        const double al = S.alpha[off + a];
        at[a] = ph == PH_NEWTON ? fma(lam, S.dir[off + a], al) : al;
        ua[a] = u[off + a];
        au = fma(at[a], ua[a], au);
        if (reg && a >= np.reg0) ar2 = fma(at[a], at[a], ar2);
    }
    bool finite = true;
#pragma unroll
    for (int c = 0; c < n2; ++c)
        finite = finite && (c < n || !h32 ? finite_bits(V[(size_t)c * B])
                                          : (__float_as_uint(Vf[(size_t)c * B]) & 0x7f800000u) != 0x7f800000u);
    const double fs = V[0] * T.rm0;
    const double ft = reg ? fma(0.5 * np.gamma, ar2, fs - au) : fs - au;
    const int ev = S.evals[cell] + 1;
    S.evals[cell] = ev;
    evals_out = ev;
    auto fail_t = [&](int code) {
        S.status[cell] = code;
        S.phase[cell] = PH_DONE;
        atomicAdd(&S.cnt[3], 1);
    };
    bool accept;
    if (ph == PH_INIT) {
        if (!finite) {
            fail_t(KITRT_ENOTREALIZABLE);
            return false;
        }
        accept = true;
    } else {
        const double fs0 = S.fsum[cell], f0 = S.f0[cell];
        const double slack = 64.0 * 2.220446049250313e-16 * (fs0 + fabs(fs0 - f0));
        accept = finite && ft <= f0 + np.c1 * lam * S.gd[cell] + slack;
    }
    if (!accept) {
        const int h = S.halv[cell] + 1;
        if (h > np.max_halvings) {
            if (h32) {
                // the line search could not follow the direction from the tensor-core Hessian:
                // restart from the accepted point with the FP64 Hessian
                hand_over(S, cell);
                S.halv[cell] = 0;
                S.phase[cell] = PH_INIT;
                return true;
            }
            fail_t(KITRT_ELINESEARCH);
            return false;
        }
        S.halv[cell] = h;
        S.lam[cell] = 0.5 * lam;
        return true;
    }
    double g[n];
#pragma unroll
    for (int a = 0; a < n; ++a) {
        g[a] = V[(size_t)a * B] - ua[a];
        if (reg && a >= np.reg0) g[a] = fma(np.gamma, at[a], g[a]);
    }
    double y[n];
    if (h32) {
        float *Lf = reinterpret_cast<float *>(Lbase + tid), *yf = reinterpret_cast<float *>(ybase + tid);
        const int B2 = 2 * B;
#pragma unroll
        for (int c = 0; c < n; ++c) Vf[(size_t)c * B] = d2f_bits(V[(size_t)c * B]);
#pragma unroll
        for (int a = 0; a < n; ++a) yf[(size_t)a * B2] = -d2f_bits(g[a]);
        if (!hess_factor_solve<NN, float>(T, T.gcoef32, np, Vf, B, Lf, yf, B2)) {
            hand_over(S, cell);  // rounding broke positive definiteness: redo this point in FP64
            return true;
        }
#pragma unroll
        for (int a = 0; a < n; ++a) y[a] = f2d_bits(yf[(size_t)a * B2]);
#pragma unroll 1
        for (int p = 0; p < npairs; ++p) S.L[(size_t)cell * npairs + p] = f2d_bits(Lf[(size_t)p * B2]);
    } else {
        double *Lsm = Lbase + tid, *ysm = ybase + tid;
#pragma unroll
        for (int a = 0; a < n; ++a) ysm[(size_t)a * B] = -g[a];
        if (!hess_factor_solve<NN, double>(T, T.gcoef, np, V, B, Lsm, ysm, B)) {
            // FP64 mode, or the FP64 Hessian of a handed-over cell: no further fallback
            fail_t(KITRT_ECHOL);
            return false;
        }
#pragma unroll
        for (int a = 0; a < n; ++a) y[a] = ysm[(size_t)a * B];
#pragma unroll 1
        for (int p = 0; p < npairs; ++p) S.L[(size_t)cell * npairs + p] = Lsm[(size_t)p * B];
    }
#pragma unroll
    for (int a = 0; a < n; ++a) {
        S.alpha[off + a] = at[a];
        S.U[off + a] = V[(size_t)a * B];
    }
    S.fsum[cell] = fs;
    S.f0[cell] = ft;
    if (S.lfac) S.lfac[cell] = 1;
    double gn2 = 0.0, un2 = 0.0, gd = 0.0;
#pragma unroll
    for (int a = 0; a < n; ++a) {
        gn2 = fma(g[a], g[a], gn2);
        un2 = fma(ua[a], ua[a], un2);
        gd = fma(g[a], y[a], gd);
        S.dir[off + a] = y[a];
    }
    int iters = S.iters[cell];
    if (ph == PH_NEWTON) ++iters;
    S.iters[cell] = iters;
    const double gn = sqrt(gn2);
    if (gn <= np.tau * sqrt(un2)) {
        S.phase[cell] = PH_DONE;
        return false;
    }
    if (iters >= np.max_iter) {
        fail_t(KITRT_ENOCONVERGE);
        return false;
    }
    if (mixed && ph == PH_NEWTON && gn > kStallRatio * S.gnorm[cell]) hand_over(S, cell);
    if (S.gnorm) S.gnorm[cell] = gn;
    S.gd[cell] = gd;
    S.lam[cell] = 1.0;
    S.halv[cell] = 0;
    S.phase[cell] = PH_NEWTON;
    return true;
}

// Newton logic of every listed cell after a round of sweeps: thread per list slot, reading the
// slot's moment row. Counters (evaluations, largest count) are warp-aggregated.
// A round's list is often a few thousand cells, about one warp per SM, so the kernel is bound by
// the latency of each thread's serial chain, not by throughput. Two things keep that chain short:
//  - the slot's n2 moments are summed over the sweep's parts into shared memory one part at a
//    time (the n2 loads of a part in flight together: `parts` round trips to memory, not n2 x
//    parts);
//  - the Gaunt tables (term ranges, moment indices, coefficients) are staged in shared memory
//    once per block, so the table-driven Hessian assembly waits on shared memory, not on L2.
// In the mixed modes the parts of a tensor-core cell's Hessian-only moments (degree > N) are FP32
// numbers (tensor-core accumulators) and are added in FP32 into the FP32 copy; the degree <= N
// moments (gradient and dual) are always added in FP64.
constexpr int kPostBlock = 64;
// N <= 3: the compact body (newton_cell: rolled loops over a shared-memory factor); N >= 4: the
// thread body with its loops rolled over a factor in local memory (the shared-memory slices of
// 120 or 231 doubles per thread would leave room for too few blocks on the large passes).
constexpr bool kUnrolledNewton = true;

// Dynamic shared memory of post_thread_kernel: [n2 x kPostBlock] doubles (moments), for N <= 3
// the compact body's [npairs x kPostBlock] and [n x kPostBlock] doubles (factor, solve vector),
// the Gaunt coefficients of the mode (FP64, or FP32 in the mixed modes), [n2 x kPostBlock] floats
// (mixed modes), the moment indices and the npairs + 1 term starts.
__host__ __device__ inline size_t post_smem_bytes(int n, int n2, int npairs, int nnz, bool mixed,
                                                  bool compact)
{
    return (size_t)n2 * kPostBlock * 8 + (compact ? (size_t)(npairs + n) * kPostBlock * 8 : 0) +
           (size_t)nnz * (mixed ? 4 : 8) + (mixed ? (size_t)n2 * kPostBlock * 4 : 0) +
           (size_t)nnz * 4 + (size_t)(npairs + 1) * 4;
}

template <int NN>
__global__ void __launch_bounds__(kPostBlock)
post_thread_kernel(Tables T, NewtonState S, const double *__restrict__ u, int k, NewtonParams np,
                   const double *__restrict__ Vacc, int vs, int mixed, int target_items, int nnz)
{
    constexpr int n = Dims<NN>::n, n2 = Dims<NN>::n2, npairs = Dims<NN>::npairs;
    constexpr bool compact = kUnrolledNewton && NN <= 3;
    extern __shared__ __align__(16) unsigned char post_smem[];
    double *sV = reinterpret_cast<double *>(post_smem);                     // [n2][thread]
    double *sL = sV + (size_t)n2 * kPostBlock;                              // [npairs][thread]
    double *sy = sL + (size_t)npairs * kPostBlock;                          // [n][thread]
    // byte layout of post_smem_bytes: sV | sL, sy (compact) | coef | sVf (mixed) | gidx | gstart
    unsigned char *coef = post_smem + (size_t)(n2 + (compact ? npairs + n : 0)) * kPostBlock * 8;
    float *sVf = reinterpret_cast<float *>(coef + (size_t)nnz * (mixed ? 4 : 8));  // [n2][thread]
    int32_t *gidx = reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(sVf) +
                                                (mixed ? (size_t)n2 * kPostBlock * 4 : 0));
    int32_t *gstart = gidx + nnz;
    const int32_t *list_in = S.list[k & 1];
    int32_t *list_out = S.list[(k + 1) & 1];
    const int cnt_in = S.cnt[k % 3];
    const int stride = gridDim.x * blockDim.x;
    if ((int)(blockIdx.x * blockDim.x) >= cnt_in) return;  // uniform: this block has no slot
    // the sweeps split the quadrature of each tile into `parts` column blocks (sweep.cuh)
    const int parts = sweep_split(cnt_in, target_items, T.Qp / 32).parts;
    int32_t *cnt_out = &S.cnt[(k + 1) % 3];
    // stage the Gaunt tables and point this block's view of them at the copies
    for (int t = threadIdx.x; t < nnz; t += blockDim.x) {
        gidx[t] = T.gidx[t];
        if (mixed) reinterpret_cast<float *>(coef)[t] = T.gcoef32[t];
        else reinterpret_cast<double *>(coef)[t] = T.gcoef[t];
    }
    for (int t = threadIdx.x; t <= npairs; t += blockDim.x) gstart[t] = T.gstart[t];
    __syncthreads();
    Tables Ts = T;
    Ts.gidx = gidx;
    Ts.gstart = gstart;
    if (mixed) Ts.gcoef32 = reinterpret_cast<const float *>(coef);
    else Ts.gcoef = reinterpret_cast<const double *>(coef);
    const int rounds = (cnt_in + stride - 1) / stride;
    for (int rd = 0; rd < rounds; ++rd) {
        const int it = rd * stride + blockIdx.x * blockDim.x + threadIdx.x;
        bool cont = false;
        int cell = -1, ev = 0;
        if (it < cnt_in) {
            cell = list_in[it];
            const bool h32 = mixed && !S.h64[cell];
            // the slot's moments are column `it` of each part's block of the [n2 x vs]
            // accumulator (every one written by this round's sweeps): consecutive slots (threads)
            // read consecutive addresses; the parts are added in order
            double *mine = sV + threadIdx.x;
            float *minef = sVf + threadIdx.x;
#pragma unroll
            for (int c = 0; c < n2; ++c) {
                if (c < n || !h32) mine[c * kPostBlock] = 0.0;
                else minef[c * kPostBlock] = 0.0f;
            }
            for (int p = 0; p < parts; ++p) {
                const double *row = Vacc + (size_t)p * cnt_in + it;
#pragma unroll
                for (int c = 0; c < n2; ++c) {
                    const double x = row[(size_t)c * vs];
                    if (c < n || !h32) mine[c * kPostBlock] += x;
                    else minef[c * kPostBlock] += d2f_bits(x);
                }
            }
            if constexpr (compact)
                cont = newton_cell<NN>(Ts, S, np, cell, mine, minef, sL, sy, threadIdx.x, kPostBlock,
                                       u, mixed != 0, ev);
            else
                cont = newton_post_thread_rolled<NN>(Ts, S, np, cell, mine, minef, kPostBlock, u, mixed != 0, ev);
        }
        // every slot taken in this round is one evaluation
        const unsigned act = __activemask();
        const unsigned live = __ballot_sync(act, it < cnt_in);
        const int evmax = __reduce_max_sync(act, ev);
        if ((threadIdx.x & 31) == __ffs(act) - 1 && live) {
            atomicAdd(&S.cnt[6], __popc(live));
            atomicMax(&S.cnt[4], evmax);
        }
        push_agg(list_out, cnt_out, cell, cont);
    }
}

}  // namespace kitrt_dev
