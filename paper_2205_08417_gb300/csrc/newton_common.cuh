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
                S.h64[cell] = 1;
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
            if (lane == 0) S.h64[cell] = 1;
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
        if (mixed && ph == PH_NEWTON && gn > kStallRatio * S.gnorm[cell]) S.h64[cell] = 1;
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

#define KITRT_PT_NAME newton_post_thread
#define KITRT_PT_UNROLL _Pragma("unroll")
#include "newton_post_thread_body.cuh"
#undef KITRT_PT_NAME
#undef KITRT_PT_UNROLL
#define KITRT_PT_NAME newton_post_thread_rolled
#define KITRT_PT_UNROLL _Pragma("unroll 1")
#include "newton_post_thread_body.cuh"
#undef KITRT_PT_NAME
#undef KITRT_PT_UNROLL

// Newton logic of every listed cell after a round of sweeps: thread per list slot, reading (and
// clearing) the slot's moment row. Counters (evaluations, largest count) are warp-aggregated.
// The slot's n2 moments are first copied to shared memory (all loads in flight together), where
// the Hessian assembly's table-driven reads then find them at shared-memory latency.
constexpr int kPostBlock = 64;
// N <= 3: the fully unrolled body (factor in registers, ~3k instructions per cell); the rolled
// body (factor in local memory) executes about four times as many instructions and measured
// slower (0.40 vs 0.30 ms per M_3 step), instruction fetch notwithstanding.
constexpr bool kUnrolledNewton = true;
template <int NN>
__global__ void __launch_bounds__(kPostBlock)
post_thread_kernel(Tables T, NewtonState S, const double *__restrict__ u, int k, NewtonParams np,
                   double *__restrict__ Vacc, int vs, int mixed, int target_items)
{
    constexpr int n2 = Dims<NN>::n2;
    __shared__ double sV[n2 * kPostBlock];  // [n2][thread]
    const int32_t *list_in = S.list[k & 1];
    int32_t *list_out = S.list[(k + 1) & 1];
    const int cnt_in = S.cnt[k % 3];
    // the sweeps split the quadrature of each tile into `parts` column blocks (sweep.cuh)
    const int parts = sweep_split(cnt_in, target_items, T.Qp / 32).parts;
    int32_t *cnt_out = &S.cnt[(k + 1) % 3];
    const int stride = gridDim.x * blockDim.x;
    const int rounds = (cnt_in + stride - 1) / stride;
    for (int rd = 0; rd < rounds; ++rd) {
        const int it = rd * stride + blockIdx.x * blockDim.x + threadIdx.x;
        bool cont = false;
        int cell = -1, ev = 0;
        if (it < cnt_in) {
            cell = list_in[it];
            // the slot's moments are column `it` of each part's block of the [n2 x vs]
            // accumulator (every one written by this round's sweeps): consecutive slots (threads)
            // read consecutive addresses; the parts are added in order
            double *mine = sV + threadIdx.x;
#pragma unroll
            for (int c = 0; c < n2; ++c) mine[c * kPostBlock] = 0.0;
            for (int p = 0; p < parts; ++p) {
                const double *row = Vacc + (size_t)p * cnt_in + it;
#pragma unroll
                for (int c = 0; c < n2; ++c) mine[c * kPostBlock] += row[(size_t)c * vs];
            }
            if constexpr (kUnrolledNewton && NN <= 3)
                cont = newton_post_thread<NN>(T, S, np, cell, mine, kPostBlock, u, mixed != 0, ev);
            else
                cont = newton_post_thread_rolled<NN>(T, S, np, cell, mine, kPostBlock, u, mixed != 0, ev);
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
