// FP64 entropy closure: Newton's method on the dual of the minimum-entropy problem
// [Sec. 3.1, Eq. entropyOCP; Maxwell-Boltzmann entropy], with Armijo backtracking.
//
// One warp owns one cell. The quadrature sums run lane-strided over the folded points:
//   z_q = alpha . m_q,  e_q = w_q exp(z_q),  V_c = sum_q e_q m~_c(q)   (c over the degree-2N
// basis), so that U = V[0:n] are the ansatz moments, <exp(alpha.m)> = V_0 / m_0 and the Hessian
// H_ab = sum_c G_abc V_c (Gaunt coefficients) comes without per-point pair products. The Cholesky
// factorisation and the triangular solves are spread over the warp (lane = matrix row).
//
// Cells that still iterate are kept in a compacted list; every launch advances each listed cell
// by one evaluation (one trial point of the line search) and writes the cells that continue into
// the next list. Counters rotate over three slots so that no launch has to clear the slot it
// fills.
#include <math.h>

#include "kitrt_internal.cuh"
#include "kexp.cuh"
#include "newton_common.cuh"
#include "sweep.cuh"

namespace {

using namespace kitrt_dev;
constexpr int kWarps = 8;  // warps per block
constexpr int kThreadBlock = 64;  // block of the thread-per-cell Newton kernels

// ---------------------------------------------------------------------------------------------
// begin: start a closure. first == 1: every cell starts from alpha_in with an evaluation.
// first == 0: the previous closure left alpha_k, its moments U, <exp>, and the Cholesky factor
// of H(alpha_k); with the new u the gradient is U - u. One thread per cell tests it: a cell
// already converged (and with no polish step to take) is done at once; the others go to the
// predictor list, where predict_kernel takes the first Newton direction from the stored factor
// without a new quadrature pass.
// first == 2: per cell, the second case when alpha_in is bit for bit the alpha the last closure
// returned for this cell (alpha_k, plus the polish step when polishing) and that closure
// succeeded, so the stored state is exactly the state behind the given alpha; the first case
// otherwise (the cell's stored <exp> is then poisoned, so that the learned pass cannot mistake
// it for a previous point).
// ---------------------------------------------------------------------------------------------

// Warp-aggregated append of `cell` to a list when pred holds (all active lanes call it).
__device__ __forceinline__ void push_if(int32_t *list, int32_t *cnt, int cell, bool pred)
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

template <int NN>
__global__ void __launch_bounds__(256)
begin_test_kernel(NewtonState S, const double *__restrict__ u, const double *__restrict__ alpha_in,
                  int first, NewtonParams np, int C, int learned)
{
    constexpr int n = Dims<NN>::n;
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < C; cell += gridDim.x * blockDim.x) {
        const size_t off = (size_t)cell * n;
        bool cold = first == 1;
        if (first == 2) {
            // the alpha the finish kernel returned: alpha_k (+ the polish step when polishing)
            bool same = S.status[cell] == 0;
#pragma unroll
            for (int a = 0; a < n; ++a) {
                double out = S.alpha[off + a];
                if (np.polish) out += S.dir[off + a];
                same = same && __double_as_longlong(out) == __double_as_longlong(alpha_in[off + a]);
            }
            cold = !same;
        }
        S.iters[cell] = 0;
        S.halv[cell] = 0;
        S.evals[cell] = 0;
        S.status[cell] = 0;
        if (S.h64) S.h64[cell] = 0;
        if (S.gnorm) S.gnorm[cell] = INFINITY;
        bool to_eval = false, to_predict = false;
        if (cold) {
#pragma unroll
            for (int a = 0; a < n; ++a) S.alpha[off + a] = alpha_in[off + a];
            S.phase[cell] = PH_INIT;
            if (first == 2) S.fsum[cell] = __longlong_as_double(0x7ff8000000000000LL);
            // learned closures go to the network first (the predictor list doubles as its list)
            to_eval = !learned;
            to_predict = learned;
        } else {
            double gn2 = 0.0, un2 = 0.0;
#pragma unroll
            for (int a = 0; a < n; ++a) {
                const double ua = u[off + a];
                double g = S.U[off + a] - ua;
                if (a >= np.reg0) g = fma(np.gamma, S.alpha[off + a], g);
                gn2 = fma(g, g, gn2);
                un2 = fma(ua, ua, un2);
            }
            if (gn2 <= kRoundoff2 * un2 || (!np.polish && gn2 <= np.tau * np.tau * un2)) {
                // already converged and no polish step to take (the polish is off, or the residual
                // is at round-off, where it would move alpha by less than its own rounding)
#pragma unroll
                for (int a = 0; a < n; ++a) S.dir[off + a] = 0.0;
                S.phase[cell] = PH_DONE;
            } else {
                to_predict = true;
            }
        }
        push_if(S.list[0], &S.cnt[0], cell, to_eval);
        push_if(S.list[1], &S.cnt[8], cell, to_predict);
    }
}

template <int NN>
__global__ void __launch_bounds__(kWarps * 32)
predict_kernel(NewtonState S, const double *__restrict__ u, NewtonParams np)
{
    constexpr int n = Dims<NN>::n, npairs = Dims<NN>::npairs;
    __shared__ double sH[kWarps][n * n];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double *H = sH[wib];
    const int cnt = S.cnt[8];
    for (int it = blockIdx.x * kWarps + wib; it < cnt; it += gridDim.x * kWarps) {
        const int cell = S.list[1][it];
        const size_t off = (size_t)cell * n;
        const double ua = lane < n ? u[off + lane] : 0.0;
        const double al = lane < n ? S.alpha[off + lane] : 0.0;
        const double g = lane < n ? fma(lane >= np.reg0 ? np.gamma : 0.0, al, S.U[off + lane] - ua) : 0.0;
        const double ar2 = warp_sum(lane < n && lane >= np.reg0 ? al * al : 0.0);
        for (int a = lane; a < n; a += 32)
            for (int b = 0; b <= a; ++b) H[a * n + b] = S.L[(size_t)cell * npairs + tri_idx(a, b)];
        __syncwarp();
        const double d = warp_chol_solve<n>(H, -g, lane);
        __syncwarp();
        const double gn2 = warp_sum(g * g), un2 = warp_sum(ua * ua);
        if (lane < n) S.dir[off + lane] = d;
        if (sqrt(gn2) <= np.tau * sqrt(un2)) {
            if (lane == 0) S.phase[cell] = PH_DONE;  // converged; d is the polish step
            continue;
        }
        const double au = warp_sum(al * ua), gd = warp_sum(g * d);
        if (lane == 0) {
            if (S.gnorm) S.gnorm[cell] = sqrt(gn2);
            const double fs = S.fsum[cell];
            S.f0[cell] = fma(0.5 * np.gamma, ar2, fs - au);
            S.gd[cell] = gd;
            S.lam[cell] = 1.0;
            S.phase[cell] = PH_NEWTON;
        }
        push(S.list[0], &S.cnt[0], cell, lane);
    }
}

// Thread-per-cell version of predict_kernel for N <= 3 (the packed factor fits in registers):
// every FP64 instruction of the triangular solves keeps all 32 lanes busy.
template <int NN>
__global__ void __launch_bounds__(256)
predict_thread_kernel(NewtonState S, const double *__restrict__ u, NewtonParams np)
{
    constexpr int n = Dims<NN>::n, npairs = Dims<NN>::npairs;
    const int cnt = S.cnt[8];
    const int stride = gridDim.x * blockDim.x;
    const int rounds = (cnt + stride - 1) / stride;
    for (int rd = 0; rd < rounds; ++rd) {
        const int it = rd * stride + blockIdx.x * blockDim.x + threadIdx.x;
        bool cont = false;
        int cell = -1;
        if (it < cnt) {
            cell = S.list[1][it];
            const size_t off = (size_t)cell * n;
            double Lp[npairs], y[n], g[n];
            double gn2 = 0.0, un2 = 0.0, au = 0.0, ar2 = 0.0;
#pragma unroll
            for (int p = 0; p < npairs; ++p) Lp[p] = S.L[(size_t)cell * npairs + p];
#pragma unroll
            for (int a = 0; a < n; ++a) {
                const double ua = u[off + a], al = S.alpha[off + a];
                g[a] = S.U[off + a] - ua;
                if (a >= np.reg0) {
                    g[a] = fma(np.gamma, al, g[a]);
                    ar2 = fma(al, al, ar2);
                }
                gn2 = fma(g[a], g[a], gn2);
                un2 = fma(ua, ua, un2);
                au = fma(al, ua, au);
                y[a] = -g[a];
            }
            // d = -H^-1 g with the stored factor (1/L_jj on its diagonal)
#pragma unroll
            for (int i = 0; i < n; ++i) {
                double t = y[i];
#pragma unroll
                for (int k = 0; k < i; ++k) t = fma(-Lp[tri_idx(i, k)], y[k], t);
                y[i] = t * Lp[tri_idx(i, i)];
            }
#pragma unroll
            for (int i = n - 1; i >= 0; --i) {
                double t = y[i];
#pragma unroll
                for (int k = i + 1; k < n; ++k) t = fma(-Lp[tri_idx(k, i)], y[k], t);
                y[i] = t * Lp[tri_idx(i, i)];
            }
            double gd = 0.0;
#pragma unroll
            for (int a = 0; a < n; ++a) {
                S.dir[off + a] = y[a];
                gd = fma(g[a], y[a], gd);
            }
            if (sqrt(gn2) <= np.tau * sqrt(un2)) {
                S.phase[cell] = PH_DONE;  // converged; d is the polish step
            } else {
                if (S.gnorm) S.gnorm[cell] = sqrt(gn2);
                S.f0[cell] = fma(0.5 * np.gamma, ar2, S.fsum[cell] - au);
                S.gd[cell] = gd;
                S.lam[cell] = 1.0;
                S.phase[cell] = PH_NEWTON;
                cont = true;
            }
        }
        push_agg(S.list[0], &S.cnt[0], cell, cont);
    }
}

// ---------------------------------------------------------------------------------------------
// eval: one trial point per listed cell (alpha + lam dir, or alpha itself for PH_INIT), then the
// Armijo decision, and on acceptance the Hessian, its Cholesky factor, the convergence test and
// the next Newton direction.
// ---------------------------------------------------------------------------------------------
// FUSED: the warp also runs the per-cell Newton logic (used by the allocation-free closure);
// otherwise the sweep writes the cell's moments to column `list slot` of Vacc [n2 x C] for the
// post kernel.
template <int NN, bool FILTER, bool FUSED>
__global__ void __launch_bounds__(kWarps * 32)
eval_kernel(Tables T, NewtonState S, const double *__restrict__ u, int k, NewtonParams np,
            float *__restrict__ psi32, double *__restrict__ Vacc, int vs)
{
    constexpr int n = Dims<NN>::n, n2 = Dims<NN>::n2;
    __shared__ double sH[kWarps][n * n];
    __shared__ double sV[kWarps][n2];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int32_t *list_in = S.list[k & 1];
    int32_t *list_out = S.list[(k + 1) & 1];
    const int cnt_in = S.cnt[k % 3];
    int32_t *cnt_out = &S.cnt[(k + 1) % 3];
    // FILTER: the FP64 companion of the mixed sweep; it only takes cells flagged for an FP64
    // Hessian and leaves the counter bookkeeping to the mixed kernel
    if (!FILTER && blockIdx.x == 0 && threadIdx.x == 0) S.cnt[(k + 2) % 3] = 0;
    double *H = sH[wib];
    double *Vs = sV[wib];
    const int Qp = T.Qp;
    const double *__restrict__ Mt = T.Mt;
    const double *__restrict__ wq = T.w;

    // one listed cell: its trial point, the quadrature sums, then (FUSED) the Newton logic or
    // (otherwise) its moments into column `it` of Vacc
    auto cell_pass = [&](int it) {
        const int cell = list_in[it];
        const size_t off = (size_t)cell * n;
        const int ph = S.phase[cell];
        const double ua = lane < n ? u[off + lane] : 0.0;
        const double al = lane < n ? S.alpha[off + lane] : 0.0;
        const double lam = ph == PH_NEWTON ? S.lam[cell] : 0.0;
        const double di = (ph == PH_NEWTON && lane < n) ? S.dir[off + lane] : 0.0;
        const double at = lane < n ? fma(lam, di, al) : 0.0;
        double atv[n];
#pragma unroll
        for (int a = 0; a < n; ++a) atv[a] = __shfl_sync(kFull, at, a);

        double V[n2];
#pragma unroll
        for (int c = 0; c < n2; ++c) V[c] = 0.0;
        for (int q = lane; q < Qp; q += 32) {
            double z = 0.0;
#pragma unroll
            for (int a = 0; a < n; ++a) z = fma(atv[a], Mt[a * Qp + q], z);
            const double ez = kexp(z, T.exptab);
            // the ansatz of the trial point: the last accepted trial of a closure leaves the
            // ansatz of its solution behind, so no separate pass is needed
            if (psi32) psi32[(size_t)cell * Qp + q] = exp_to_float(ez);
            const double e = wq[q] * ez;
#pragma unroll
            for (int c = 0; c < n2; ++c) V[c] = fma(e, Mt[c * Qp + q], V[c]);
        }
#pragma unroll
        for (int c = 0; c < n2; ++c) V[c] = warp_sum(V[c]);
        if (!FUSED) {
#pragma unroll
            for (int c = 0; c < n2; ++c)
                if (lane == (c & 31)) Vacc[(size_t)c * vs + it] = V[c];
            return;
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < n2; ++c)
            if (lane == (c & 31)) Vs[c] = V[c];
        __syncwarp();
        newton_post<NN>(T, S, np, cell, ph, lam, at, ua, Vs, H, list_out, cnt_out, lane, false);
        __syncwarp();
    };
    if (FILTER) {
        // the FP64 companion of the mixed sweep takes only the (rare) cells flagged for an FP64
        // Hessian: each warp tests 32 list entries at once and evaluates the flagged ones
        for (int b0 = (blockIdx.x * kWarps + wib) * 32; b0 < cnt_in; b0 += gridDim.x * kWarps * 32) {
            const int e = b0 + lane;
            unsigned m = __ballot_sync(kFull, e < cnt_in && S.h64[list_in[e]] != 0);
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                cell_pass(b0 + b);
            }
        }
    } else {
        for (int it = blockIdx.x * kWarps + wib; it < cnt_in; it += gridDim.x * kWarps) cell_pass(it);
    }
}

// ---------------------------------------------------------------------------------------------
// FP64 sweep of the FP64 mode: one thread per listed cell (tiles of 128), every degree-2N moment
// in the sum-factorised form of sweep.cuh. Work items are (tile, part of the quadrature); each
// stores its partial moments with plain stores into its own column block of Vacc, which the
// Newton kernel adds in order, so the result does not depend on scheduling.
// ---------------------------------------------------------------------------------------------
constexpr int kSweepThreads = 128;

template <int NN>
__global__ void __launch_bounds__(kSweepThreads)
sweep64_kernel(Tables T, NewtonState S, int k, double *__restrict__ Vacc, int vs, int target_items)
{
    constexpr int n = Dims<NN>::n, n2 = Dims<NN>::n2, NA = 2 * NN + 1, NB = 4 * NN + 1;
    constexpr int TW = 4 * NN + 1;
    __shared__ double sV[n2 * kSweepThreads];  // [n2][thread]
    const int32_t *list_in = S.list[k & 1];
    const int cnt_in = S.cnt[k % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) S.cnt[(k + 2) % 3] = 0;
    const int nunits = T.Qp / 32;
    const SweepSplit sp = sweep_split(cnt_in, target_items, nunits);
    const int items = sp.tiles * sp.parts;
    double *mine = sV + threadIdx.x;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int tile = item / sp.parts, part = item % sp.parts;
        const int slot = tile * kSweepThreads + threadIdx.x;
        if (slot >= cnt_in) continue;  // threads are independent: no block barrier below
        const int p_begin = part * sp.units_per_part * 16;
        // padding pairs (w = 0) add nothing: stop at the last real pair
        const int p_end = min(T.npair, min(nunits, (part + 1) * sp.units_per_part) * 16);
        const int cell = list_in[slot];
        const size_t off = (size_t)cell * n;
        const int ph = S.phase[cell];
        const double lam = ph == PH_NEWTON ? S.lam[cell] : 0.0;
        double at[n], A[NA], B[NB];
#pragma unroll
        for (int a = 0; a < n; ++a) {
            const double al = S.alpha[off + a];
            at[a] = ph == PH_NEWTON ? fma(lam, S.dir[off + a], al) : al;
        }
#pragma unroll
        for (int c = 0; c < n2; ++c) mine[c * kSweepThreads] = 0.0;
#pragma unroll
        for (int j = 0; j < NB; ++j) B[j] = 0.0;
        auto V = [&](int c) -> double & { return mine[c * kSweepThreads]; };
        int ring = -1;
        for (int pr = p_begin; pr < p_end; ++pr) {
            const int rg = pr < T.npair ? pr / T.P : T.R;
            if (rg != ring) {
                if (ring >= 0) ring_flush<2 * NN>(T.ringWP + (size_t)ring * n2, B, V);
                ring_coeffs<NN>(at, T.ringP + (size_t)rg * n2, A);
                ring = rg;
            }
            double e1, e2;
            pair_eval<NN, 2 * NN>(A, T.ptrig + (size_t)pr * TW, pr < T.npair && pr % T.P == 0,
                                  T.exptab, B, e1, e2);
        }
        if (ring >= 0) ring_flush<2 * NN>(T.ringWP + (size_t)ring * n2, B, V);
        double *col = Vacc + (size_t)part * cnt_in + slot;
#pragma unroll
        for (int c = 0; c < n2; ++c) col[(size_t)c * vs] = mine[c * kSweepThreads];
    }
}

// ---------------------------------------------------------------------------------------------
// finish: final alpha (alpha_k plus the polish step if enabled) to the caller, and optionally the
// ansatz psi at every folded point (FP64 and/or FP32).
// ---------------------------------------------------------------------------------------------
template <int NN>
__global__ void __launch_bounds__(kWarps * 32)
finish_kernel(Tables T, NewtonState S, double *__restrict__ alpha_out, double *__restrict__ psi,
              float *__restrict__ psi32, int polish, int compare_prev, int C)
{
    constexpr int n = Dims<NN>::n;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int Qp = T.Qp;
    for (int cell = blockIdx.x * kWarps + wib; cell < C; cell += gridDim.x * kWarps) {
        const size_t off = (size_t)cell * n;
        const bool ok = S.status[cell] == 0;
        double a = lane < n ? S.alpha[off + lane] : 0.0;
        if (ok && polish && lane < n) a += S.dir[off + lane];
        // alpha_out still holds the previous step's alpha (and psi its ansatz) when compare_prev
        // is set: a bitwise-unchanged alpha leaves psi as it is
        if (compare_prev) {
            const double prev = lane < n ? alpha_out[off + lane] : 0.0;
            if (__all_sync(kFull, prev == a)) continue;
        }
        if (lane < n) alpha_out[off + lane] = a;
        if (!psi && !psi32) continue;
        double av[n];
#pragma unroll
        for (int b = 0; b < n; ++b) av[b] = __shfl_sync(kFull, a, b);
        for (int q = lane; q < T.Qf; q += 32) {
            double z = 0.0;
#pragma unroll
            for (int b = 0; b < n; ++b) z = fma(av[b], T.Mt[b * Qp + q], z);
            if (psi) {
                const double e = kexp(z, T.exptab);
                psi[(size_t)cell * Qp + q] = e;
                if (psi32) psi32[(size_t)cell * Qp + q] = (float)e;
            } else {
                // FP32 ansatz for the mixed modes: exact FP64 exponent split into z_hi + z_lo,
                // exp(z) = expf(z_hi) (1 + z_lo) to FP32 accuracy without an FP64 exp
                const float zh = (float)z;
                const float zl = (float)(z - (double)zh);
                psi32[(size_t)cell * Qp + q] = expf(zh) * (1.0f + zl);
            }
        }
    }
}

// finish without an ansatz to write (the mixed modes' sweeps already wrote it): the final alpha,
// element-wise over the C x n entries (coalesced, every lane busy).
__global__ void finish_alpha_kernel(NewtonState S, double *__restrict__ alpha_out, int polish, int n,
                                    int C)
{
    const size_t total = (size_t)C * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int cell = (int)(e / n);
        double a = S.alpha[e];
        if (polish && S.status[cell] == 0) a += S.dir[e];
        alpha_out[e] = a;
    }
}

// Degree-2N moments V_c = sum_q w_q exp(alpha.m_q) m~_c(q) of given alphas, in FP64.
template <int NN>
__global__ void __launch_bounds__(kWarps * 32)
moments_kernel(Tables T, const double *__restrict__ alpha, double *__restrict__ V, int C)
{
    constexpr int n = Dims<NN>::n, n2 = Dims<NN>::n2;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int Qp = T.Qp;
    for (int cell = blockIdx.x * kWarps + wib; cell < C; cell += gridDim.x * kWarps) {
        double av[n], acc[n2];
#pragma unroll
        for (int a = 0; a < n; ++a) av[a] = alpha[(size_t)cell * n + a];
#pragma unroll
        for (int c = 0; c < n2; ++c) acc[c] = 0.0;
        for (int q = lane; q < Qp; q += 32) {
            double z = 0.0;
#pragma unroll
            for (int a = 0; a < n; ++a) z = fma(av[a], T.Mt[a * Qp + q], z);
            const double e = T.w[q] * kexp(z, T.exptab);
#pragma unroll
            for (int c = 0; c < n2; ++c) acc[c] = fma(e, T.Mt[c * Qp + q], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < n2; ++c) {
            const double v = warp_sum(acc[c]);
            if (lane == 0) V[(size_t)cell * n2 + c] = v;
        }
    }
}

// Full Hessian H_ab = sum_c G_abc V_c (row-major n x n per cell) from degree-2N moments.
__global__ void gaunt_kernel(Tables T, const double *__restrict__ V, double *__restrict__ H, int C)
{
    const int n = T.n, n2 = T.n2, npairs = n * (n + 1) / 2;
    const size_t total = (size_t)C * npairs;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int cell = (int)(i / npairs), p = (int)(i % npairs);
        int a = 0;
        while ((a + 1) * (a + 2) / 2 <= p) ++a;
        const int b = p - a * (a + 1) / 2;
        double h = 0.0;
        for (int t = T.gstart[p]; t < T.gstart[p + 1]; ++t) h = fma(T.gcoef[t], V[(size_t)cell * n2 + T.gidx[t]], h);
        H[(size_t)cell * n * n + a * n + b] = h;
        H[(size_t)cell * n * n + b * n + a] = h;
    }
}

__global__ void isotropic_kernel(int n, double m0, const double *__restrict__ u,
                                 double *__restrict__ alpha, int C)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        const double u0 = u[(size_t)c * n];
        alpha[(size_t)c * n] = log(u0 / (4.0 * 3.14159265358979323846 * m0)) / m0;
        for (int a = 1; a < n; ++a) alpha[(size_t)c * n + a] = 0.0;
    }
}

__global__ void ansatz_kernel(Tables T, const double *__restrict__ alpha, double *__restrict__ psi,
                              int C)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int n = T.n, Qp = T.Qp, Qf = T.Qf;
    for (int cell = blockIdx.x * kWarps + wib; cell < C; cell += gridDim.x * kWarps) {
        for (int q = lane; q < Qf; q += 32) {
            double z = 0.0;
            for (int b = 0; b < n; ++b) z = fma(alpha[(size_t)cell * n + b], T.Mt[b * Qp + q], z);
            psi[(size_t)cell * Qf + q] = kexp(z, T.exptab);
        }
    }
}

int grid_for(const kitrt_mn *mn, int C, int per_sm)
{
    const int need = (C + kWarps - 1) / kWarps;
    const int cap = mn->nsm * per_sm;
    return need < cap ? (need > 0 ? need : 1) : cap;
}

// The predictor: thread per cell while the packed factor fits in registers (N <= 3), else warp
// per cell with the factor in shared memory.
template <int NN>
void predict_launch(kitrt_mn *mn, const NewtonState &S, int C, const double *u, NewtonParams np,
                    cudaStream_t s)
{
    if constexpr (NN <= 3) {
        int tb = (C + kThreadBlock - 1) / kThreadBlock;
        if (tb > mn->nsm * 32) tb = mn->nsm * 32;
        predict_thread_kernel<NN><<<tb > 0 ? tb : 1, kThreadBlock, 0, s>>>(S, u, np);
    } else {
        predict_kernel<NN><<<grid_for(mn, C, 8), kWarps * 32, 0, s>>>(S, u, np);
    }
}

}  // namespace

#define KITRT_DISPATCH_N(N, ...)                        \
    switch (N) {                                        \
    case 1: { constexpr int NN = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int NN = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int NN = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int NN = 4; __VA_ARGS__; } break; \
    case 5: { constexpr int NN = 5; __VA_ARGS__; } break; \
    default: return KITRT_EINVAL;                       \
    }

int launch_isotropic(const Tables &T, int C, const double *u, double *alpha, cudaStream_t s)
{
    const int blocks = (C + 255) / 256;
    isotropic_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(T.n, T.m0, u, alpha, C);
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

// Sum of each listed slot's quadrature parts (written by the sweeps, sweep.cuh) into its part-0
// column, in order, element-wise over the [n2 x cnt] moments with every SM taking part, so that
// the Newton kernel's serial per-cell chain reads one column instead of `parts`. Tensor-core
// rows' Hessian-only moments (degree > N) are FP32 accumulator values and are added in FP32; the
// gradient moments, and every moment of a row handed to the FP64 sweep (its part 0 holds the
// FP64 sums, its other parts zeros), in FP64.
__global__ void sum_parts_kernel(NewtonState S, int k, double *__restrict__ Vacc, int vs, int n,
                                 int n2, int target_items, int nunits, int mixed)
{
    const int cnt = S.cnt[k % 3];
    const int parts = sweep_split(cnt, target_items, nunits).parts;
    if (parts <= 1) return;
    const int32_t *list = S.list[k & 1];
    const size_t total = (size_t)n2 * cnt, pstride = (size_t)cnt;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / cnt), j = (int)(e - (size_t)c * cnt);
        double *col = Vacc + (size_t)c * vs + j;
        if (mixed && c >= n && !S.h64[list[j]]) {
            float v = d2f_bits(col[0]);
            for (int p = 1; p < parts; ++p) v += d2f_bits(col[(size_t)p * pstride]);
            col[0] = f2d_bits(v);
        } else {
            double v = col[0];
            for (int p = 1; p < parts; ++p) v += col[(size_t)p * pstride];
            col[0] = v;
        }
    }
}

int launch_sum_parts(kitrt_mn *mn, const NewtonState &S, int k, double *Vacc, cudaStream_t s)
{
    const int mixed = mn->p.mode != KITRT_FP64;
    LaunchScope ls(mn, PK_POST, s, 0);
    sum_parts_kernel<<<mn->nsm * 8, 256, 0, s>>>(S, k, Vacc, mn->vs, mn->n, mn->n2,
                                                 mixed ? mn->target_mixed : mn->target_fp64,
                                                 mn->Qp / 32, mixed);
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

int launch_post(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C, const double *u, int k,
                NewtonParams np, double *Vacc, cudaStream_t s)
{
    // 64-thread blocks: the listed cells (often a few thousand) fill the low block indices, and
    // small blocks spread them over every SM instead of a few
    int blocks = (C + kPostBlock - 1) / kPostBlock;
    if (blocks > mn->nsm * 32) blocks = mn->nsm * 32;
    const int mixed = mn->p.mode != KITRT_FP64;
    // sum_parts_kernel has added the sweeps' parts into part 0 (target 0 gives one part)
    const int target = 0;
    const size_t smem = post_smem_bytes(mn->n, mn->n2, mn->npairs, mn->gaunt_nnz, mixed != 0,
                                        kUnrolledNewton && mn->N <= 3);
    int rc = KITRT_OK;
    KITRT_DISPATCH_N(mn->N, rc = ensure_dyn_smem(post_thread_kernel<NN>, smem));
    if (rc) return rc;
    LaunchScope ls(mn, PK_POST, s, 0);
    KITRT_DISPATCH_N(mn->N, post_thread_kernel<NN><<<blocks > 0 ? blocks : 1, kPostBlock, smem, s>>>(T, S, u, k, np, Vacc, mn->vs, mixed, target, mn->gaunt_nnz));
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

int launch_moments_fp64(kitrt_mn *mn, const Tables &T, int C, const double *alpha, double *V, cudaStream_t s)
{
    const int grid = grid_for(mn, C, 8);
    LaunchScope ls(mn, PK_OTHER, s, C);
    KITRT_DISPATCH_N(mn->N, moments_kernel<NN><<<grid, kWarps * 32, 0, s>>>(T, alpha, V, C));
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

int launch_gaunt(kitrt_mn *mn, const Tables &T, int C, const double *V, double *H, cudaStream_t s)
{
    const long total = (long)C * (T.n * (T.n + 1) / 2);
    int blocks = (int)((total + 255) / 256);
    if (blocks > mn->nsm * 16) blocks = mn->nsm * 16;
    LaunchScope ls(mn, PK_OTHER, s, C);
    gaunt_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(T, V, H, C);
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

int launch_ansatz(const Tables &T, int C, const double *alpha, double *psi, cudaStream_t s)
{
    const int blocks = (C + kWarps - 1) / kWarps;
    ansatz_kernel<<<blocks > 0 ? blocks : 1, kWarps * 32, 0, s>>>(T, alpha, psi, C);
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

int launch_begin(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C,
                 const double *u, const double *alpha_in, int first, NewtonParams np,
                 cudaStream_t s, int learned)
{
    (void)T;
    int blocks = (C + 255) / 256;
    if (blocks > mn->nsm * 8) blocks = mn->nsm * 8;
    {
        LaunchScope ls(mn, PK_BEGIN, s, C);
        KITRT_DISPATCH_N(mn->N, begin_test_kernel<NN><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(S, u, alpha_in, first, np, C, learned));
        if (cudaGetLastError() != cudaSuccess) return KITRT_ECUDA;
    }
    if (first == 1 || learned) return KITRT_OK;
    LaunchScope ls(mn, PK_BEGIN, s, 0);
    KITRT_DISPATCH_N(mn->N, predict_launch<NN>(mn, S, C, u, np, s));
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

// Grid of the FP64 sweep: as many CTAs as are resident on all SMs at once.
int fp64_sweep_grid(const kitrt_mn *mn)
{
    int resident = 1;
    switch (mn->N) {
    case 1: resident = resident_ctas(sweep64_kernel<1>, kSweepThreads, 0, 8); break;
    case 2: resident = resident_ctas(sweep64_kernel<2>, kSweepThreads, 0, 8); break;
    case 3: resident = resident_ctas(sweep64_kernel<3>, kSweepThreads, 0, 8); break;
    case 4: resident = resident_ctas(sweep64_kernel<4>, kSweepThreads, 0, 8); break;
    case 5: resident = resident_ctas(sweep64_kernel<5>, kSweepThreads, 0, 8); break;
    default: break;
    }
    return mn->nsm * resident;
}

int launch_eval_fp64(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C,
                     const double *u, int k, NewtonParams np, cudaStream_t s, bool filter,
                     float *psi32, double *Vacc)
{
    const int grid = grid_for(mn, C, 4);
    LaunchScope ls(mn, PK_EVAL, s, 0);
    if (!Vacc) {
        // fused sweep: no accumulator (the caller may pass a launch-only view without a mesh)
        KITRT_DISPATCH_N(mn->N, (eval_kernel<NN, false, true><<<grid, kWarps * 32, 0, s>>>(T, S, u, k, np, psi32, Vacc, 0)));
    } else if (filter) {
        // cells handed to the FP64 Hessian: whole sums into part 0 of their list slots
        KITRT_DISPATCH_N(mn->N, (eval_kernel<NN, true, false><<<grid, kWarps * 32, 0, s>>>(T, S, u, k, np, psi32, Vacc, mn->vs)));
    } else {
        KITRT_DISPATCH_N(mn->N, (sweep64_kernel<NN><<<mn->grid_fp64, kSweepThreads, 0, s>>>(T, S, k, Vacc, mn->vs, mn->target_fp64)));
    }
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

int launch_finish(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C,
                  double *alpha_out, double *psi, float *psi32, int polish, int compare_prev,
                  cudaStream_t s)
{
    const int grid = grid_for(mn, C, 8);
    LaunchScope ls(mn, PK_FINISH, s, C);
    if (!psi && !psi32) {
        const size_t total = (size_t)C * T.n;
        int blocks = (int)((total + 255) / 256);
        if (blocks > mn->nsm * 8) blocks = mn->nsm * 8;
        finish_alpha_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(S, alpha_out, polish, T.n, C);
        return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
    }
    KITRT_DISPATCH_N(mn->N, finish_kernel<NN><<<grid, kWarps * 32, 0, s>>>(T, S, alpha_out, psi, psi32, polish, compare_prev, C));
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}
