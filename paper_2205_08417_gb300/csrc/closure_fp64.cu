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

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 8;  // warps per block

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

// Warp Cholesky of the n x n matrix in sH (row-major); on success the lower triangle holds L.
template <int n>
__device__ bool warp_cholesky(double *sH, int lane)
{
    for (int j = 0; j < n; ++j) {
        const double djj = sH[j * n + j];
        if (!(djj > 0.0)) return false;  // warp-uniform: every lane read the same value
        const double ljj = sqrt(djj);
        const double rinv = 1.0 / ljj;
        __syncwarp();
        if (lane > j && lane < n) sH[lane * n + j] *= rinv;
        if (lane == j) sH[j * n + j] = ljj;
        __syncwarp();
        if (lane > j && lane < n) {
            const double lij = sH[lane * n + j];
            for (int k = j + 1; k <= lane; ++k) sH[lane * n + k] = fma(-lij, sH[k * n + j], sH[lane * n + k]);
        }
        __syncwarp();
    }
    return true;
}

// Solve L L^T x = b with lane a holding b_a; returns x_a in lane a.
template <int n>
__device__ double warp_chol_solve(const double *sH, double b, int lane)
{
    double y = b;
    for (int j = 0; j < n; ++j) {
        const double yj = __shfl_sync(kFull, y, j) / sH[j * n + j];
        if (lane == j) y = yj;
        if (lane > j && lane < n) y = fma(-sH[lane * n + j], yj, y);
    }
    for (int j = n - 1; j >= 0; --j) {
        const double xj = __shfl_sync(kFull, y, j) / sH[j * n + j];
        if (lane == j) y = xj;
        if (lane < j) y = fma(-sH[j * n + lane], xj, y);
    }
    return lane < n ? y : 0.0;
}

template <int NN>
struct Dims {
    static constexpr int n = (NN + 1) * (NN + 2) / 2;
    static constexpr int n2 = (2 * NN + 1) * (2 * NN + 2) / 2;
    static constexpr int npairs = n * (n + 1) / 2;
};

// ---------------------------------------------------------------------------------------------
// begin: start a closure. first != 0: every cell starts from alpha_in with an evaluation.
// first == 0: the previous closure left alpha_k, its moments U, <exp>, and the Cholesky factor
// of H(alpha_k); with the new u the gradient is U - u, so the first Newton direction needs no
// new quadrature pass (a cell already within tolerance is done at once).
// ---------------------------------------------------------------------------------------------
template <int NN>
__global__ void __launch_bounds__(kWarps * 32)
begin_kernel(Tables T, NewtonState S, const double *__restrict__ u, const double *__restrict__ alpha_in,
             int first, NewtonParams np, int C)
{
    constexpr int n = Dims<NN>::n, npairs = Dims<NN>::npairs;
    __shared__ double sH[kWarps][n * n];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double *H = sH[wib];
    for (int cell = blockIdx.x * kWarps + wib; cell < C; cell += gridDim.x * kWarps) {
        const size_t off = (size_t)cell * n;
        if (lane == 0) {
            S.iters[cell] = 0;
            S.halv[cell] = 0;
            S.evals[cell] = 0;
            S.status[cell] = 0;
        }
        if (first) {
            if (lane < n) S.alpha[off + lane] = alpha_in[off + lane];
            if (lane == 0) S.phase[cell] = PH_INIT;
            push(S.list[0], &S.cnt[0], cell, lane);
            continue;
        }
        const double ua = lane < n ? u[off + lane] : 0.0;
        const double al = lane < n ? S.alpha[off + lane] : 0.0;
        const double g = lane < n ? S.U[off + lane] - ua : 0.0;
        for (int a = lane; a < n; a += 32)
            for (int b = 0; b <= a; ++b) {
                const double v = S.L[(size_t)cell * npairs + tri_idx(a, b)];
                H[a * n + b] = v;
            }
        __syncwarp();
        const double d = warp_chol_solve<n>(H, -g, lane);
        __syncwarp();
        const double gn2 = warp_sum(g * g), un2 = warp_sum(ua * ua);
        if (lane < n) S.dir[off + lane] = d;
        if (sqrt(gn2) <= np.tau * sqrt(un2)) {
            if (lane == 0) S.phase[cell] = PH_DONE;
            continue;
        }
        const double au = warp_sum(al * ua), gd = warp_sum(g * d);
        if (lane == 0) {
            const double fs = S.fsum[cell];
            S.f0[cell] = fs - au;
            S.gd[cell] = gd;
            S.lam[cell] = 1.0;
            S.phase[cell] = PH_NEWTON;
        }
        push(S.list[0], &S.cnt[0], cell, lane);
    }
}

// ---------------------------------------------------------------------------------------------
// eval: one trial point per listed cell (alpha + lam dir, or alpha itself for PH_INIT), then the
// Armijo decision, and on acceptance the Hessian, its Cholesky factor, the convergence test and
// the next Newton direction.
// ---------------------------------------------------------------------------------------------
template <int NN>
__global__ void __launch_bounds__(kWarps * 32)
eval_kernel(Tables T, NewtonState S, const double *__restrict__ u, int k, NewtonParams np)
{
    constexpr int n = Dims<NN>::n, n2 = Dims<NN>::n2, npairs = Dims<NN>::npairs;
    __shared__ double sH[kWarps][n * n];
    __shared__ double sV[kWarps][n2];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int32_t *list_in = S.list[k & 1];
    int32_t *list_out = S.list[(k + 1) & 1];
    const int cnt_in = S.cnt[k % 3];
    int32_t *cnt_out = &S.cnt[(k + 1) % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) S.cnt[(k + 2) % 3] = 0;
    double *H = sH[wib];
    double *Vs = sV[wib];
    const int Qp = T.Qp;
    const double *__restrict__ Mt = T.Mt;
    const double *__restrict__ wq = T.w;

    for (int it = blockIdx.x * kWarps + wib; it < cnt_in; it += gridDim.x * kWarps) {
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
            const double e = wq[q] * exp(z);
#pragma unroll
            for (int c = 0; c < n2; ++c) V[c] = fma(e, Mt[c * Qp + q], V[c]);
        }
        bool finite = true;
#pragma unroll
        for (int c = 0; c < n2; ++c) {
            V[c] = warp_sum(V[c]);
            finite = finite && isfinite(V[c]);
        }
        const double fs = V[0] / T.m0;
        const double au = warp_sum(at * ua);
        const double ft = fs - au;
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
                continue;
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
                fail(S, cell, KITRT_ELINESEARCH, lane);
            } else {
                if (lane == 0) {
                    S.halv[cell] = h;
                    S.lam[cell] = 0.5 * lam;
                }
                push(list_out, cnt_out, cell, lane);
            }
            continue;
        }

        // accepted: store the new point and its moments
        if (lane < n) S.alpha[off + lane] = at;
#pragma unroll
        for (int c = 0; c < n2; ++c)
            if (lane == (c & 31)) Vs[c] = V[c];
        __syncwarp();
        const double Ua = lane < n ? Vs[lane] : 0.0;
        if (lane < n) S.U[off + lane] = Ua;
        if (lane == 0) {
            S.fsum[cell] = fs;
            S.f0[cell] = ft;
        }
        // Hessian from Gaunt coefficients
        for (int p = lane; p < npairs; p += 32) {
            int a = 0;
            while ((a + 1) * (a + 2) / 2 <= p) ++a;
            const int b = p - a * (a + 1) / 2;
            double h = 0.0;
            for (int t = T.gstart[p]; t < T.gstart[p + 1]; ++t) h = fma(T.gcoef[t], Vs[T.gidx[t]], h);
            H[a * n + b] = h;
            H[b * n + a] = h;
        }
        __syncwarp();
        if (!warp_cholesky<n>(H, lane)) {
            fail(S, cell, KITRT_ECHOL, lane);
            __syncwarp();
            continue;
        }
        for (int a = lane; a < n; a += 32)
            for (int b = 0; b <= a; ++b) S.L[(size_t)cell * npairs + tri_idx(a, b)] = H[a * n + b];
        const double g = lane < n ? Ua - ua : 0.0;
        const double d = warp_chol_solve<n>(H, -g, lane);
        __syncwarp();
        const double gn2 = warp_sum(g * g), un2 = warp_sum(ua * ua), gd = warp_sum(g * d);
        if (lane < n) S.dir[off + lane] = d;
        int iters = S.iters[cell];
        if (ph == PH_NEWTON) ++iters;
        if (lane == 0) S.iters[cell] = iters;
        if (sqrt(gn2) <= np.tau * sqrt(un2)) {
            if (lane == 0) S.phase[cell] = PH_DONE;
            continue;
        }
        if (iters >= np.max_iter) {
            fail(S, cell, KITRT_ENOCONVERGE, lane);
            continue;
        }
        if (lane == 0) {
            S.gd[cell] = gd;
            S.lam[cell] = 1.0;
            S.halv[cell] = 0;
            S.phase[cell] = PH_NEWTON;
        }
        push(list_out, cnt_out, cell, lane);
    }
}

// ---------------------------------------------------------------------------------------------
// finish: final alpha (alpha_k plus the polish step if enabled) to the caller, and optionally the
// ansatz psi at every folded point (FP64 and/or FP32).
// ---------------------------------------------------------------------------------------------
template <int NN>
__global__ void __launch_bounds__(kWarps * 32)
finish_kernel(Tables T, NewtonState S, double *__restrict__ alpha_out, double *__restrict__ psi,
              float *__restrict__ psi32, int polish, int C)
{
    constexpr int n = Dims<NN>::n;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int Qp = T.Qp;
    for (int cell = blockIdx.x * kWarps + wib; cell < C; cell += gridDim.x * kWarps) {
        const size_t off = (size_t)cell * n;
        const bool ok = S.status[cell] == 0;
        double a = lane < n ? S.alpha[off + lane] : 0.0;
        if (ok && polish && lane < n) a += S.dir[off + lane];
        if (lane < n) alpha_out[off + lane] = a;
        if (!psi && !psi32) continue;
        double av[n];
#pragma unroll
        for (int b = 0; b < n; ++b) av[b] = __shfl_sync(kFull, a, b);
        for (int q = lane; q < Qp; q += 32) {
            double z = 0.0;
#pragma unroll
            for (int b = 0; b < n; ++b) z = fma(av[b], T.Mt[b * Qp + q], z);
            const double e = exp(z);
            if (psi) psi[(size_t)cell * Qp + q] = e;
            if (psi32) psi32[(size_t)cell * Qp + q] = (float)e;
        }
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
            psi[(size_t)cell * Qf + q] = exp(z);
        }
    }
}

int grid_for(const kitrt_mn *mn, int C, int per_sm)
{
    const int need = (C + kWarps - 1) / kWarps;
    const int cap = mn->nsm * per_sm;
    return need < cap ? (need > 0 ? need : 1) : cap;
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

int launch_ansatz(const Tables &T, int C, const double *alpha, double *psi, cudaStream_t s)
{
    const int blocks = (C + kWarps - 1) / kWarps;
    ansatz_kernel<<<blocks > 0 ? blocks : 1, kWarps * 32, 0, s>>>(T, alpha, psi, C);
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

int launch_begin(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C,
                 const double *u, const double *alpha_in, int first, NewtonParams np,
                 cudaStream_t s)
{
    const int grid = grid_for(mn, C, 8);
    LaunchScope ls(mn, PK_BEGIN, s, C);
    KITRT_DISPATCH_N(mn->N, begin_kernel<NN><<<grid, kWarps * 32, 0, s>>>(T, S, u, alpha_in, first, np, C));
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

int launch_eval_fp64(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C,
                     const double *u, int k, NewtonParams np, cudaStream_t s)
{
    const int grid = grid_for(mn, C, 4);
    LaunchScope ls(mn, PK_EVAL, s, 0);
    KITRT_DISPATCH_N(mn->N, eval_kernel<NN><<<grid, kWarps * 32, 0, s>>>(T, S, u, k, np));
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

int launch_finish(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C,
                  double *alpha_out, double *psi, float *psi32, int polish, cudaStream_t s)
{
    const int grid = grid_for(mn, C, 8);
    LaunchScope ls(mn, PK_FINISH, s, C);
    KITRT_DISPATCH_N(mn->N, finish_kernel<NN><<<grid, kWarps * 32, 0, s>>>(T, S, alpha_out, psi, psi32, polish, C));
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}
