// Learned entropy closure: the MLP's alpha_{1..n-1}, the exact mass constraint for alpha_0, the
// FP64 moment-residual test and the hand-over of failing cells to Newton; plus the generator of
// training moments (von Mises-Fisher mixtures integrated with the solver's own quadrature).
//
// Mass constraint [Sec. 3.1: the ansatz must reproduce u; its zeroth moment is the particle
// density]: with z'_q = sum_{a>=1} alpha_a m_a(q) and U'_a = sum_q w_q exp(z'_q) m_a(q), the
// choice exp(alpha_0 m_0) = u_0 / U'_0 makes the zeroth moment of exp(alpha.m) equal to u_0, and
// every other moment is U_a = (u_0 / U'_0) U'_a. The cell keeps the network's answer when
// ||U - u||_2 <= fallback_tol ||u||_2 (computed in FP64); otherwise Newton starts from the better
// (by dual objective) of that point and the previous closure's, the latter with a step from its
// stored factor when the cell has one.
#include <cuda_bf16.h>
#include <math.h>

#include "kexp.cuh"
#include "kitrt_internal.cuh"
#include "newton_common.cuh"

namespace {

using namespace kitrt_dev;
constexpr int kWarps = 8;

template <int NN>
__global__ void __launch_bounds__(kWarps * 32)
learned_pass_kernel(Tables T, NewtonState S, const double *__restrict__ u,
                    const double *__restrict__ alpha_nn, double tol, float *__restrict__ psi32,
                    int first)
{
    constexpr int n = Dims<NN>::n, npairs = Dims<NN>::npairs;
    __shared__ double sH[kWarps][n * n];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int Qp = T.Qp;
    const int count = S.cnt[8];
    for (int it = blockIdx.x * kWarps + wib; it < count; it += gridDim.x * kWarps) {
        const int cell = S.list[1][it];
        const size_t off = (size_t)cell * n;
        const double ua = lane < n ? u[off + lane] : 0.0;
        const double al = (lane >= 1 && lane < n) ? alpha_nn[off + lane] : 0.0;
        double atv[n];
#pragma unroll
        for (int a = 0; a < n; ++a) atv[a] = __shfl_sync(kFull, al, a);
        double Up[n];
#pragma unroll
        for (int a = 0; a < n; ++a) Up[a] = 0.0;
        for (int q = lane; q < Qp; q += 32) {
            double z = 0.0;
#pragma unroll
            for (int a = 1; a < n; ++a) z = fma(atv[a], T.Mt[a * Qp + q], z);
            const double ez = kexp(z, T.exptab);
            if (psi32) psi32[(size_t)cell * Qp + q] = exp_to_float(ez);
            const double e = T.w[q] * ez;
#pragma unroll
            for (int a = 0; a < n; ++a) Up[a] = fma(e, T.Mt[a * Qp + q], Up[a]);
        }
        double Ua = 0.0;
#pragma unroll
        for (int a = 0; a < n; ++a) {
            const double v = warp_sum(Up[a]);
            if (lane == a) Ua = v;
        }
        const double u0 = __shfl_sync(kFull, ua, 0), U0p = __shfl_sync(kFull, Ua, 0);
        const double c = u0 / U0p;                // exp(alpha_0 m_0)
        const double alpha0 = log(c) / T.m0;
        const double U = c * Ua;                  // moments of the mass-corrected ansatz
        const double r = (lane >= 1 && lane < n) ? U - ua : 0.0;
        const double r2 = warp_sum(r * r), un2 = warp_sum(ua * ua);
        // dual objective of the network's point: <exp(alpha.m)> = u_0 / m_0 after the mass fix
        const double f_nn = u0 / T.m0 - (alpha0 * u0 + warp_sum(al * ua));
        if (lane == 0) atomicAdd(&S.cnt[10], 1);  // a quadrature pass of this cell (the network's)
        const bool finite = isfinite(alpha0) && isfinite(r2) && isfinite(f_nn) && u0 > 0.0;
        const bool ok = finite && r2 <= tol * tol * un2;
        if (ok) {
            if (lane == 0) S.alpha[off] = alpha0;
            if (lane >= 1 && lane < n) S.alpha[off + lane] = al;
            if (lane < n) S.U[off + lane] = lane == 0 ? u0 : U;
            if (lane == 0) {
                S.fsum[cell] = u0 / T.m0;
                S.phase[cell] = PH_DONE;
            }
            if (psi32) {
                const float cf = (float)c;
                for (int q = lane; q < Qp; q += 32) psi32[(size_t)cell * Qp + q] *= cf;
            }
        } else {
            // Newton starts from the better of the network's point and the cell's previous alpha
            // (its objective needs no quadrature: <exp> of the previous point is stored)
            bool use_nn = finite;
            if (first != 1 && finite) {
                const double ap = lane < n ? S.alpha[off + lane] : 0.0;
                const double f_prev = S.fsum[cell] - warp_sum(ap * ua);
                use_nn = !(isfinite(f_prev) && f_prev <= f_nn);
            }
            if (use_nn) {
                if (lane == 0) S.alpha[off] = alpha0;
                if (lane >= 1 && lane < n) S.alpha[off + lane] = al;
            }
            if (!use_nn && first != 1 && S.lfac && S.lfac[cell]) {
                // the previous closure's point is the better start, and its moments and a
                // factor of this cell are stored: take the Newton step from them at once, as the
                // predictor of the other modes does, instead of evaluating that point again
                double *H = sH[wib];
                const double ap = lane < n ? S.alpha[off + lane] : 0.0;
                const double g = lane < n ? S.U[off + lane] - ua : 0.0;
                for (int a = lane; a < n; a += 32)
                    for (int b = 0; b <= a; ++b) H[a * n + b] = S.L[(size_t)cell * npairs + tri_idx(a, b)];
                __syncwarp();
                const double d = warp_chol_solve<n>(H, -g, lane);
                __syncwarp();
                const double gn2 = warp_sum(g * g), au = warp_sum(ap * ua), gd = warp_sum(g * d);
                if (lane < n) S.dir[off + lane] = d;
                if (lane == 0) {
                    if (S.gnorm) S.gnorm[cell] = sqrt(gn2);
                    S.f0[cell] = S.fsum[cell] - au;
                    S.gd[cell] = gd;
                    S.lam[cell] = 1.0;
                    S.phase[cell] = PH_NEWTON;
                    atomicAdd(&S.cnt[5], 1);
                    atomicAdd(&S.cnt[9], 1);  // a step from the stored factor
                }
            } else if (lane == 0) {
                S.phase[cell] = PH_INIT;
                atomicAdd(&S.cnt[5], 1);
            }
            push(S.list[0], &S.cnt[0], cell, lane);
        }
    }
}

// Moments of mixtures of von Mises-Fisher densities on S^2 on the folded rule: each folded point
// stands for the pair (Omega_2D, +-mu), and the basis is even in mu, so the pair contributes
// w/2 (f(mu) + f(-mu)) m. f(x) = sum_l weight_l kappa_l / (2 pi (1 - exp(-2 kappa_l)))
// exp(kappa_l (c_l . x - 1)). One warp per sample.
__global__ void vmf_moments_kernel(Tables T, const double *__restrict__ centres, const double *__restrict__ kappa,
                                   const double *__restrict__ weight, int lobes, int count,
                                   double *__restrict__ uout)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int n = T.n, Qp = T.Qp;
    for (int s = blockIdx.x * kWarps + wib; s < count; s += gridDim.x * kWarps) {
        double acc[21];
        for (int a = 0; a < n; ++a) acc[a] = 0.0;
        for (int q = lane; q < T.Qf; q += 32) {
            const double wx = T.wox[q], wy = T.woy[q], w = T.w[q];
            const double ox = w > 0 ? wx / w : 0.0, oy = w > 0 ? wy / w : 0.0;
            const double mu = sqrt(fmax(0.0, 1.0 - ox * ox - oy * oy));
            double f = 0.0;
            for (int l = 0; l < lobes; ++l) {
                const double *cc = centres + ((size_t)s * lobes + l) * 3;
                const double k = kappa[(size_t)s * lobes + l], wt = weight[(size_t)s * lobes + l];
                if (wt == 0.0) continue;
                const double nrm = k / (2.0 * 3.14159265358979323846 * (1.0 - exp(-2.0 * k)));
                const double dp = cc[0] * ox + cc[1] * oy;
                f += wt * nrm * 0.5 * (exp(k * (dp + cc[2] * mu - 1.0)) + exp(k * (dp - cc[2] * mu - 1.0)));
            }
            for (int a = 0; a < n; ++a) acc[a] = fma(w * f, T.Mt[a * Qp + q], acc[a]);
        }
        for (int a = 0; a < n; ++a) {
            const double v = warp_sum(acc[a]);
            if (lane == 0) uout[(size_t)s * n + a] = v;
        }
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, int P)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x)
        y[k] = __float2bfloat16_rn(x[k]);
}

}  // namespace

int launch_learned_pass(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C, const double *u,
                        float *psi32, int first, cudaStream_t s)
{
    int need = (C + kWarps - 1) / kWarps;
    const int cap = mn->nsm * 8;
    const int grid = need < cap ? (need > 0 ? need : 1) : cap;
    LaunchScope ls(mn, PK_MLP, s, 0);
#define LP_CASE(NNv)                                                                               \
    case NNv:                                                                                      \
        learned_pass_kernel<NNv><<<grid, kWarps * 32, 0, s>>>(T, S, u, mn->d_alpha_nn, mn->p.fallback_tol, \
                                                              psi32, first);                           \
        break;
    switch (mn->N) {
        LP_CASE(1)
        LP_CASE(2)
        LP_CASE(3)
        LP_CASE(4)
        LP_CASE(5)
    default: return KITRT_EINVAL;
    }
#undef LP_CASE
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

extern "C" {

int32_t kitrt_mn_set_mlp(kitrt_mn *mn, const float *params, const float *norm, int32_t hidden, void *stream)
{
    if (!mn || !params || !norm || hidden != 64) return KITRT_EINVAL;
    const int dio = mn->n - 1;
    const int P = kitrt_mlp_param_count(dio, hidden, dio);
    cudaStream_t s = (cudaStream_t)stream;
    if (!mn->d_mlp16) {
        if (cudaMalloc(&mn->d_mlp16, sizeof(uint16_t) * P) != cudaSuccess) return KITRT_ENOMEM;
        mn->allocs.push_back(mn->d_mlp16);
        if (cudaMalloc(&mn->d_mlp_norm, sizeof(float) * 4 * dio) != cudaSuccess) return KITRT_ENOMEM;
        mn->allocs.push_back(mn->d_mlp_norm);
    }
    to_bf16_kernel<<<(P + 255) / 256, 256, 0, s>>>(params, (__nv_bfloat16 *)mn->d_mlp16, P);
    if (cudaMemcpyAsync(mn->d_mlp_norm, norm, sizeof(float) * 4 * dio, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return KITRT_ECUDA;
    mn->has_mlp = true;
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

int32_t kitrt_vmf_moments(kitrt_mn *mn, const double *centres, const double *kappa, const double *weight,
                          int32_t lobes, int32_t count, double *u, void *stream)
{
    if (!mn || !centres || !kappa || !weight || !u || lobes < 1 || count < 0) return KITRT_EINVAL;
    if (count == 0) return KITRT_OK;
    int blocks = (count + kWarps - 1) / kWarps;
    if (blocks > mn->nsm * 16) blocks = mn->nsm * 16;
    vmf_moments_kernel<<<blocks, kWarps * 32, 0, (cudaStream_t)stream>>>(mn->tables(), centres, kappa, weight, lobes,
                                                                         count, u);
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

}  // extern "C"
