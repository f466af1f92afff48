// Discrete adjoint of the FP64 M_N step, for the gradient of the absorbed energy in a target
// region with respect to per-block absorption and scattering coefficients.
//
// Step map [Sec. 4.2 explicit iteration, Sec. 4.4 kinetic flux, Sec. 3.1 isotropic scattering]:
//   u^{s+1}_i = u^s_i - dt/A_i F_i(psi(alpha(u^s))) + dt R_i(u^s_i),
//   R_i(u) = -sigma_a,i u - sigma_s,i (u - u_0 e_0) + q_i <m>.
// Objective: J = sum_{s<nsteps} dt sum_{i in target} A_i sigma_a,i <psi_i>, <psi_i> = u^s_i0 / m_0.
// Reverse sweep with lambda^{nsteps} = 0:
//   lambda^s_i = lambda^{s+1}_i + dt (-sigma_t,i lambda_i + sigma_s,i lambda_i0 e_0)
//              + H_i^-1 sum_q mu_iq psi_iq m_q + [i in target] dt A_i sigma_a,i / m_0 e_0,
// where d psi_iq / d u_i = psi_iq m_q^T H_i^-1 (implicit-function theorem on the closure, H the
// Hessian of the dual at the converged alpha) and mu_iq = d(sum_c lambda_c . u^{s+1}_c)/d psi_iq
// is the transposed upwind flux, gathered per cell from its own and its neighbours' lambda:
//   mu_iq = -dt w_q [ (L_iq/A_i) sum_f (Omega_q.n_if)(H_f + [Neumann boundary f](1 - H_f))
//                     - sum_{f interior} (L_jq/A_j) (Omega_q.n_if) H_f ],  L_cq = lambda_c . m_q,
// H_f = [Omega_q.n_if > 0]. Parameter gradients per block accumulate
//   dJ/dsigma_a += -dt lambda^{s+1}_i . u^s_i + [i in target] dt A_i u^s_i0 / m_0,
//   dJ/dsigma_s += -dt lambda^{s+1}_i . (u^s_i - u^s_i0 e_0).
// Memory: forward states are checkpointed every `ckpt_every` steps; each segment is recomputed
// forward (storing its alphas) before its reverse steps.
#include <math.h>
#include <string.h>

#include <vector>

#include "kexp.cuh"
#include "kitrt_internal.cuh"
#include "newton_common.cuh"

namespace {

using namespace kitrt_dev;
constexpr int kWarps = 8;

__global__ void objective_kernel(const double *__restrict__ u, int n, const double *__restrict__ sa,
                                 const uint8_t *__restrict__ target, const double *__restrict__ area,
                                 double dt, double inv_m0, int C, double *__restrict__ J)
{
    double part = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x)
        if (target[i]) part += dt * area[i] * sa[i] * u[(size_t)i * n] * inv_m0;
    part = warp_sum(part);
    if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(J, part);
}

// L_cq = lambda_c . m_q at every folded point.
__global__ void lambda_dot_m_kernel(Tables T, const double *__restrict__ lam, double *__restrict__ Lq, int C)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int n = T.n, Qp = T.Qp;
    for (int c = blockIdx.x * kWarps + wib; c < C; c += gridDim.x * kWarps) {
        double l[KITRT_MAX_NMOM];
        for (int a = 0; a < n; ++a) l[a] = lam[(size_t)c * n + a];
        for (int q = lane; q < Qp; q += 32) {
            double s = 0.0;
            for (int a = 0; a < n; ++a) s = fma(l[a], T.Mt[a * Qp + q], s);
            Lq[(size_t)c * Qp + q] = s;
        }
    }
}

template <int NN>
__global__ void __launch_bounds__(kWarps * 32)
adjoint_cell_kernel(Tables T, const int4 *__restrict__ nbr, const double *__restrict__ nrm,
                    const double *__restrict__ area, const double *__restrict__ u,
                    const double *__restrict__ alpha, const double *__restrict__ lam_next,
                    const double *__restrict__ Lq, const double *__restrict__ sa,
                    const double *__restrict__ ss, const uint8_t *__restrict__ target,
                    const int32_t *__restrict__ block, double dt, int bc, int C,
                    double *__restrict__ lam, double *__restrict__ gsa, double *__restrict__ gss,
                    int32_t *__restrict__ fail)
{
    constexpr int n = Dims<NN>::n, n2 = Dims<NN>::n2, npairs = Dims<NN>::npairs;
    __shared__ double sH[kWarps][n * n];
    __shared__ double sV[kWarps][n2];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int Qp = T.Qp;
    double *H = sH[wib], *Vs = sV[wib];
    for (int i = blockIdx.x * kWarps + wib; i < C; i += gridDim.x * kWarps) {
        const size_t off = (size_t)i * n;
        const int4 nb = nbr[i];
        const int js[3] = {nb.x, nb.y, nb.z};
        double nx[3], ny[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            nx[f] = nrm[6 * (size_t)i + 2 * f];
            ny[f] = nrm[6 * (size_t)i + 2 * f + 1];
        }
        const double inv_Ai = 1.0 / area[i];
        double inv_Aj[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) inv_Aj[f] = js[f] >= 0 ? 1.0 / area[js[f]] : 0.0;
        const double al = lane < n ? alpha[off + lane] : 0.0;
        double av[n];
#pragma unroll
        for (int a = 0; a < n; ++a) av[a] = __shfl_sync(kFull, al, a);
        double V[n2], r[n];
#pragma unroll
        for (int c = 0; c < n2; ++c) V[c] = 0.0;
#pragma unroll
        for (int a = 0; a < n; ++a) r[a] = 0.0;
        for (int q = lane; q < Qp; q += 32) {
            double z = 0.0;
#pragma unroll
            for (int a = 0; a < n; ++a) z = fma(av[a], T.Mt[a * Qp + q], z);
            const double psi = kexp(z, T.exptab);
            const double e = T.w[q] * psi;
#pragma unroll
            for (int c = 0; c < n2; ++c) V[c] = fma(e, T.Mt[c * Qp + q], V[c]);
            const double Li = Lq[(size_t)i * Qp + q];
            double acc = 0.0;
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const double d = fma(T.wox[q], nx[f], T.woy[q] * ny[f]);  // w_q Omega_q . n_if
                if (d > 0.0) {
                    acc = fma(Li * inv_Ai, d, acc);
                    if (js[f] >= 0) acc = fma(-Lq[(size_t)js[f] * Qp + q] * inv_Aj[f], d, acc);
                } else if (js[f] < 0 && bc == 0) {
                    acc = fma(Li * inv_Ai, d, acc);
                }
            }
            const double t = -dt * acc * psi;  // mu_iq psi_iq
#pragma unroll
            for (int a = 0; a < n; ++a) r[a] = fma(t, T.Mt[a * Qp + q], r[a]);
        }
#pragma unroll
        for (int c = 0; c < n2; ++c) V[c] = warp_sum(V[c]);
        double ra = 0.0;
#pragma unroll
        for (int a = 0; a < n; ++a) {
            const double v = warp_sum(r[a]);
            if (lane == a) ra = v;
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < n2; ++c)
            if (lane == (c & 31)) Vs[c] = V[c];
        __syncwarp();
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
        double x = 0.0;
        if (warp_cholesky<n>(H, lane)) {
            x = warp_chol_solve<n>(H, ra, lane);
        } else if (lane == 0) {
            atomicAdd(fail, 1);
        }
        __syncwarp();
        const double li = lane < n ? lam_next[off + lane] : 0.0;
        const double l0 = __shfl_sync(kFull, li, 0);
        const double ua = lane < n ? u[off + lane] : 0.0;
        const double u0 = __shfl_sync(kFull, ua, 0);
        const double sai = sa[i], ssi = ss[i];
        const bool tgt = target[i] != 0;
        if (lane < n) {
            double v = li + dt * (-(sai + ssi) * li + (lane == 0 ? ssi * l0 : 0.0)) + x;
            if (lane == 0 && tgt) v += dt * area[i] * sai / T.m0;
            lam[off + lane] = v;
        }
        const double lu = warp_sum(li * ua);
        const double lus = warp_sum(li * (ua - (lane == 0 ? u0 : 0.0)));
        if (lane == 0) {
            const int b = block[i];
            atomicAdd(&gsa[b], -dt * lu + (tgt ? dt * area[i] * u0 / T.m0 : 0.0));
            atomicAdd(&gss[b], -dt * lus);
        }
    }
}

}  // namespace

// Device-side step used by the adjoint: closure (FP64, warm start), finish (alpha_out), flux.
// Declared in host.cu.
int kitrt_internal_step(kitrt_mn *mn, double *u, double *alpha, const double *sa, const double *ss,
                        const double *q, double dt, int first, cudaStream_t s);
int check_stability(kitrt_mn *mn, const double *sa, const double *ss, double dt, cudaStream_t s,
                    bool wait);

extern "C" int32_t kitrt_adjoint(kitrt_mn *mn, const double *u0, const double *alpha0,
                                 const double *sigma_a, const double *sigma_s, const double *q,
                                 const int32_t *block_of_cell, int32_t nblocks, const uint8_t *target,
                                 double dt, int32_t nsteps, int32_t ckpt_every, double *J,
                                 double *dJ_dsa, double *dJ_dss, void *stream)
{
    if (!mn || !u0 || !alpha0 || !sigma_a || !sigma_s || !q || !block_of_cell || !target || !J ||
        !dJ_dsa || !dJ_dss || nblocks < 1 || nsteps < 0 || ckpt_every < 1 || mn->p.mode != KITRT_FP64 ||
        mn->p.order != 1 || mn->p.reg_gamma != 0.0 || mn->d_invrho)
        return KITRT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int C = mn->mesh->C, n = mn->n, Qp = mn->Qp;
    if (dt <= 0.0) dt = mn->p.cfl * mn->mesh->min_inradius;
    const size_t Cn = (size_t)C * n;
    const int nck = (nsteps + ckpt_every - 1) / ckpt_every;
    // the adjoint's buffers live in the solver's workspace: allocated by the first call that
    // needs them (or needs more than the last), kept for later calls, freed by kitrt_mn_destroy
    const size_t a256 = 255;
    const size_t sizes[] = {sizeof(double) * Cn * (nck > 0 ? nck : 1),  // ck_u
                            sizeof(double) * Cn * (nck > 0 ? nck : 1),  // ck_a
                            sizeof(double) * Cn * ckpt_every,           // seg_u
                            sizeof(double) * Cn * ckpt_every,           // seg_a
                            sizeof(double) * Cn, sizeof(double) * Cn,   // u, a
                            sizeof(double) * Cn, sizeof(double) * Cn,   // lam, lam2
                            sizeof(double) * (size_t)C * Qp,            // Lq
                            sizeof(double) * (1 + 2 * (size_t)nblocks), // J, dJ_dsa, dJ_dss
                            sizeof(int32_t)};                           // fail
    constexpr int kBufs = sizeof(sizes) / sizeof(sizes[0]);
    size_t offs[kBufs], total = 0;
    for (int i = 0; i < kBufs; ++i) {
        offs[i] = total;
        total += (sizes[i] + a256) & ~a256;
    }
    if (mn->adj_bytes < total) {
        if (mn->d_adj) cudaFree(mn->d_adj);
        mn->d_adj = nullptr;
        mn->adj_bytes = 0;
        if (cudaMalloc(&mn->d_adj, total) != cudaSuccess) {
            mn->d_adj = nullptr;
            return KITRT_ENOMEM;
        }
        mn->adj_bytes = total;
    }
    unsigned char *base = (unsigned char *)mn->d_adj;
    double *ck_u = (double *)(base + offs[0]);
    double *ck_a = (double *)(base + offs[1]);
    double *seg_u = (double *)(base + offs[2]);
    double *seg_a = (double *)(base + offs[3]);
    double *u = (double *)(base + offs[4]);
    double *a = (double *)(base + offs[5]);
    double *lam = (double *)(base + offs[6]);
    double *lam2 = (double *)(base + offs[7]);
    double *Lq = (double *)(base + offs[8]);
    double *dJ = (double *)(base + offs[9]);  // J, then dJ/dsigma_a, then dJ/dsigma_s
    double *dJ_sa = dJ + 1, *dJ_ss = dJ + 1 + nblocks;
    int32_t *fail = (int32_t *)(base + offs[10]);
    auto cleanup = [](int rc) { return rc; };
    int rc0 = check_stability(mn, sigma_a, sigma_s, dt, s, true);
    if (rc0) return rc0;
    const Tables T = mn->tables();
    const kitrt_mesh *m = mn->mesh;
    const double inv_m0 = 1.0 / T.m0;
    const int tb = (C + 255) / 256 < mn->nsm * 8 ? (C + 255) / 256 : mn->nsm * 8;
    const int wb = (C + kWarps - 1) / kWarps < mn->nsm * 8 ? (C + kWarps - 1) / kWarps : mn->nsm * 8;
#define CK(x)                                          \
    do {                                               \
        if ((x) != cudaSuccess) return cleanup(KITRT_ECUDA); \
    } while (0)
    CK(cudaMemsetAsync(dJ, 0, sizeof(double) * (1 + 2 * (size_t)nblocks), s));
    CK(cudaMemsetAsync(fail, 0, sizeof(int32_t), s));
    CK(cudaMemcpyAsync(u, u0, sizeof(double) * Cn, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(a, alpha0, sizeof(double) * Cn, cudaMemcpyDeviceToDevice, s));
    // forward sweep: objective and checkpoints (state and warm start at each segment start)
    for (int st = 0; st < nsteps; ++st) {
        if (st % ckpt_every == 0) {
            CK(cudaMemcpyAsync(ck_u + Cn * (st / ckpt_every), u, sizeof(double) * Cn, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(ck_a + Cn * (st / ckpt_every), a, sizeof(double) * Cn, cudaMemcpyDeviceToDevice, s));
        }
        {
            LaunchScope ls(mn, PK_ADJOINT, s, C);
            objective_kernel<<<tb, 256, 0, s>>>(u, n, sigma_a, target, m->d_area, dt, inv_m0, C, dJ);
        }
        const int rc = kitrt_internal_step(mn, u, a, sigma_a, sigma_s, q, dt, st == 0, s);
        if (rc) return cleanup(rc);
    }
    // reverse sweep, segment by segment
    CK(cudaMemsetAsync(lam, 0, sizeof(double) * Cn, s));
    for (int seg = nck - 1; seg >= 0; --seg) {
        const int s0 = seg * ckpt_every, s1 = (s0 + ckpt_every < nsteps) ? s0 + ckpt_every : nsteps;
        CK(cudaMemcpyAsync(u, ck_u + Cn * seg, sizeof(double) * Cn, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(a, ck_a + Cn * seg, sizeof(double) * Cn, cudaMemcpyDeviceToDevice, s));
        for (int st = s0; st < s1; ++st) {
            CK(cudaMemcpyAsync(seg_u + Cn * (st - s0), u, sizeof(double) * Cn, cudaMemcpyDeviceToDevice, s));
            const int rc = kitrt_internal_step(mn, u, a, sigma_a, sigma_s, q, dt, st == s0, s);
            if (rc) return cleanup(rc);
            // a holds the converged alpha of u^st after the step
            CK(cudaMemcpyAsync(seg_a + Cn * (st - s0), a, sizeof(double) * Cn, cudaMemcpyDeviceToDevice, s));
        }
        for (int st = s1 - 1; st >= s0; --st) {
            LaunchScope ls(mn, PK_ADJOINT, s, C);
            lambda_dot_m_kernel<<<wb, kWarps * 32, 0, s>>>(T, lam, Lq, C);
#define ADJ_CASE(NNv)                                                                                       \
    case NNv:                                                                                               \
        adjoint_cell_kernel<NNv><<<wb, kWarps * 32, 0, s>>>(T, m->d_nbr, m->d_nrm, m->d_area,               \
                                                            seg_u + Cn * (st - s0), seg_a + Cn * (st - s0), \
                                                            lam, Lq, sigma_a, sigma_s, target,              \
                                                            block_of_cell, dt, mn->p.bc, C, lam2, dJ_sa,    \
                                                            dJ_ss, fail);                                   \
        break;
            switch (mn->N) {
                ADJ_CASE(1)
                ADJ_CASE(2)
                ADJ_CASE(3)
                ADJ_CASE(4)
                ADJ_CASE(5)
            default: return cleanup(KITRT_EINVAL);
            }
#undef ADJ_CASE
            CK(cudaGetLastError());
            double *t = lam;
            lam = lam2;
            lam2 = t;
        }
    }
    int32_t nf = 0;
    CK(cudaMemcpyAsync(&nf, fail, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(J, dJ, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(dJ_dsa, dJ_sa, sizeof(double) * nblocks, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(dJ_dss, dJ_ss, sizeof(double) * nblocks, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
#undef CK
    return cleanup(nf ? KITRT_ECHOL : KITRT_OK);
}
