// Kinetic upwind flux of the closed ansatz and the explicit first-order update
// [Sec. 4.4 kinetic numerical flux; Sec. 4.2 explicit iteration; Sec. 3.1 isotropic scattering].
//
// Cell-centric gather: one warp per cell i, lanes over the folded quadrature points. The upwind
// flux sum_f sum_q w_q m_q (Omega_q.n_f) psi_up is evaluated in its fluctuation form
//     F_i = sum_f sum_{q: Omega_q.n_f < 0} w_q m_q (Omega_q.n_f) (psi_up,f,q - psi_iq),
// which equals it exactly in exact arithmetic because the scaled normals of a closed cell sum to
// zero (sum_f n_f = 0), so psi_iq sum_f Omega_q.n_f vanishes: outflow directions drop out, the
// upwind value is the neighbour's psi (the ghost: psi_iq for Neumann, 0 for vacuum), and a
// uniform state gives exactly zero flux at any working precision. F is projected on the basis,
// warp-reduced, and u <- u - dt/A F + dt R(u) is applied in place (the flux reads psi only).
// psi rows are contiguous per cell, so each face gather is a coalesced row segment.
#include <string.h>

#include "kitrt_internal.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 8;
constexpr int kBatch = 4;     // cells per warp batch in the FP32 flux
constexpr int kTogether = 2;  // cells of a batch whose points one pass over the tables serves

template <int NN, typename PsiT>
__global__ void __launch_bounds__(kWarps * 32)
flux_update_kernel(Tables T, const int4 *__restrict__ nbr, const double *__restrict__ nrm,
                   const double *__restrict__ area, const PsiT *__restrict__ psi,
                   double *__restrict__ u, const double *__restrict__ sa,
                   const double *__restrict__ ss, const double *__restrict__ qs, double dt,
                   int bc, int C)
{
    constexpr int n = (NN + 1) * (NN + 2) / 2;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int Qp = T.Qp;
    for (int i = blockIdx.x * kWarps + wib; i < C; i += gridDim.x * kWarps) {
        const int4 nb = nbr[i];
        const double nx0 = nrm[6 * (size_t)i], ny0 = nrm[6 * (size_t)i + 1];
        const double nx1 = nrm[6 * (size_t)i + 2], ny1 = nrm[6 * (size_t)i + 3];
        const double nx2 = nrm[6 * (size_t)i + 4], ny2 = nrm[6 * (size_t)i + 5];
        const PsiT *pi_row = psi + (size_t)i * Qp;
        double F[n];
#pragma unroll
        for (int a = 0; a < n; ++a) F[a] = 0.0;
        for (int q = lane; q < Qp; q += 32) {
            const double pi = (double)pi_row[q];
            const double wx = T.wox[q], wy = T.woy[q];
            const double ghost = bc == 0 ? pi : 0.0;
            double s = 0.0;
            {
                const double d = fma(wx, nx0, wy * ny0);
                if (d < 0.0) s = fma(d, (nb.x >= 0 ? (double)psi[(size_t)nb.x * Qp + q] : ghost) - pi, s);
            }
            {
                const double d = fma(wx, nx1, wy * ny1);
                if (d < 0.0) s = fma(d, (nb.y >= 0 ? (double)psi[(size_t)nb.y * Qp + q] : ghost) - pi, s);
            }
            {
                const double d = fma(wx, nx2, wy * ny2);
                if (d < 0.0) s = fma(d, (nb.z >= 0 ? (double)psi[(size_t)nb.z * Qp + q] : ghost) - pi, s);
            }
#pragma unroll
            for (int a = 0; a < n; ++a) F[a] = fma(T.Mt[a * Qp + q], s, F[a]);
        }
#pragma unroll
        for (int a = 0; a < n; ++a) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) F[a] += __shfl_xor_sync(kFull, F[a], o);
        }
        double Fa = 0.0;
#pragma unroll
        for (int a = 0; a < n; ++a)
            if (lane == a) Fa = F[a];
        const double u0 = u[(size_t)i * n];
        if (lane < n) {
            const double ua = u[(size_t)i * n + lane];
            const double R = -sa[i] * ua - ss[i] * (ua - (lane == 0 ? u0 : 0.0)) + qs[i] * T.mbar[lane];
            u[(size_t)i * n + lane] = ua - dt / area[i] * Fa + dt * R;
        }
    }
}

// FP32 variant for the mixed modes: FP32 ansatz and upwind sums, Kahan-compensated FP32
// projection per lane, a compensated (two-sum) FP32 reduce-scatter across the warp, and the FP64
// update applied afterwards with every lane busy. A warp takes a batch of kBatch consecutive cells:
// their flux moments go to shared memory, then the warp updates all (cell, moment) pairs of the
// batch (FP64 instructions on a partly idle warp cost as much as on a full one).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// Compensated reduce-scatter of n per-lane sums (F - Fc) across the warp. The sums are padded to
// S slots (the next power of two >= n). At each of the log2(S) halving levels (offsets 16, 8, ...)
// a lane keeps one half of its slots, sends the other half to its partner and adds the partner's
// copy of the kept half with a two-sum; the remaining levels are compensated butterflies between
// lanes holding the same slot. Lane L ends with the total of slot L >> (5 - log2 S) (value s + e);
// every lane whose low 5 - log2 S bits are zero holds a distinct slot. That is S - 1 two-sums per
// lane (plus 5 - log2 S for the butterflies) instead of 5 n for a butterfly per sum.
template <int n>
__device__ __forceinline__ int warp_reduce_scatter(const float (&F)[n], const float (&Fc)[n], int lane,
                                                   float &rs, float &re)
{
    constexpr int S = n <= 1 ? 1 : n <= 2 ? 2 : n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : 32;
    constexpr int H = S == 1 ? 0 : S == 2 ? 1 : S == 4 ? 2 : S == 8 ? 3 : S == 16 ? 4 : 5;
    float sv[S], ev[S];
#pragma unroll
    for (int k = 0; k < S; ++k) {
        sv[k] = k < n ? F[k < n ? k : 0] : 0.0f;
        ev[k] = k < n ? -Fc[k < n ? k : 0] : 0.0f;
    }
#pragma unroll
    for (int lvl = 0; lvl < H; ++lvl) {
        const int o = 16 >> lvl;
        const int half = S >> (lvl + 1);
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const float ks = upper ? sv[k + half] : sv[k], ke = upper ? ev[k + half] : ev[k];
            const float xs = upper ? sv[k] : sv[k + half], xe = upper ? ev[k] : ev[k + half];
            const float ps = __shfl_xor_sync(kFull, xs, o), pe = __shfl_xor_sync(kFull, xe, o);
            float t, e;
            two_sum(ks, ps, t, e);
            sv[k] = t;
            ev[k] = ke + pe + e;
        }
    }
    float s0 = sv[0], e0 = ev[0];
#pragma unroll
    for (int o = 16 >> H; o > 0; o >>= 1) {
        const float so = __shfl_xor_sync(kFull, s0, o), eo = __shfl_xor_sync(kFull, e0, o);
        float t, e;
        two_sum(s0, so, t, e);
        s0 = t;
        e0 = e0 + eo + e;
    }
    rs = s0;
    re = e0;
    // the lane's slot, or -1 for a lane that only duplicates another's slot
    return (lane & ((1 << (5 - H)) - 1)) == 0 ? lane >> (5 - H) : -1;
}

// The FP32 flux of the mixed modes. FP64 instructions are rare on this GPU (2 per clock per SM), so
// none is spent on warp-uniform values: normals and inverse areas come from the mesh's FP32
// copies, the per-cell coefficients are converted by different lanes at once, and the update
// increment dt (-F/A + R(u)) is formed in FP32; only u += increment is FP64 (lanes over the
// (cell, moment) elements of a batch). Each lane sums its ~Q'/32 points in plain FP32; the warp
// reduction of the 32 lane sums is compensated.
template <int NN>
__global__ void __launch_bounds__(kWarps * 32)
flux_update32_kernel(Tables T, const int4 *__restrict__ nbr, const float *__restrict__ nrm32,
                     const float *__restrict__ inva32, const float *__restrict__ psi,
                     double *__restrict__ u, const double *__restrict__ sa,
                     const double *__restrict__ ss, const double *__restrict__ qs, float dt,
                     int bc, int C)
{
    constexpr int n = (NN + 1) * (NN + 2) / 2;
    __shared__ float sF[kWarps][kBatch * n];
    __shared__ float sK[kWarps][kBatch][4];  // per cell: sigma_a, sigma_s, q, 1/A (FP32)
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int Qp = T.Qp;
    for (int base = (blockIdx.x * kWarps + wib) * kBatch; base < C; base += gridDim.x * kWarps * kBatch) {
        const int nb_cells = C - base < kBatch ? C - base : kBatch;
        if (lane < 4 * nb_cells) {
            const int ci = lane >> 2, which = lane & 3, i = base + ci;
            const double v = which == 0 ? sa[i] : which == 1 ? ss[i] : qs[i];
            sK[wib][ci][which] = which == 3 ? inva32[i] : (float)v;
        }
        // kTogether cells at a time share each point's table loads (directions, weights, basis)
        for (int c0 = 0; c0 < nb_cells; c0 += kTogether) {
            int4 nb[kTogether];
            float nx[kTogether][3], ny[kTogether][3], g[kTogether][3];
            const float *own[kTogether], *up[kTogether][3];
#pragma unroll
            for (int t = 0; t < kTogether; ++t) {
                // a missing partner cell repeats the last real one; its sums are not stored
                const int i = base + min(c0 + t, nb_cells - 1);
                nb[t] = nbr[i];
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    nx[t][f] = nrm32[6 * (size_t)i + 2 * f];
                    ny[t][f] = nrm32[6 * (size_t)i + 2 * f + 1];
                }
                own[t] = psi + (size_t)i * Qp;
                // upwind rows: the neighbour's row, or the cell's own row as the Neumann ghost
                // (its fluctuation is then zero) scaled by 0 for the vacuum ghost; loads are
                // issued unconditionally so that all rows of a point are in flight together
                const int nbf[3] = {nb[t].x, nb[t].y, nb[t].z};
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    up[t][f] = nbf[f] >= 0 ? psi + (size_t)nbf[f] * Qp : own[t];
                    g[t][f] = (nbf[f] >= 0 || bc == 0) ? 1.0f : 0.0f;
                }
            }
            float F[kTogether][n], Fc[n];
#pragma unroll
            for (int a = 0; a < n; ++a) Fc[a] = 0.0f;
#pragma unroll
            for (int t = 0; t < kTogether; ++t)
#pragma unroll
                for (int a = 0; a < n; ++a) F[t][a] = 0.0f;
#pragma unroll 2
            for (int q = lane; q < Qp; q += 32) {
                const float wx = T.wox32[q], wy = T.woy32[q];
                float Mq[n];
#pragma unroll
                for (int a = 0; a < n; ++a) Mq[a] = T.Mt32[a * Qp + q];
#pragma unroll
                for (int t = 0; t < kTogether; ++t) {
                    const float pi = __ldg(own[t] + q);
                    float s = 0.0f;
#pragma unroll
                    for (int f = 0; f < 3; ++f) {
                        const float d = fmaf(wx, nx[t][f], wy * ny[t][f]);
                        s = fmaf(fminf(d, 0.0f), fmaf(g[t][f], __ldg(up[t][f] + q), -pi), s);
                    }
#pragma unroll
                    for (int a = 0; a < n; ++a) F[t][a] = fmaf(Mq[a], s, F[t][a]);
                }
            }
            // compensated reduce-scatter of the 32 lane sums of each cell
#pragma unroll
            for (int t = 0; t < kTogether; ++t) {
                float rs, re;
                const int slot = warp_reduce_scatter<n>(F[t], Fc, lane, rs, re);
                if (c0 + t < nb_cells && slot >= 0 && slot < n) sF[wib][(c0 + t) * n + slot] = rs + re;
            }
        }
        __syncwarp();
        for (int idx = lane; idx < nb_cells * n; idx += 32) {
            const int ci = idx / n, a = idx - ci * n, i = base + ci;
            const double ua = u[(size_t)i * n + a];
            const float* k = sK[wib][ci];
            // R = -sigma_a u - sigma_s (u - u_0 e_0) + q <m>: the scattering term of moment 0
            // cancels exactly
            const float sig = a == 0 ? k[0] : k[0] + k[1];
            const float R = fmaf(-sig, (float)ua, k[2] * T.mbar32[a]);
            const float inc = dt * fmaf(-k[3], sF[wib][idx], R);
            u[(size_t)i * n + a] = ua + (double)inc;
        }
        __syncwarp();
    }
}

}  // namespace

int launch_flux_update(kitrt_mn *mn, const Tables &T, int C, const double *psi,
                       const float *psi32, double *u, const double *sa, const double *ss,
                       const double *q, double dt, int bc, cudaStream_t s)
{
    const kitrt_mesh *m = mn->mesh;
    int need = (C + kWarps - 1) / kWarps;
    int cap = mn->nsm * 8;
    int grid = need < cap ? (need > 0 ? need : 1) : cap;
    // persistent grid of as many blocks as fit at once, batches of kBatch cells dealt round-robin
    // to warps (no partial second wave)
    int resident = 0;
    switch (mn->N) {
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, flux_update32_kernel<1>, kWarps * 32, 0); break;
    case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, flux_update32_kernel<2>, kWarps * 32, 0); break;
    case 3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, flux_update32_kernel<3>, kWarps * 32, 0); break;
    case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, flux_update32_kernel<4>, kWarps * 32, 0); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, flux_update32_kernel<5>, kWarps * 32, 0); break;
    }
    if (resident < 1) resident = 1;
    const int need32 = (C + kWarps * kBatch - 1) / (kWarps * kBatch);
    const int grid32 = need32 < mn->nsm * resident ? (need32 > 0 ? need32 : 1) : mn->nsm * resident;
    LaunchScope ls(mn, PK_FLUX, s, C);
#define FLUX_CASE(NN)                                                                          \
    case NN:                                                                                   \
        if (psi)                                                                               \
            flux_update_kernel<NN, double><<<grid, kWarps * 32, 0, s>>>(                        \
                T, m->d_nbr, m->d_nrm, m->d_area, psi, u, sa, ss, q, dt, bc, C);               \
        else                                                                                   \
            flux_update32_kernel<NN><<<grid32, kWarps * 32, 0, s>>>(                            \
                T, m->d_nbr, m->d_nrm32, m->d_inva32, psi32, u, sa, ss, q, (float)dt, bc, C);  \
        break;
    switch (mn->N) {
        FLUX_CASE(1)
        FLUX_CASE(2)
        FLUX_CASE(3)
        FLUX_CASE(4)
        FLUX_CASE(5)
    default: return KITRT_EINVAL;
    }
#undef FLUX_CASE
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

// Stability of the explicit step. The first-order kinetic update of the ansatz at quadrature
// point q keeps psi_iq (1 - dt/A_i sum_f (Omega_q.n_f)^+ - dt sigma_t,i) of the cell's own value;
// for a triangle sum_f (Omega.n_f)^+ = 1/2 sum_f |Omega.n_f| <= P_i / 2, so
//     dt (P_i / (2 A_i) + sigma_a,i + sigma_s,i) <= 1
// in every cell keeps every updated ordinate a non-negative combination of non-negative values
// (scattering and source only add), and the updated moments realizable. This is the cell-wise
// form of dt sigma_t,max <= 1 - CFL with CFL = dt / min_i (2 A_i / P_i), which implies it.
namespace {

__global__ void stability_kernel(const double *__restrict__ hpa, const double *__restrict__ sa,
                                 const double *__restrict__ ss, double dt, int C,
                                 unsigned long long *__restrict__ out)
{
    double worst = 0.0;
    unsigned bad = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
        const double a = sa[i], b = ss[i];
        if (!(a >= 0.0) || !(b >= 0.0) || !isfinite(a) || !isfinite(b)) ++bad;
        else worst = fmax(worst, dt * (hpa[i] + a + b));
    }
    // non-negative doubles order like their bit patterns
    unsigned long long wb = __double_as_longlong(worst);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, wb, o);
        wb = x > wb ? x : wb;
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[0], wb);
        if (bad) atomicAdd(&out[1], (unsigned long long)bad);
    }
}

}  // namespace

int check_stability(kitrt_mn *mn, const double *sa, const double *ss, double dt, cudaStream_t s,
                    bool wait)
{
    const int C = mn->mesh->C;
    if (!(dt > 0.0) || !isfinite(dt)) return KITRT_EINVAL;
    if (cudaMemsetAsync(mn->d_check, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess)
        return KITRT_ECUDA;
    int blocks = (C + 255) / 256;
    if (blocks > mn->nsm * 4) blocks = mn->nsm * 4;
    {
        LaunchScope ls(mn, PK_OTHER, s, C);
        stability_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(mn->mesh->d_hpa, sa, ss, dt, C,
                                                                  mn->d_check);
    }
    if (cudaGetLastError() != cudaSuccess) return KITRT_ECUDA;
    if (cudaMemcpyAsync(mn->h_check, mn->d_check, 2 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return KITRT_ECUDA;
    if (!wait) return KITRT_OK;
    if (cudaStreamSynchronize(s) != cudaSuccess) return KITRT_ECUDA;
    return stability_verdict(mn);
}

// Reads the test's result (the stream must have passed the copy in check_stability).
int stability_verdict(const kitrt_mn *mn)
{
    if (mn->h_check[1] != 0) return KITRT_EINVAL;
    double worst;
    memcpy(&worst, &mn->h_check[0], sizeof(double));
    // a relative slack of 1e-12 keeps dt = 1 / max(...) itself admissible after rounding
    return worst <= 1.0 + 1e-12 ? KITRT_OK : KITRT_EINVAL;
}
