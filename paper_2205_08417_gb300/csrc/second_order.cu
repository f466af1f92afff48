// Second-order M_N step [Sec. 4.3]: a linear reconstruction of the closed ansatz at every
// quadrature point (the inputs of the kinetic upwind flux are the ordinate values psi_q), limited
// by Barth and Jespersen, the upwind flux of the reconstructed face values, and Heun time
// stepping.
//
//   gradient   g_i = 1/A_i sum_f 1/2 (psi_i + psi_j(f)) n_if            (Green-Gauss)
//   limiter    Psi_i = min(1, min_f ratio_f), ratio_f = (max(psi_i, psi_j) - psi_i) / D_f for
//              D_f = g_i . r_if > 0, (min(psi_i, psi_j) - psi_i) / D_f for D_f < 0, none for 0
//   face value psif_if = psi_i + Psi_i g_i . r_if
// (r_if: centroid to face midpoint; across a boundary face psi_j is the ghost: psi_i for
// Neumann, 0 for vacuum). The limited face value lies between psi_i and psi_j, so positive
// ordinates stay positive. The flux in fluctuation form (exact: sum_f n_f = 0),
//   F_i = sum_f sum_q w_q m_q [(Omega.n_f)^+ (psif_if - psi_i) + (Omega.n_f)^- (up_f - psi_i)],
// up_f = psif_j(f)f' (the neighbour's face value at the shared face; ghost: psif_if for Neumann,
// 0 for vacuum), is zero on uniform states. One Heun stage writes
//   out = c0 base + c1 (in + dt (-F/A + R(in))):  stage 1 (c0, c1) = (0, 1), stage 2 (1/2, 1/2)
// with base = u^n, in = u*.
// Kernels: warp per cell, lanes over the folded quadrature points; FP64 (FP64 mode) or FP32
// ordinates and arithmetic with an FP64 update (mixed modes, as the first-order FP32 flux).
#include "flux_group.cuh"
#include "kitrt_internal.cuh"

namespace {

using kitrt_flux::kFull;
constexpr int kWarps = 8;

template <typename P>
__device__ __forceinline__ P across(int j, const P *__restrict__ psi, size_t jq, P pi, int bc)
{
    return j >= 0 ? psi[jq] : (bc == 0 ? pi : P(0));
}

// Reconstruction: psif [C x 3 x Qp] from psi [C x Qp]. nrm, r: [C x 6]; inva: [C] (type P).
template <typename P>
__global__ void __launch_bounds__(kWarps * 32)
recon_kernel(int Qp, const int4 *__restrict__ nbr, const P *__restrict__ nrm,
             const P *__restrict__ r, const P *__restrict__ inva, const P *__restrict__ psi,
             P *__restrict__ psif, int bc, int C)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int i = blockIdx.x * kWarps + wib; i < C; i += gridDim.x * kWarps) {
        const int4 nb = nbr[i];
        const int j[3] = {nb.x, nb.y, nb.z};
        P nx[3], ny[3], rx[3], ry[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            nx[f] = nrm[6 * (size_t)i + 2 * f];
            ny[f] = nrm[6 * (size_t)i + 2 * f + 1];
            rx[f] = r[6 * (size_t)i + 2 * f];
            ry[f] = r[6 * (size_t)i + 2 * f + 1];
        }
        const P half_inva = P(0.5) * inva[i];
        for (int q = lane; q < Qp; q += 32) {
            const P pi = psi[(size_t)i * Qp + q];
            P pj[3];
#pragma unroll
            for (int f = 0; f < 3; ++f) pj[f] = across(j[f], psi, (size_t)(j[f] < 0 ? 0 : j[f]) * Qp + q, pi, bc);
            P gx = 0, gy = 0;
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const P s = pi + pj[f];
                gx += s * nx[f];
                gy += s * ny[f];
            }
            gx *= half_inva;
            gy *= half_inva;
            // the smallest ratio bound / D over the faces, kept as a fraction (num >= 0, den > 0)
            // and divided once
            P num = 1, den = 1;
            P D[3];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                D[f] = gx * rx[f] + gy * ry[f];
                P a = 0, b = 0;
                if (D[f] > P(0)) {
                    a = (pi > pj[f] ? pi : pj[f]) - pi;
                    b = D[f];
                } else if (D[f] < P(0)) {
                    a = pi - (pi < pj[f] ? pi : pj[f]);
                    b = -D[f];
                }
                if (b > P(0) && a * den < num * b) {
                    num = a;
                    den = b;
                }
            }
            const P L = num < den ? num / den : P(1);
#pragma unroll
            for (int f = 0; f < 3; ++f) psif[((size_t)i * 3 + f) * Qp + q] = pi + L * D[f];
        }
    }
}

// FP32 reconstruction of the mixed modes, laid out as the FP32 fluxes: a group of 8 lanes per
// cell, 4 cells per warp, 16-byte pieces (4 consecutive points) of the cell's row and of its
// neighbours' rows (on the boundary the cell's own row, Neumann, or the zero row, vacuum), the
// same arithmetic as recon_kernel per point, the three face values stored as 16-byte pieces.
__global__ void __launch_bounds__(kWarps * 32)
recon32_kernel(int Qp, const int4 *__restrict__ nbr, const float *__restrict__ nrm,
               const float *__restrict__ r, const float *__restrict__ inva,
               const float *__restrict__ psi, const float *__restrict__ zrow,
               float *__restrict__ psif, int bc, int C)
{
    using namespace kitrt_flux;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane >> kGroupLog, gl = lane & (kGroup - 1);
    const int nq4 = Qp / 4;
    for (int b0 = (blockIdx.x * kWarps + wib) * kCellsPerWarp; b0 < C;
         b0 += gridDim.x * kWarps * kCellsPerWarp) {
        const int i = b0 + grp;
        if (i >= C) continue;  // no warp-collective operation below
        const int4 nb = nbr[i];
        const int j[3] = {nb.x, nb.y, nb.z};
        float nx[3], ny[3], rx[3], ry[3];
        const float4 *own = reinterpret_cast<const float4 *>(psi + (size_t)i * Qp);
        const float4 *nrow[3];
        float4 *frow[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            nx[f] = nrm[6 * (size_t)i + 2 * f];
            ny[f] = nrm[6 * (size_t)i + 2 * f + 1];
            rx[f] = r[6 * (size_t)i + 2 * f];
            ry[f] = r[6 * (size_t)i + 2 * f + 1];
            nrow[f] = j[f] >= 0 ? reinterpret_cast<const float4 *>(psi + (size_t)j[f] * Qp)
                      : bc == 0 ? own
                                : reinterpret_cast<const float4 *>(zrow);
            frow[f] = reinterpret_cast<float4 *>(psif + ((size_t)i * 3 + f) * Qp);
        }
        const float half_inva = 0.5f * inva[i];
#pragma unroll 1
        for (int q4 = gl; q4 < nq4; q4 += kGroup) {
            const float4 p4 = __ldg(own + q4);
            float4 n4[3];
#pragma unroll
            for (int f = 0; f < 3; ++f) n4[f] = __ldg(nrow[f] + q4);
            float out[3][4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float pi = c == 0 ? p4.x : c == 1 ? p4.y : c == 2 ? p4.z : p4.w;
                float pj[3];
#pragma unroll
                for (int f = 0; f < 3; ++f)
                    pj[f] = c == 0 ? n4[f].x : c == 1 ? n4[f].y : c == 2 ? n4[f].z : n4[f].w;
                float gx = 0.0f, gy = 0.0f;
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    const float sf = pi + pj[f];
                    gx += sf * nx[f];
                    gy += sf * ny[f];
                }
                gx *= half_inva;
                gy *= half_inva;
                // the smallest ratio bound / D over the faces, kept as a fraction, divided once
                float num = 1.0f, den = 1.0f, D[3];
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    D[f] = gx * rx[f] + gy * ry[f];
                    float a = 0.0f, b = 0.0f;
                    if (D[f] > 0.0f) {
                        a = (pi > pj[f] ? pi : pj[f]) - pi;
                        b = D[f];
                    } else if (D[f] < 0.0f) {
                        a = pi - (pi < pj[f] ? pi : pj[f]);
                        b = -D[f];
                    }
                    if (b > 0.0f && a * den < num * b) {
                        num = a;
                        den = b;
                    }
                }
                const float L = num < den ? num / den : 1.0f;
#pragma unroll
                for (int f = 0; f < 3; ++f) out[f][c] = pi + L * D[f];
            }
#pragma unroll
            for (int f = 0; f < 3; ++f) frow[f][q4] = make_float4(out[f][0], out[f][1], out[f][2], out[f][3]);
        }
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Upwind flux of the face values and one Heun stage, FP64 (warp per cell).
template <int NN>
__global__ void __launch_bounds__(kWarps * 32)
flux2_kernel(Tables T, const int4 *__restrict__ nbr, const double *__restrict__ nrm,
             const double *__restrict__ inva, const double *__restrict__ psi,
             const double *__restrict__ psif, const double *__restrict__ uin,
             const double *__restrict__ base, double *__restrict__ uout,
             const double *__restrict__ sa, const double *__restrict__ ss,
             const double *__restrict__ qs, double dt, double c0, double c1, int bc, int C)
{
    constexpr int n = (NN + 1) * (NN + 2) / 2;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int Qp = T.Qp;
    for (int i = blockIdx.x * kWarps + wib; i < C; i += gridDim.x * kWarps) {
        const int4 nb = nbr[i];
        const int j[3] = {nb.x, nb.y, nb.z};
        const int kk[3] = {nb.w & 3, (nb.w >> 2) & 3, (nb.w >> 4) & 3};
        double nx[3], ny[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            nx[f] = nrm[6 * (size_t)i + 2 * f];
            ny[f] = nrm[6 * (size_t)i + 2 * f + 1];
        }
        double F[n];
#pragma unroll
        for (int a = 0; a < n; ++a) F[a] = 0.0;
        for (int q = lane; q < Qp; q += 32) {
            const double pi = psi[(size_t)i * Qp + q];
            const double wx = T.wox[q], wy = T.woy[q];
            double s = 0.0;
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const double d = fma(wx, nx[f], wy * ny[f]);
                const double own = psif[((size_t)i * 3 + f) * Qp + q];
                double up;
                if (d > 0.0) {
                    up = own;
                } else {
                    up = j[f] >= 0 ? psif[((size_t)j[f] * 3 + kk[f]) * Qp + q] : (bc == 0 ? own : 0.0);
                }
                s = fma(d, up - pi, s);
            }
#pragma unroll
            for (int a = 0; a < n; ++a) F[a] = fma(T.Mt[a * Qp + q], s, F[a]);
        }
        double Fa = 0.0;
#pragma unroll
        for (int a = 0; a < n; ++a) {
            const double v = warp_sum(F[a]);
            if (lane == a) Fa = v;
        }
        if (lane < n) {
            const double ua = uin[(size_t)i * n + lane];
            const double u0 = uin[(size_t)i * n];
            const double R = -sa[i] * ua - ss[i] * (ua - (lane == 0 ? u0 : 0.0)) + qs[i] * T.mbar[lane];
            const double next = ua + dt * (R - inva[i] * Fa);
            const double b = c0 != 0.0 ? base[(size_t)i * n + lane] : 0.0;
            uout[(size_t)i * n + lane] = c0 * b + c1 * next;
        }
    }
}

// FP32 variant for the mixed modes: FP32 ordinates, face values and sums, the increment in FP32
// and the Heun combination in FP64. Layout as the first-order FP32 flux (flux_group.cuh): a group
// of 8 lanes per cell, 4 cells per warp, 16-byte pieces (4 consecutive points) of the cell's row,
// of its three face rows and of the three upwind face rows, the group's lane sums reduced with a
// compensated reduce-scatter, then lanes over the (cell, moment) elements of the warp's cells.
template <int NN>
__global__ void __launch_bounds__(kWarps * 32, NN <= 3 ? 3 : 2)
flux2_32_kernel(Tables T, const int4 *__restrict__ nbr, const float *__restrict__ nrm32,
                const float *__restrict__ inva32, const float *__restrict__ psi,
                const float *__restrict__ psif, const float *__restrict__ zrow,
                const double *__restrict__ uin, const double *__restrict__ base,
                double *__restrict__ uout, const double *__restrict__ sa,
                const double *__restrict__ ss, const double *__restrict__ qs, float dt, double c0,
                double c1, int bc, int C)
{
    using namespace kitrt_flux;
    constexpr int n = (NN + 1) * (NN + 2) / 2;
    constexpr int K = GroupRS<n>::K;
    __shared__ float sF[kWarps][kCellsPerWarp * n];
    __shared__ float sK[kWarps][kCellsPerWarp][4];  // per cell: sigma_a, sigma_s, q, 1/A
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane >> kGroupLog, gl = lane & (kGroup - 1);
    const int Qp = T.Qp, nq4 = Qp / 4;
    const float4 *__restrict__ wx4 = reinterpret_cast<const float4 *>(T.wox32);
    const float4 *__restrict__ wy4 = reinterpret_cast<const float4 *>(T.woy32);
    const float4 *__restrict__ M4 = reinterpret_cast<const float4 *>(T.Mt32);
    for (int b0 = (blockIdx.x * kWarps + wib) * kCellsPerWarp; b0 < C;
         b0 += gridDim.x * kWarps * kCellsPerWarp) {
        const int nb_cells = C - b0 < kCellsPerWarp ? C - b0 : kCellsPerWarp;
        if (lane < 4 * nb_cells) {
            const int ci = lane >> 2, which = lane & 3, i = b0 + ci;
            const double v = which == 0 ? sa[i] : which == 1 ? ss[i] : qs[i];
            sK[wib][ci][which] = which == 3 ? inva32[i] : (float)v;
        }
        // a group without a cell repeats the warp's last one; its sums are not stored
        const int i = b0 + (grp < nb_cells ? grp : nb_cells - 1);
        const int4 nb = nbr[i];
        const int j[3] = {nb.x, nb.y, nb.z};
        const int kk[3] = {nb.w & 3, (nb.w >> 2) & 3, (nb.w >> 4) & 3};
        float nx[3], ny[3];
        const float4 *own = reinterpret_cast<const float4 *>(psi + (size_t)i * Qp);
        const float4 *ofr[3], *ufr[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            nx[f] = nrm32[6 * (size_t)i + 2 * f];
            ny[f] = nrm32[6 * (size_t)i + 2 * f + 1];
            ofr[f] = reinterpret_cast<const float4 *>(psif + ((size_t)i * 3 + f) * Qp);
            // upwind face value: the neighbour's at the shared face; across a boundary the
            // cell's own face value (Neumann) or zero (vacuum)
            ufr[f] = j[f] >= 0 ? reinterpret_cast<const float4 *>(psif + ((size_t)j[f] * 3 + kk[f]) * Qp)
                     : bc == 0 ? ofr[f]
                               : reinterpret_cast<const float4 *>(zrow);
        }
        float F[n];
#pragma unroll
        for (int a = 0; a < n; ++a) F[a] = 0.0f;
#pragma unroll 1
        for (int q4 = gl; q4 < nq4; q4 += kGroup) {
            const float4 po = __ldg(own + q4);
            const float4 wx = __ldg(wx4 + q4), wy = __ldg(wy4 + q4);
            float4 of[3], uf[3];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                of[f] = __ldg(ofr[f] + q4);
                uf[f] = __ldg(ufr[f] + q4);
            }
            float sv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float pi = c == 0 ? po.x : c == 1 ? po.y : c == 2 ? po.z : po.w;
                const float wxc = c == 0 ? wx.x : c == 1 ? wx.y : c == 2 ? wx.z : wx.w;
                const float wyc = c == 0 ? wy.x : c == 1 ? wy.y : c == 2 ? wy.z : wy.w;
                float acc = 0.0f;
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    const float o = c == 0 ? of[f].x : c == 1 ? of[f].y : c == 2 ? of[f].z : of[f].w;
                    const float uu = c == 0 ? uf[f].x : c == 1 ? uf[f].y : c == 2 ? uf[f].z : uf[f].w;
                    const float d = fmaf(wxc, nx[f], wyc * ny[f]);
                    acc = fmaf(d, (d > 0.0f ? o : uu) - pi, acc);
                }
                sv[c] = acc;
            }
#pragma unroll
            for (int a = 0; a < n; ++a) {
                const float4 m = __ldg(M4 + (size_t)a * nq4 + q4);
                F[a] = fmaf(m.w, sv[3], fmaf(m.z, sv[2], fmaf(m.y, sv[1], fmaf(m.x, sv[0], F[a]))));
            }
        }
        float rs[K], re[K];
        int slot0;
        const bool uniq = group_reduce_scatter<n>(F, gl, rs, re, slot0);
        if (grp < nb_cells && uniq) {
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (slot0 + k < n) sF[wib][grp * n + slot0 + k] = rs[k] + re[k];
        }
        __syncwarp();
        for (int idx = lane; idx < nb_cells * n; idx += 32) {
            const int ci = idx / n, a = idx - ci * n, ic = b0 + ci;
            const double ua = uin[(size_t)ic * n + a];
            const float *k = sK[wib][ci];
            const float sig = a == 0 ? k[0] : k[0] + k[1];
            const float R = fmaf(-sig, (float)ua, k[2] * T.mbar32[a]);
            const float inc = dt * fmaf(-k[3], sF[wib][idx], R);
            const double next = ua + (double)inc;
            const double b = c0 != 0.0 ? base[(size_t)ic * n + a] : 0.0;
            uout[(size_t)ic * n + a] = c0 * b + c1 * next;
        }
        __syncwarp();
    }
}

}  // namespace

int launch_recon(kitrt_mn *mn, const Tables &T, const void *psi, void *psif, bool fp32, int bc,
                 cudaStream_t s)
{
    const kitrt_mesh *m = mn->mesh;
    const int C = m->C;
    int blocks = (C + kWarps - 1) / kWarps;
    if (blocks > mn->nsm * 16) blocks = mn->nsm * 16;
    LaunchScope ls(mn, PK_RECON, s, C);
    if (fp32) {
        if (T.Qp % 32 != 0 || !mn->d_zero32) return KITRT_EINVAL;
        const int cells_per_block = kWarps * kitrt_flux::kCellsPerWarp;
        int blocks32 = (C + cells_per_block - 1) / cells_per_block;
        if (blocks32 > mn->nsm * 8) blocks32 = mn->nsm * 8;
        recon32_kernel<<<blocks32, kWarps * 32, 0, s>>>(T.Qp, m->d_nbr, m->d_nrm32, m->d_r32,
                                                       m->d_inva32, (const float *)psi,
                                                       mn->d_zero32, (float *)psif, bc, C);
    } else
        recon_kernel<double><<<blocks, kWarps * 32, 0, s>>>(T.Qp, m->d_nbr, m->d_nrm, m->d_r,
                                                            m->d_inva, (const double *)psi,
                                                            (double *)psif, bc, C);
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

int launch_flux2(kitrt_mn *mn, const Tables &T, const void *psi, const void *psif, bool fp32,
                 const double *uin, const double *base, double *uout, const double *sa,
                 const double *ss, const double *q, double dt, double c0, double c1, int bc,
                 cudaStream_t s)
{
    const kitrt_mesh *m = mn->mesh;
    const int C = m->C;
    int blocks = (C + kWarps - 1) / kWarps;
    if (blocks > mn->nsm * 16) blocks = mn->nsm * 16;
    if (fp32 && (T.Qp % 32 != 0 || !mn->d_zero32)) return KITRT_EINVAL;
    const int cells_per_block = kWarps * kitrt_flux::kCellsPerWarp;
    int blocks32 = (C + cells_per_block - 1) / cells_per_block;
    if (blocks32 > mn->nsm * 3) blocks32 = mn->nsm * 3;  // persistent: the CTAs resident at once
    LaunchScope ls(mn, PK_FLUX, s, C);
#define FLUX2_CASE(NNv)                                                                           \
    case NNv:                                                                                     \
        if (fp32)                                                                                 \
            flux2_32_kernel<NNv><<<blocks32, kWarps * 32, 0, s>>>(                                \
                T, m->d_nbr, m->d_nrm32, m->d_inva32, (const float *)psi, (const float *)psif,    \
                mn->d_zero32, uin, base, uout, sa, ss, q, (float)dt, c0, c1, bc, C);              \
        else                                                                                      \
            flux2_kernel<NNv><<<blocks, kWarps * 32, 0, s>>>(                                     \
                T, m->d_nbr, m->d_nrm, m->d_inva, (const double *)psi, (const double *)psif, uin, \
                base, uout, sa, ss, q, dt, c0, c1, bc, C);                                        \
        break;
    switch (mn->N) {
        FLUX2_CASE(1)
        FLUX2_CASE(2)
        FLUX2_CASE(3)
        FLUX2_CASE(4)
        FLUX2_CASE(5)
    default: return KITRT_EINVAL;
    }
#undef FLUX2_CASE
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}
