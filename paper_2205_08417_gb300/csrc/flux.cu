// Kinetic upwind flux of the closed ansatz and the explicit first-order update
// [Sec. 4.4 kinetic numerical flux; Sec. 4.2 explicit iteration; Sec. 3.1 isotropic scattering].
//
// Cell-centric gather (lanes over the folded quadrature points of a cell). The upwind
// flux sum_f sum_q w_q m_q (Omega_q.n_f) psi_up is evaluated in its fluctuation form
//     F_i = sum_f sum_{q: Omega_q.n_f < 0} w_q m_q (Omega_q.n_f) (psi_up,f,q - psi_iq),
// which equals it exactly in exact arithmetic because the scaled normals of a closed cell sum to
// zero (sum_f n_f = 0), so psi_iq sum_f Omega_q.n_f vanishes: outflow directions drop out, the
// upwind value is the neighbour's psi (the ghost: psi_iq for Neumann, 0 for vacuum), and a
// uniform state gives exactly zero flux at any working precision. F is projected on the basis,
// warp-reduced, and u <- u - dt/A F + dt R(u) is applied in place (the flux reads psi only).
// psi rows are contiguous per cell, so each face gather is a coalesced row segment.
#include <string.h>

#include "flux_group.cuh"
#include "kitrt_internal.cuh"

namespace {

using namespace kitrt_flux;
constexpr int kWarps = 8;

// Plain FP64 reduce-scatter of n per-lane sums across the warp: at each of log2(S) halving levels
// (offsets 16, 8, ...) a lane keeps one half of its slots and adds its partner's copy of that half;
// the remaining levels are butterflies between lanes holding the same slot. Lane L ends with the
// total of slot L >> (5 - H): S - 1 + 5 - H additions per lane instead of 5 n for a butterfly per
// sum (each one a warp-wide FP64 instruction).
template <int n>
__device__ __forceinline__ double warp_reduce_scatter64(const double (&F)[n], int lane)
{
    constexpr int S = Slots<n>::S, H = Slots<n>::H;
    double sv[S];
#pragma unroll
    for (int k = 0; k < S; ++k) sv[k] = k < n ? F[k < n ? k : 0] : 0.0;
#pragma unroll
    for (int lvl = 0; lvl < H; ++lvl) {
        const int o = 16 >> lvl;
        const int half = S >> (lvl + 1);
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const double keep = upper ? sv[k + half] : sv[k];
            const double give = upper ? sv[k] : sv[k + half];
            sv[k] = keep + __shfl_xor_sync(kFull, give, o);
        }
    }
    double r = sv[0];
#pragma unroll
    for (int o = 16 >> H; o > 0; o >>= 1) r += __shfl_xor_sync(kFull, r, o);
    return r;
}

// FP64 flux (FP64 mode): one warp per cell, lanes over the points. The FP64 pipe is the bound
// (a warp-wide FP64 instruction occupies it for 16 cycles), so the inflow test reads the sign
// bit of Omega.n in integer arithmetic instead of comparing in FP64, and the moments are reduced
// with a reduce-scatter.
// RHO: the transformed CSD equation's density (Sec. 2, Eq. BoltzmannCSDTrafo): the transported
// value is psi / rho, so each row is scaled by its cell's 1/rho (invrho) before differencing.
template <int NN, bool RHO>
__global__ void __launch_bounds__(kWarps * 32)
flux_update_kernel(Tables T, const int4 *__restrict__ nbr, const double *__restrict__ nrm,
                   const double *__restrict__ area, const double *__restrict__ psi,
                   const double *__restrict__ invrho, double *__restrict__ u,
                   const double *__restrict__ sa, const double *__restrict__ ss,
                   const double *__restrict__ qs, double dt, int bc, int C)
{
    constexpr int n = (NN + 1) * (NN + 2) / 2;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int Qp = T.Qp;
    for (int i = blockIdx.x * kWarps + wib; i < C; i += gridDim.x * kWarps) {
        const int4 nb = nbr[i];
        const int nbf[3] = {nb.x, nb.y, nb.z};
        double nx[3], ny[3], g[3];
        const double *up[3];
        const double *own = psi + (size_t)i * Qp;
        const double ri = RHO ? invrho[i] : 1.0;
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            nx[f] = nrm[6 * (size_t)i + 2 * f];
            ny[f] = nrm[6 * (size_t)i + 2 * f + 1];
            // upwind row: the neighbour's, or the cell's own as the ghost (Neumann: fluctuation
            // 0; vacuum: scaled by 0, so the fluctuation is -psi_i)
            up[f] = nbf[f] >= 0 ? psi + (size_t)nbf[f] * Qp : own;
            g[f] = (nbf[f] >= 0 || bc == 0) ? 1.0 : 0.0;
            if (RHO) {
                g[f] *= nbf[f] >= 0 ? invrho[nbf[f]] : ri;
                // Neumann ghost: its fluctuation is exactly zero, so the face drops out (the
                // scaled difference ri psi_i - ri psi_i would leave a rounding residue)
                if (nbf[f] < 0 && bc == 0) nx[f] = ny[f] = 0.0;
            }
        }
        double F[n];
#pragma unroll
        for (int a = 0; a < n; ++a) F[a] = 0.0;
        for (int q = lane; q < Qp; q += 32) {
            const double pi = RHO ? ri * own[q] : own[q];
            const double wx = T.wox[q], wy = T.woy[q];
            double s = 0.0;
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const double d = fma(wx, nx[f], wy * ny[f]);
                const double dm = __double2hiint(d) < 0 ? d : 0.0;  // min(d, 0); -0 adds nothing
                s = fma(dm, fma(g[f], up[f][q], -pi), s);
            }
#pragma unroll
            for (int a = 0; a < n; ++a) F[a] = fma(T.Mt[a * Qp + q], s, F[a]);
        }
        const double r = warp_reduce_scatter64<n>(F, lane);
        // slot a is held by lane a << (5 - H)
        const double Fa = __shfl_sync(kFull, r, (lane << (5 - Slots<n>::H)) & 31);
        const double u0 = u[(size_t)i * n];
        if (lane < n) {
            const double ua = u[(size_t)i * n + lane];
            const double R = -sa[i] * ua - ss[i] * (ua - (lane == 0 ? u0 : 0.0)) + qs[i] * T.mbar[lane];
            u[(size_t)i * n + lane] = ua - dt / area[i] * Fa + dt * R;
        }
    }
}

// FP32 flux of the mixed modes. FP64 instructions are rare on this GPU (2 per clock per SM), so
// none is spent on warp-uniform values: normals and inverse areas come from the mesh's FP32
// copies, the per-cell coefficients are converted by different lanes at once, and the update
// increment dt (-F/A + R(u)) is formed in FP32; only u += increment is FP64 (lanes over the
// (cell, moment) elements of a warp's cells).
//
// Layout of the work: a group of kGroup = 8 lanes per cell, 4 cells per warp. Each lane reads
// 16-byte pieces (4 consecutive points) of the cell's row and of its three upwind rows, and the
// matching pieces of the tables, which the warp's 4 cells read at the same addresses (one
// request serves them). Q' padded to a multiple of 32 gives every lane the same number of pieces.
// Each lane sums its points in plain FP32; the 8 lane sums of a cell are reduced with a
// compensated (two-sum) reduce-scatter.
// Upwind fluctuation sum of one point: s = sum_f min(Omega.n_f, 0) (psi_up,f - psi_i), or with a
// density (RHO) sum_f min(Omega.n_f, 0) (psi_up,f / rho_up,f - psi_i / rho_i) (r: the 1/rho).
template <bool RHO>
__device__ __forceinline__ float point_fluct(float wx, float wy, const float (&nx)[3],
                                             const float (&ny)[3], float ri, const float (&r)[3],
                                             float pi, float u0, float u1, float u2)
{
    if (RHO) {
        const float tp = ri * pi;
        float s = fminf(fmaf(wx, nx[0], wy * ny[0]), 0.0f) * fmaf(r[0], u0, -tp);
        s = fmaf(fminf(fmaf(wx, nx[1], wy * ny[1]), 0.0f), fmaf(r[1], u1, -tp), s);
        return fmaf(fminf(fmaf(wx, nx[2], wy * ny[2]), 0.0f), fmaf(r[2], u2, -tp), s);
    }
    float s = fminf(fmaf(wx, nx[0], wy * ny[0]), 0.0f) * (u0 - pi);
    s = fmaf(fminf(fmaf(wx, nx[1], wy * ny[1]), 0.0f), u1 - pi, s);
    return fmaf(fminf(fmaf(wx, nx[2], wy * ny[2]), 0.0f), u2 - pi, s);
}

// Latency bound: 3 resident blocks per SM (at most 85 registers) measured 0.127 ms per M_3 launch
// on 99,458 cells against 0.179 ms at the unconstrained 94 registers (2 blocks).
template <int NN, bool RHO>
__global__ void __launch_bounds__(kWarps * 32, NN <= 3 ? 3 : 2)
flux_update32_kernel(Tables T, const int4 *__restrict__ nbr, const float *__restrict__ nrm32,
                     const float *__restrict__ inva32, const float *__restrict__ psi,
                     const float *__restrict__ zrow, const float *__restrict__ invrho32,
                     double *__restrict__ u,
                     const double *__restrict__ sa, const double *__restrict__ ss,
                     const double *__restrict__ qs, float dt, int bc, int C)
{
    constexpr int n = (NN + 1) * (NN + 2) / 2;
    constexpr int K = GroupRS<n>::K;
    __shared__ float sF[kWarps][kCellsPerWarp * n];
    __shared__ float sK[kWarps][kCellsPerWarp][4];  // per cell: sigma_a, sigma_s, q, 1/A (FP32)
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane >> kGroupLog, gl = lane & (kGroup - 1);
    const int Qp = T.Qp, nq4 = Qp / 4;
    const float4 *__restrict__ wx4 = reinterpret_cast<const float4 *>(T.wox32);
    const float4 *__restrict__ wy4 = reinterpret_cast<const float4 *>(T.woy32);
    const float4 *__restrict__ M4 = reinterpret_cast<const float4 *>(T.Mt32);
    for (int base = (blockIdx.x * kWarps + wib) * kCellsPerWarp; base < C;
         base += gridDim.x * kWarps * kCellsPerWarp) {
        const int nb_cells = C - base < kCellsPerWarp ? C - base : kCellsPerWarp;
        if (lane < 4 * nb_cells) {
            const int ci = lane >> 2, which = lane & 3, i = base + ci;
            const double v = which == 0 ? sa[i] : which == 1 ? ss[i] : qs[i];
            sK[wib][ci][which] = which == 3 ? inva32[i] : (float)v;
        }
        // a group without a cell repeats the warp's last one; its sums are not stored
        const int i = base + (grp < nb_cells ? grp : nb_cells - 1);
        const int4 nb = nbr[i];
        const int nbf[3] = {nb.x, nb.y, nb.z};
        float nx[3], ny[3], r[3];
        const float4 *own = reinterpret_cast<const float4 *>(psi + (size_t)i * Qp);
        const float4 *up[3];
        const float ri = RHO ? invrho32[i] : 1.0f;
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            nx[f] = nrm32[6 * (size_t)i + 2 * f];
            ny[f] = nrm32[6 * (size_t)i + 2 * f + 1];
            r[f] = RHO && nbf[f] >= 0 ? invrho32[nbf[f]] : ri;
            if (RHO && nbf[f] < 0 && bc == 0) nx[f] = ny[f] = 0.0f;  // Neumann ghost drops out
            // upwind row: the neighbour's; on the boundary the cell's own (Neumann ghost:
            // fluctuation 0) or the zero row (vacuum ghost: fluctuation -psi_i)
            up[f] = nbf[f] >= 0 ? reinterpret_cast<const float4 *>(psi + (size_t)nbf[f] * Qp)
                    : bc == 0   ? own
                                : reinterpret_cast<const float4 *>(zrow);
        }
        float F[n];
#pragma unroll
        for (int a = 0; a < n; ++a) F[a] = 0.0f;
#pragma unroll 2
        for (int j = gl; j < nq4; j += kGroup) {
            const float4 po = __ldg(own + j);
            const float4 p0 = __ldg(up[0] + j), p1 = __ldg(up[1] + j), p2 = __ldg(up[2] + j);
            const float4 wx = __ldg(wx4 + j), wy = __ldg(wy4 + j);
            const float s0 = point_fluct<RHO>(wx.x, wy.x, nx, ny, ri, r, po.x, p0.x, p1.x, p2.x);
            const float s1 = point_fluct<RHO>(wx.y, wy.y, nx, ny, ri, r, po.y, p0.y, p1.y, p2.y);
            const float s2 = point_fluct<RHO>(wx.z, wy.z, nx, ny, ri, r, po.z, p0.z, p1.z, p2.z);
            const float s3 = point_fluct<RHO>(wx.w, wy.w, nx, ny, ri, r, po.w, p0.w, p1.w, p2.w);
#pragma unroll
            for (int a = 0; a < n; ++a) {
                const float4 m = __ldg(M4 + (size_t)a * nq4 + j);
                F[a] = fmaf(m.w, s3, fmaf(m.z, s2, fmaf(m.y, s1, fmaf(m.x, s0, F[a]))));
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
            const int ci = idx / n, a = idx - ci * n, ic = base + ci;
            const double ua = u[(size_t)ic * n + a];
            const float *k = sK[wib][ci];
            // R = -sigma_a u - sigma_s (u - u_0 e_0) + q <m>: the scattering term of moment 0
            // cancels exactly
            const float sig = a == 0 ? k[0] : k[0] + k[1];
            const float R = fmaf(-sig, (float)ua, k[2] * T.mbar32[a]);
            const float inc = dt * fmaf(-k[3], sF[wib][idx], R);
            u[(size_t)ic * n + a] = ua + (double)inc;
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
    // persistent grid of as many blocks as fit at once, groups of 4 cells dealt round-robin to
    // warps (no partial second wave)
    int resident = 0;
    switch (mn->N) {
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, flux_update32_kernel<1, false>, kWarps * 32, 0); break;
    case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, flux_update32_kernel<2, false>, kWarps * 32, 0); break;
    case 3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, flux_update32_kernel<3, false>, kWarps * 32, 0); break;
    case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, flux_update32_kernel<4, false>, kWarps * 32, 0); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, flux_update32_kernel<5, false>, kWarps * 32, 0); break;
    }
    if (resident < 1) resident = 1;
    const int need32 = (C + kWarps * kCellsPerWarp - 1) / (kWarps * kCellsPerWarp);
    const int grid32 = need32 < mn->nsm * resident ? (need32 > 0 ? need32 : 1) : mn->nsm * resident;
    if (!psi && (T.Qp % 32 != 0 || !mn->d_zero32)) return KITRT_EINVAL;
    const bool rho = mn->d_invrho != nullptr;
    LaunchScope ls(mn, PK_FLUX, s, C);
#define FLUX_LAUNCH(NN, R)                                                                     \
    if (psi)                                                                                   \
        flux_update_kernel<NN, R><<<grid, kWarps * 32, 0, s>>>(                                 \
            T, m->d_nbr, m->d_nrm, m->d_area, psi, mn->d_invrho, u, sa, ss, q, dt, bc, C);     \
    else                                                                                       \
        flux_update32_kernel<NN, R><<<grid32, kWarps * 32, 0, s>>>(                             \
            T, m->d_nbr, m->d_nrm32, m->d_inva32, psi32, mn->d_zero32, mn->d_invrho32, u, sa,  \
            ss, q, (float)dt, bc, C);
#define FLUX_CASE(NN)                                                                          \
    case NN:                                                                                   \
        if (rho) {                                                                             \
            FLUX_LAUNCH(NN, true)                                                              \
        } else {                                                                               \
            FLUX_LAUNCH(NN, false)                                                             \
        }                                                                                      \
        break;
    switch (mn->N) {
        FLUX_CASE(1)
        FLUX_CASE(2)
        FLUX_CASE(3)
        FLUX_CASE(4)
        FLUX_CASE(5)
    default: return KITRT_EINVAL;
    }
#undef FLUX_LAUNCH
#undef FLUX_CASE
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

// Stability of the explicit step. The first-order kinetic update of the ansatz at quadrature
// point q keeps psi_iq (1 - dt/A_i sum_f (Omega_q.n_f)^+ - dt sigma_t,i) of the cell's own value;
// for a triangle sum_f (Omega.n_f)^+ = 1/2 sum_f |Omega.n_f| <= P_i / 2, so
//     dt (P_i / (2 A_i) + sigma_a,i + sigma_s,i) <= 1
// in every cell keeps every updated ordinate a non-negative combination of non-negative values
// (scattering and source only add), and the updated moments realizable. This is the cell-wise
// form of dt sigma_t,max <= 1 - CFL with CFL = dt / min_i (2 A_i / P_i), which implies it. With a
// density (transported value psi / rho) the outflow rate of cell i is P_i / (2 A_i rho_i).
namespace {

__global__ void stability_kernel(const double *__restrict__ hpa, const double *__restrict__ invrho,
                                 const double *__restrict__ sa, const double *__restrict__ ss,
                                 double dt, int C, unsigned long long *__restrict__ out)
{
    double worst = 0.0;
    unsigned bad = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
        const double a = sa[i], b = ss[i];
        // with a density the transport speed of cell i is 1 / rho_i
        const double h = invrho ? hpa[i] * invrho[i] : hpa[i];
        if (!(a >= 0.0) || !(b >= 0.0) || !isfinite(a) || !isfinite(b)) ++bad;
        else worst = fmax(worst, dt * (h + a + b));
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
        stability_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(mn->mesh->d_hpa, mn->d_invrho, sa,
                                                                  ss, dt, C, mn->d_check);
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
