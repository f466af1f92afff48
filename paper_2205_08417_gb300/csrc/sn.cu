// S_N step of the nodal (discrete-ordinates) system [Sec. 2, Eq. SNEqns2], explicit first-order
// finite volumes [Sec. 4.2] with the upwind flux applied to every ordinate [Sec. 4.4]:
//   psi'_iq = psi_iq - dt/A_i sum_f (Omega_q . n_if) psi_up - dt sigma_t,i psi_iq
//             + dt (O Sigma_i M psi_i)_q + dt q_i,
// on the solver's folded quadrature (the +-mu ordinates of the 2D problem are equal, so one
// folded point of weight 2w carries both). The scattering is the P_N form of Eq. SNEqns2
// truncated at the solver's degree N: the n moments M psi_i = sum_q w_q m(Omega_q) psi_iq are
// scaled by sigma_s,i g_l(a) (g_0 = 1) and mapped back by O = m(Omega_q); sigma_t = sigma_a +
// sigma_s. Isotropic scattering keeps the zeroth moment only.
//
// The flux is evaluated in fluctuation form, sum over faces with Omega.n < 0 of
// (Omega.n)(psi_up - psi_i), which equals the upwind form because the scaled normals of a closed
// cell sum to zero; a uniform state then sees exactly zero transport.
//
// The step streams the ordinates once: a persistent CTA takes tiles of TC consecutive cells,
// whose rows are one contiguous block of [C x Q'] memory, and stages each tile in shared memory
// with one TMA bulk copy (cp.async.bulk, completion on an mbarrier), double-buffered so that the
// next tile is in flight while the current one is computed. A warp per cell then forms the
// cell's moments from shared memory and writes its updated row straight to global memory
// (coalesced). Upwind rows are read from global memory, where the tile copies of this and the
// neighbouring CTAs have just brought them into L2 (Morton-ordered cells keep neighbours close).
// Every mbarrier wait is bounded; an expired wait records KITRT_ETIMEOUT in a device flag, waits
// (bounded) for the CTA's copies in flight and leaves the CTA.
#include <math.h>
#include <stdint.h>

#include "async_copy.cuh"
#include "kitrt_internal.cuh"

namespace {

using namespace kitrt_async;

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kTileBytes = 16384;  // target size of one staged tile
constexpr int kHeader = 128;       // shared-memory header: two mbarriers and the abort flag

template <typename P>
struct SnTab {
    const P *w;        // [Qp] folded weights (0 on padding)
    const P *ox, *oy;  // [Qp] folded directions
    const P *M;        // [n2 x Qp] basis at the folded points (rows 0..n-1 used)
    int Qf, Qp;
};

// Per-basis-function scattering coefficient g_l(a), a < n, in the ordinates' precision.
template <typename P>
struct SnScat {
    P ga[KITRT_MAX_NMOM];
};

// Per-cell coefficients of the step in the ordinates' precision, formed once per call so that
// the step itself has no FP64 work in FP32 mode: scaled normals of the three faces, dt / A_i,
// 1 - dt sigma_t,i, dt q_i and sigma_s,i (12 slots, the last two unused).
constexpr int kCellSlots = 12;
template <typename P>
__global__ void sn_cell_prep_kernel(const double *__restrict__ nrm, const double *__restrict__ area,
                                    const double *__restrict__ sa, const double *__restrict__ ss,
                                    const double *__restrict__ qs, double dt, P *__restrict__ cell, int C)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
        P *c = cell + (size_t)i * kCellSlots;
#pragma unroll
        for (int k = 0; k < 6; ++k) c[k] = (P)nrm[6 * (size_t)i + k];
        c[6] = (P)(dt / area[i]);
        c[7] = (P)(1.0 - dt * (sa[i] + ss[i]));
        c[8] = (P)(dt * qs[i]);
        c[9] = (P)ss[i];
        c[10] = P(0);
        c[11] = P(0);
    }
}

template <typename P>
__device__ __forceinline__ P warp_sum_p(P v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// V consecutive elements as one 16-byte access when V * sizeof(P) == 16 (rows and tables are
// then 16-byte aligned), else element by element.
template <typename P, int V>
struct Vec16 {
    P e[V];
};
template <typename P, int V>
__device__ __forceinline__ void ldv(const P *p, P (&v)[V])
{
    if constexpr (V * sizeof(P) == 16) {
        const Vec16<P, V> t = *reinterpret_cast<const Vec16<P, V> *>(p);
#pragma unroll
        for (int k = 0; k < V; ++k) v[k] = t.e[k];
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) v[k] = p[k];
    }
}
template <typename P, int V>
__device__ __forceinline__ void ldgv(const P *p, P (&v)[V])
{
    if constexpr (V * sizeof(P) == 16 && sizeof(P) == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    } else if constexpr (V * sizeof(P) == 16) {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
        v[0] = t.x, v[1] = t.y;
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) v[k] = __ldg(p + k);
    }
}
template <typename P, int V>
__device__ __forceinline__ void stv(P *p, const P (&v)[V])
{
    if constexpr (V * sizeof(P) == 16) {
        Vec16<P, V> t;
#pragma unroll
        for (int k = 0; k < V; ++k) t.e[k] = v[k];
        *reinterpret_cast<Vec16<P, V> *>(p) = t;
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) p[k] = v[k];
    }
}

// Bytes of a tile's rows moved by the bulk copy (the rest, below 16 bytes, by plain loads).
__device__ __forceinline__ uint32_t bulk_part(size_t bytes) { return (uint32_t)(bytes & ~(size_t)15); }

// Thread 0: start the copy of tile t into buf.
template <typename P>
__device__ __forceinline__ void issue_tile(const P *psi, int t, int TC, int C, int Qf, P *buf, uint64_t *bar)
{
    const int rows = min(TC, C - t * TC);
    const uint32_t nb = bulk_part((size_t)rows * Qf * sizeof(P));
    // the buffer was last read through the generic proxy: order those reads before the async
    // proxy writes it again
    fence_proxy_async_smem();
    mbar_expect_tx(bar, nb);
    if (nb > 0) bulk_g2s(buf, psi + (size_t)t * TC * Qf, nb, bar);
}

template <typename P, int NN, bool ISO, int V>
__global__ void __launch_bounds__(kThreads, 4)
sn_tile_kernel(SnTab<P> T, const int4 *__restrict__ nbr, const P *__restrict__ cellc,
               const P *__restrict__ psi, P *__restrict__ out, SnScat<P> sc, P dts, int bc, int C,
               int TC, int32_t *__restrict__ flag)
{
    constexpr int n = (NN + 1) * (NN + 2) / 2;
    constexpr int nm = ISO ? 1 : n;  // moments the scattering needs
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = (uint64_t *)smem;
    int *abort_flag = (int *)(smem + 16);
    const int Qf = T.Qf, Qp = T.Qp;
    const size_t tile_elems = (size_t)TC * Qf;
    const size_t buf_bytes = (tile_elems * sizeof(P) + 127) / 128 * 128;
    P *buf[2] = {(P *)(smem + kHeader), (P *)(smem + kHeader + buf_bytes)};
    P *sS = (P *)(smem + kHeader + 2 * buf_bytes);  // [TC x nm] scattered moments
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ntiles = (C + TC - 1) / TC;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int t = blockIdx.x;
    if (t < ntiles && tid == 0) issue_tile(psi, t, TC, C, Qf, buf[0], &bar[0]);
    // copies issued into and completed waits on each buffer (thread 0 issues and waits)
    uint32_t issued[2] = {t < ntiles ? 1u : 0u, 0u}, waited[2] = {0u, 0u};
    for (int k = 0; t < ntiles; t += gridDim.x, ++k) {
        const int b = k & 1;
        const int tn = t + gridDim.x;
        // prefetch the next tile into the other buffer (read completely in the last iteration)
        if (tn < ntiles && tid == 0) {
            issue_tile(psi, tn, TC, C, Qf, buf[b ^ 1], &bar[b ^ 1]);
            ++issued[b ^ 1];
        }
        const int base = t * TC;
        const int rows = min(TC, C - base);
        P *tile = buf[b];
        if (tid == 0) {
            if (mbar_wait_bounded(&bar[b], waited[b] & 1))
                ++waited[b];
            else
                *abort_flag = 1;
        }
        // the bytes of a ragged last tile past its last 16-byte boundary, by plain loads
        const size_t tail0 = bulk_part((size_t)rows * Qf * sizeof(P)) / sizeof(P);
        for (size_t e = tail0 + tid; e < (size_t)rows * Qf; e += kThreads) tile[e] = psi[(size_t)base * Qf + e];
        __syncthreads();
        if (*abort_flag) break;  // uniform: read after the barrier

        // moments of each cell of the tile, then the scattered moments sigma_s g_a u_a
        for (int c = warp; c < rows; c += kWarps) {
            const P *row = tile + (size_t)c * Qf;
            P acc[nm];
#pragma unroll
            for (int a = 0; a < nm; ++a) acc[a] = P(0);
            for (int q0 = lane * V; q0 < Qf; q0 += 32 * V) {
                P pv[V], wv[V];
                ldv<P, V>(row + q0, pv);
                ldgv<P, V>(T.w + q0, wv);
#pragma unroll
                for (int a = 0; a < nm; ++a) {
                    P mv[V];
                    ldgv<P, V>(T.M + a * Qp + q0, mv);
#pragma unroll
                    for (int k = 0; k < V; ++k) acc[a] = fma(wv[k] * pv[k], mv[k], acc[a]);
                }
            }
            const P sig_s = cellc[(size_t)(base + c) * kCellSlots + 9];
#pragma unroll
            for (int a = 0; a < nm; ++a) {
                const P v = sc.ga[a] * sig_s * warp_sum_p(acc[a]);
                if (lane == 0) sS[c * nm + a] = v;
            }
        }
        __syncwarp();

        // update of each cell's ordinates (the cell's own moments were formed by this warp)
        for (int c = warp; c < rows; c += kWarps) {
            const int i = base + c;
            const P *pi_row = tile + (size_t)c * Qf;
            const int4 nb = nbr[i];
            const P *cf = cellc + (size_t)i * kCellSlots;
            const P nx0 = cf[0], ny0 = cf[1], nx1 = cf[2], ny1 = cf[3], nx2 = cf[4], ny2 = cf[5];
            // upwind rows from global memory (L2: the tile copies of this and the neighbouring
            // CTAs bring them in), or the cell's own row as the boundary ghost (scaled by 0 for
            // vacuum); global loads keep the address arithmetic of the loop simple
            const P *own_g = psi + (size_t)i * Qf;
            const P *r0 = nb.x >= 0 ? psi + (size_t)nb.x * Qf : own_g;
            const P *r1 = nb.y >= 0 ? psi + (size_t)nb.y * Qf : own_g;
            const P *r2 = nb.z >= 0 ? psi + (size_t)nb.z * Qf : own_g;
            const P g0 = (nb.x >= 0 || bc == 0) ? P(1) : P(0);
            const P g1 = (nb.y >= 0 || bc == 0) ? P(1) : P(0);
            const P g2 = (nb.z >= 0 || bc == 0) ? P(1) : P(0);
            P s[nm];
#pragma unroll
            for (int a = 0; a < nm; ++a) s[a] = sS[c * nm + a];
            const P dtA = cf[6], keep = cf[7], src = cf[8];  // dt/A, 1 - dt sigma_t, dt q
            P *o_row = out + (size_t)i * Qf;
            for (int q0 = lane * V; q0 < Qf; q0 += 32 * V) {
                P p[V], p0[V], p1[V], p2[V], ox[V], oy[V], scat[V], o[V];
                ldv<P, V>(pi_row + q0, p);
                ldgv<P, V>(r0 + q0, p0);
                ldgv<P, V>(r1 + q0, p1);
                ldgv<P, V>(r2 + q0, p2);
                ldgv<P, V>(T.ox + q0, ox);
                ldgv<P, V>(T.oy + q0, oy);
#pragma unroll
                for (int k = 0; k < V; ++k) scat[k] = P(0);
#pragma unroll
                for (int a = 0; a < nm; ++a) {
                    P mv[V];
                    ldgv<P, V>(T.M + a * Qp + q0, mv);
#pragma unroll
                    for (int k = 0; k < V; ++k) scat[k] = fma(mv[k], s[a], scat[k]);
                }
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const P d0 = fma(ox[k], nx0, oy[k] * ny0);
                    const P d1 = fma(ox[k], nx1, oy[k] * ny1);
                    const P d2 = fma(ox[k], nx2, oy[k] * ny2);
                    P fl = P(0);
                    fl = fma(fmin(d0, P(0)), fma(g0, p0[k], -p[k]), fl);
                    fl = fma(fmin(d1, P(0)), fma(g1, p1[k], -p[k]), fl);
                    fl = fma(fmin(d2, P(0)), fma(g2, p2[k], -p[k]), fl);
                    o[k] = fma(keep, p[k], fma(-dtA, fl, fma(dts, scat[k], src)));
                }
                stv<P, V>(o_row + q0, o);
            }
        }
        // every read of this buffer is done before it is refilled two tiles later
        __syncthreads();
    }
    if (tid == 0 && *abort_flag) {
        atomicExch(flag, KITRT_ETIMEOUT);
        // copies still in flight must land before the CTA's shared memory is released
        for (int b = 0; b < 2; ++b)
            while (issued[b] > waited[b]) {
                if (!mbar_wait_bounded(&bar[b], waited[b] & 1)) break;
                ++waited[b];
            }
    }
}

template <typename P, int NN, bool ISO, int V>
int launch_sn_v(kitrt_mn *mn, const SnTab<P> &T, const P *psi, P *out, const P *cellc,
                const SnScat<P> &sc, double dt, cudaStream_t s)
{
    const kitrt_mesh *m = mn->mesh;
    const int C = m->C;
    constexpr int nm = ISO ? 1 : (NN + 1) * (NN + 2) / 2;
    // tile: about kTileBytes of rows, a multiple of 4 cells (so that every full tile starts on a
    // 16-byte boundary), at least 4 and at most 32 cells
    int TC = kTileBytes / (int)(T.Qf * sizeof(P));
    TC = TC < 4 ? 4 : (TC > 32 ? 32 : TC & ~3);
    const size_t buf_bytes = ((size_t)TC * T.Qf * sizeof(P) + 127) / 128 * 128;
    const size_t smem = kHeader + 2 * buf_bytes + (size_t)TC * nm * sizeof(P);
    if (ensure_dyn_smem(sn_tile_kernel<P, NN, ISO, V>, smem)) return KITRT_ECUDA;
    int resident = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, sn_tile_kernel<P, NN, ISO, V>, kThreads,
                                                      smem) != cudaSuccess ||
        resident < 1)
        resident = 1;
    const int ntiles = (C + TC - 1) / TC;
    const int cap = mn->nsm * resident;
    const int grid = ntiles < cap ? (ntiles > 0 ? ntiles : 1) : cap;
    LaunchScope ls(mn, PK_SN, s, C);
    sn_tile_kernel<P, NN, ISO, V><<<grid, kThreads, smem, s>>>(T, m->d_nbr, cellc, psi, out, sc, (P)dt,
                                                            mn->p.bc, C, TC, mn->d_sn_flag);
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

// 16-byte accesses when every row (Q' elements) is a whole number of them.
template <typename P, int NN, bool ISO>
int launch_sn(kitrt_mn *mn, const SnTab<P> &T, const P *psi, P *out, const P *cellc,
              const SnScat<P> &sc, double dt, cudaStream_t s)
{
    constexpr int V = 16 / sizeof(P);
    if (T.Qf % V == 0) return launch_sn_v<P, NN, ISO, V>(mn, T, psi, out, cellc, sc, dt, s);
    return launch_sn_v<P, NN, ISO, 1>(mn, T, psi, out, cellc, sc, dt, s);
}

template <typename P, bool ISO>
int dispatch_sn(kitrt_mn *mn, const SnTab<P> &T, const P *psi, P *out, const P *cellc,
                const SnScat<P> &sc, double dt, cudaStream_t s)
{
    switch (mn->N) {
    case 1: return launch_sn<P, 1, ISO>(mn, T, psi, out, cellc, sc, dt, s);
    case 2: return launch_sn<P, 2, ISO>(mn, T, psi, out, cellc, sc, dt, s);
    case 3: return launch_sn<P, 3, ISO>(mn, T, psi, out, cellc, sc, dt, s);
    case 4: return launch_sn<P, 4, ISO>(mn, T, psi, out, cellc, sc, dt, s);
    case 5: return launch_sn<P, 5, ISO>(mn, T, psi, out, cellc, sc, dt, s);
    default: return KITRT_EINVAL;
    }
}

template <typename P>
int run_sn(kitrt_mn *mn, const SnTab<P> &T, P *psi, P *work, const double *sa, const double *ss,
           const double *q, const SnScat<P> &sc, bool iso, double dt, int nsteps, cudaStream_t s)
{
    if (cudaMemsetAsync(mn->d_sn_flag, 0, sizeof(int32_t), s) != cudaSuccess) return KITRT_ECUDA;
    const kitrt_mesh *m = mn->mesh;
    P *cellc = (P *)mn->d_sn_cell;
    {
        int blocks = (m->C + 255) / 256;
        if (blocks > mn->nsm * 8) blocks = mn->nsm * 8;
        LaunchScope ls(mn, PK_OTHER, s, m->C);
        sn_cell_prep_kernel<P><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(m->d_nrm, m->d_area, sa, ss, q, dt,
                                                                        cellc, m->C);
        if (cudaGetLastError() != cudaSuccess) return KITRT_ECUDA;
    }
    P *a = psi, *b = work;
    for (int it = 0; it < nsteps; ++it) {
        const int rc = iso ? dispatch_sn<P, true>(mn, T, a, b, cellc, sc, dt, s)
                           : dispatch_sn<P, false>(mn, T, a, b, cellc, sc, dt, s);
        if (rc) return rc;
        P *t = a;
        a = b;
        b = t;
    }
    // an odd number of steps leaves the result in the scratch buffer
    if (a != psi &&
        cudaMemcpyAsync(psi, a, sizeof(P) * (size_t)mn->mesh->C * mn->Qf, cudaMemcpyDeviceToDevice,
                        s) != cudaSuccess)
        return KITRT_ECUDA;
    if (cudaMemcpyAsync(mn->h_sn_flag, mn->d_sn_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return KITRT_ECUDA;
    return *mn->h_sn_flag ? *mn->h_sn_flag : KITRT_OK;
}

}  // namespace

extern "C" {

int32_t kitrt_sn_step(kitrt_mn *mn, void *psi, void *work, int32_t fp32, const double *sigma_a,
                      const double *sigma_s, const double *q, const double *g, double dt,
                      int32_t nsteps, void *stream)
{
    if (!mn || !psi || !work || !sigma_a || !sigma_s || !q || nsteps < 0 || mn->d_invrho)
        return KITRT_EINVAL;
    // rows are staged with 16-byte bulk copies
    if (((uintptr_t)psi | (uintptr_t)work) & 15) return KITRT_EINVAL;
    const size_t bytes = (fp32 ? 4 : 8) * (size_t)mn->mesh->C * mn->Qf;
    const uintptr_t pa = (uintptr_t)psi, pb = (uintptr_t)work;
    if (pa < pb + bytes && pb < pa + bytes) return KITRT_EINVAL;  // the buffers overlap
    double ga[KITRT_MAX_NMOM] = {};
    bool iso = true;
    {
        // degree of each basis function, in the basis order (l ascending, then k)
        int a = 0;
        for (int l = 0; l <= mn->N; ++l)
            for (int k = -l; k <= l; ++k) {
                if ((l + (k < 0 ? -k : k)) % 2) continue;
                const double gl = g ? g[l] : (l == 0 ? 1.0 : 0.0);
                if (l == 0 && gl != 1.0) return KITRT_EINVAL;
                if (!isfinite(gl)) return KITRT_EINVAL;
                if (l > 0 && gl != 0.0) iso = false;
                ga[a++] = gl;
            }
    }
    if (nsteps == 0) return KITRT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (dt <= 0.0) dt = mn->p.cfl * mn->mesh->min_inradius;
    if (fp32) {
        SnTab<float> T{mn->d_w32, mn->d_ox32, mn->d_oy32, mn->d_Mt32, mn->Qf, mn->Qp};
        SnScat<float> sc{};
        for (int a = 0; a < KITRT_MAX_NMOM; ++a) sc.ga[a] = (float)ga[a];
        return run_sn<float>(mn, T, (float *)psi, (float *)work, sigma_a, sigma_s, q, sc, iso, dt,
                             nsteps, s);
    }
    SnTab<double> T{mn->d_w, mn->d_ox, mn->d_oy, mn->d_Mt, mn->Qf, mn->Qp};
    SnScat<double> sc{};
    for (int a = 0; a < KITRT_MAX_NMOM; ++a) sc.ga[a] = ga[a];
    return run_sn<double>(mn, T, (double *)psi, (double *)work, sigma_a, sigma_s, q, sc, iso, dt,
                          nsteps, s);
}

}  // extern "C"
