// Internal declarations of the kitrt library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "kitrt.h"

#define KITRT_MAX_DEGREE 5
#define KITRT_MAX_NMOM 21     // (5+1)(5+2)/2
#define KITRT_MAX_NMOM2 66    // degree-10 2D basis: (10+1)(10+2)/2

// FP64-pipe instructions of one kexp on its common path (kexp.cuh): 2 for the rounding to the
// table index, 2 for the two-part reduction, 3 for the polynomial, 1 for the table scaling.
constexpr int kExpFp64Ops = 8;
// FP64-pipe instructions of one kexp_scaled (sweep.cuh, the mixed sweep): r = s - k and the
// final fused multiply-add.
constexpr int kExpScaledFp64Ops = 2;

// Per-cell Newton phase.
enum : int32_t { PH_DONE = 0, PH_INIT = 1, PH_NEWTON = 2 };

struct kitrt_mesh {
    int32_t C = 0;
    int device = 0;
    double min_inradius = 0.0;
    std::vector<double> area, perim, cen, nrm, r;
    std::vector<int32_t> nbr;
    int4 *d_nbr = nullptr;     // [C] neighbours across faces 0..2 (-1 = boundary); .w: the
                               // neighbour's index of each shared face, 2 bits per face
    double *d_nrm = nullptr;   // [C x 6] scaled outward normals (nx0, ny0, nx1, ny1, nx2, ny2)
    double *d_area = nullptr;  // [C]
    double *d_hpa = nullptr;   // [C] P_i / (2 A_i): largest outflow rate of the cell per unit speed
    float *d_nrm32 = nullptr;  // [C x 6] FP32 copy of the scaled normals (FP32 flux)
    float *d_inva32 = nullptr; // [C] FP32 1 / A_i
    double *d_inva = nullptr;  // [C] 1 / A_i
    double *d_r = nullptr;     // [C x 6] centroid-to-face-midpoint offsets (second order)
    float *d_r32 = nullptr;    // FP32 copy
};

// Device views handed to kernels by value.
struct Tables {
    int n, n2, Qf, Qp;        // moments, degree-2N moments, folded points, padded points
    double m0;                // m_0 = 1/sqrt(4 pi)
    double rm0;               // 1 / m_0 = sqrt(4 pi)
    const double *Mt;         // [n2 x Qp] extended basis at folded points (first n rows = basis)
    const double *w;          // [Qp] folded weights (0 on padding)
    const double *wox, *woy;  // [Qp] w * Omega_x, w * Omega_y
    const double *mbar;       // [n] sum_q w_q m_q
    const int32_t *gstart;    // [npairs + 1] Gaunt term ranges per packed pair (a >= b)
    const int32_t *gidx;      // [nnz] extended-moment index c
    const double *gcoef;      // [nnz] <m_a m_b m~_c>
    const float *gcoef32;     // [nnz] FP32 copy (the mixed modes' FP32 Hessian)
    const float *Mt32;        // [n2 x Qp] FP32 copy
    const float *w32;
    const float *wox32, *woy32;  // FP32 copies of w * Omega
    const float *mbar32;         // [n] FP32 copy of <m>
    const double *exptab;     // [2 x 2048] 2^(j/2048) (kexp), then 2^(j/2048) ln2/2048 (kexp_scaled)
    // sum-factorised sweeps (sweep.cuh): rings of P pairs of points; R rings (row R of the ring
    // tables is zero, for padding pairs); npair = Qf / 2 pairs
    int R, P, npair;
    const double *ptrig;      // [Qp/2 x (4N+1)] azimuthal factors of each pair
    const double *ringP;      // [(R+1) x n2] P_c(mu_r)
    const double *ringWP;     // [(R+1) x n2] w_r P_c(mu_r)
};

struct NewtonState {
    double *alpha;     // [C x n] current iterate alpha_k (pre-polish)
    double *dir;       // [C x n] Newton direction at alpha_k (polish direction once converged)
    double *U;         // [C x n] moments <m exp(alpha_k.m)>
    double *fsum;      // [C] <exp(alpha_k.m)>
    double *f0;        // [C] f(alpha_k; u) for the Armijo test
    double *gd;        // [C] g(alpha_k).dir
    double *L;         // [C x npairs] packed lower Cholesky factor of H(alpha_k)
    double *lam;       // [C] line-search step
    int32_t *phase;    // [C]
    int32_t *iters;    // [C] accepted Newton iterations in this closure
    int32_t *halv;     // [C] halvings in the current iteration
    int32_t *evals;    // [C] evaluations in this closure
    int32_t *status;   // [C]
    int32_t *h64;      // [C] mixed modes: 1 = this cell evaluates its Hessian in FP64 (else NULL)
    double *gnorm;     // [C] mixed modes: ||g|| at the last accepted point (else NULL)
    int32_t *lfac;     // [C] learned mode: 1 once S.L holds a factor of this cell (else NULL)
    int32_t *list[2];  // active cell lists (ping-pong)
    int32_t *cnt;      // [16]: cnt[0..2] rotating list counters, cnt[3] failures, cnt[4] max
                       //   evals, cnt[5] fallbacks, cnt[6] evaluations, cnt[7] timeout status,
                       //   cnt[8] predictor list length, cnt[9] learned-mode steps taken
                       //   from a stored factor, cnt[10] learned-mode residual passes of the
                       //   network's proposals, cnt[11] mixed-mode hand-overs to the FP64 Hessian
};

struct NewtonParams {
    double tau, c1;
    int max_iter, max_halvings, polish;
    // (partially) regularized closure: the dual gains gamma/2 |alpha^r|^2 over the moments
    // r = reg0..n-1 (gamma = 0: the entropy closure)
    double gamma;
    int reg0;
};

// Kernel kinds recorded by the tracer.
enum ProfKind : int { PK_BEGIN = 0, PK_EVAL = 1, PK_FINISH = 2, PK_FLUX = 3, PK_EVAL_MIXED = 4,
                      PK_MLP = 5, PK_ADJOINT = 6, PK_OTHER = 7, PK_POST = 8, PK_SN = 9,
                      PK_RECON = 10, PK_COUNT = 11 };

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
};

struct kitrt_mn {
    const kitrt_mesh *mesh = nullptr;
    kitrt_mn_params p{};
    int N = 0, n = 0, n2 = 0, npairs = 0, Q = 0, Qf = 0, Qp = 0;
    int nsm = 0;
    int gaunt_nnz = 0;
    std::vector<double> h_w, h_ox, h_oy, h_M;  // folded tables (host copies; M is [Qf x n])
    // device tables
    double *d_Mt = nullptr, *d_w = nullptr, *d_wox = nullptr, *d_woy = nullptr;
    double *d_mbar = nullptr, *d_gcoef = nullptr;
    float *d_gcoef32 = nullptr;
    int32_t *d_gstart = nullptr, *d_gidx = nullptr;
    float *d_Mt32 = nullptr, *d_w32 = nullptr;
    float *d_Mhi32 = nullptr;            // [NP x Qp] TF32-rounded degree-(N+1..2N) basis (mixed)
    unsigned short *d_Mhi16 = nullptr;   // [NP x Qp] BF16 copy
    float *d_wox32 = nullptr, *d_woy32 = nullptr, *d_mbar32 = nullptr;
    double *d_ox = nullptr, *d_oy = nullptr;  // [Qp] folded directions (0 on padding), S_N step
    float *d_ox32 = nullptr, *d_oy32 = nullptr;
    double *d_V = nullptr;               // [C x n2] moments scratch (kitrt_hessian)
    double *d_Vacc = nullptr;            // [n2 x vs] sweeps: partial moments per list slot and part
    int vs = 0;                          // column stride of d_Vacc (C + room for split parts)
    int target_mixed = 0, target_fp64 = 0;  // work items the sweeps aim at per launch
    int grid_mixed = 0, grid_fp64 = 0;      // persistent grids of the sweeps
    int R = 0, P = 0;                    // rings and pairs per ring of the folded rule
    double *d_ptrig = nullptr, *d_ringP = nullptr, *d_ringWP = nullptr;
    double *d_exptab = nullptr;          // [2 x 2048] exp tables (Tables::exptab)
    void *d_mlp16 = nullptr;             // learned closure: BF16 network parameters
    float *d_mlp_norm = nullptr;         // [4 (n-1)] feature and output means / scales
    bool has_mlp = false;
    double *d_alpha_nn = nullptr;        // [C x n] network proposals (learned mode)
    // workspace
    NewtonState st{};
    double *d_psi = nullptr;   // [C x Qp] FP64 ansatz
    void *d_psif = nullptr;    // second order: [C x 3 x Qp] reconstructed face values (FP64/FP32)
    double *d_ustage = nullptr;  // second order: [C x n] the Heun stage u*
    float *d_psi32 = nullptr;  // [C x Qp] FP32 ansatz (mixed modes)
    float *d_zero32 = nullptr; // [Qp] zeros: the vacuum ghost's row in the FP32 flux
    // transformed CSD equation (kitrt_mn_set_density): 1 / rho per cell, FP64 and FP32 (NULL:
    // no density, rho = 1)
    double *d_invrho = nullptr;
    float *d_invrho32 = nullptr;
    double *d_rho_store = nullptr;  // [2 C] owned storage behind d_invrho / d_invrho32
    int32_t *h_cnt = nullptr;  // pinned copy of st.cnt
    // kitrt_mn_reset: the next kitrt_step starts every cell from its given alpha (otherwise each
    // cell whose given alpha is the one the solver last returned continues from its stored state)
    bool force_cold = false;
    int pass_hint = 4;  // rounds in the first batch of a closure (the last closure's evaluations)
    // stability test of kitrt_step / kitrt_adjoint: [0] largest dt (P/2A + sigma_a + sigma_s) as
    // the bits of a non-negative double, [1] cells with a negative or non-finite coefficient
    unsigned long long *d_check = nullptr, *h_check = nullptr;
    void *d_adj = nullptr;     // kitrt_adjoint workspace (grown on demand)
    size_t adj_bytes = 0;
    int32_t *d_sn_flag = nullptr;  // S_N step: device status (KITRT_ETIMEOUT on an expired wait)
    int32_t *h_sn_flag = nullptr;  // pinned copy
    void *d_sn_cell = nullptr;     // [C x 12] per-cell coefficients of the S_N step (FP32 or FP64)
    std::vector<void *> allocs;
    // tracing
    bool prof_on = false;
    std::vector<ProfRec> prof_recs;
    size_t prof_used = 0;
    int64_t prof_launches[PK_COUNT] = {}, prof_units[PK_COUNT] = {};
    int64_t launch_count = 0;  // kernels launched (all calls)
    Tables tables() const;
};

// Records CUDA events around one kernel launch when tracing is on, and counts the launch.
struct LaunchScope {
    kitrt_mn *mn;
    int kind;
    cudaStream_t s;
    ProfRec *rec = nullptr;
    LaunchScope(kitrt_mn *m, int k, cudaStream_t st, int64_t units);
    ~LaunchScope();
};

// Raise a kernel's dynamic shared-memory limit to at least `smem` bytes on the current device.
// The attribute is per device, so the record is keyed by (kernel, device).
template <typename Kern>
inline int ensure_dyn_smem(Kern *kernel, size_t smem)
{
    static std::mutex mtx;
    static std::map<std::pair<const void *, int>, size_t> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return KITRT_ECUDA;
    std::lock_guard<std::mutex> lock(mtx);
    size_t &have = done[std::make_pair((const void *)kernel, dev)];
    if (have >= smem) return KITRT_OK;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return KITRT_ECUDA;
    have = smem;
    return KITRT_OK;
}

// CTAs of a kernel that fit on one SM at once, from its register and shared-memory use and the
// device's per-SM limits (asks for the largest shared-memory carveout first), at most `cap`.
template <typename Kern>
inline int resident_ctas(Kern *kernel, int threads, size_t dyn_smem, int cap)
{
    int dev = 0;
    cudaFuncAttributes fa;
    int regs_sm = 0, smem_sm = 0, thr_sm = 0, reserved = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&fa, kernel) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
        return 1;
    if (cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
        reserved = 1024;
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    const int warps = (threads + 31) / 32;
    const int regs_cta = warps * 32 * ((fa.numRegs + 7) / 8 * 8);  // allocated per warp in 256s
    int n = thr_sm / threads;
    if (regs_cta > 0) n = std::min(n, regs_sm / regs_cta);
    const size_t smem_cta = dyn_smem + fa.sharedSizeBytes + (size_t)reserved;
    if (smem_cta > 0) n = std::min(n, (int)((size_t)smem_sm / smem_cta));
    return std::max(1, std::min(n, cap));
}

// Kernel launchers (closure_fp64.cu, flux.cu).
int launch_isotropic(const Tables &T, int C, const double *u, double *alpha, cudaStream_t s);
int launch_begin(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C,
                 const double *u, const double *alpha_in, int first, NewtonParams np,
                 cudaStream_t s, int learned = 0);
int launch_mlp_infer(kitrt_mn *mn, const double *u, const int32_t *list, const int32_t *cnt, int C,
                     double *alpha, cudaStream_t s);
int launch_learned_pass(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C, const double *u,
                        float *psi32, int first, cudaStream_t s);
int fp64_sweep_grid(const kitrt_mn *mn);
int mixed_sweep_grid(const kitrt_mn *mn);
int launch_eval_fp64(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C,
                     const double *u, int k, NewtonParams np, cudaStream_t s,
                     bool filter = false, float *psi32 = nullptr, double *Vacc = nullptr);
int launch_sum_parts(kitrt_mn *mn, const NewtonState &S, int k, double *Vacc, cudaStream_t s);
int launch_post(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C, const double *u, int k,
                NewtonParams np, double *Vacc, cudaStream_t s);
int launch_finish(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C,
                  double *alpha_out, double *psi, float *psi32, int polish, int compare_prev,
                  cudaStream_t s);
int launch_ansatz(const Tables &T, int C, const double *alpha, double *psi, cudaStream_t s);
int launch_moments_fp64(kitrt_mn *mn, const Tables &T, int C, const double *alpha, double *V,
                        cudaStream_t s);
int launch_gaunt(kitrt_mn *mn, const Tables &T, int C, const double *V, double *H, cudaStream_t s);
int launch_eval_mixed(kitrt_mn *mn, const Tables &T, const NewtonState &S, int C, const double *u,
                      int k, NewtonParams np, cudaStream_t s, float *psi32);
int launch_moments_mixed(kitrt_mn *mn, const Tables &T, int C, const double *alpha, double *Vout,
                         cudaStream_t s);
int check_stability(kitrt_mn *mn, const double *sa, const double *ss, double dt, cudaStream_t s,
                    bool wait);
int stability_verdict(const kitrt_mn *mn);
int launch_recon(kitrt_mn *mn, const Tables &T, const void *psi, void *psif, bool fp32, int bc,
                 cudaStream_t s);
int launch_flux2(kitrt_mn *mn, const Tables &T, const void *psi, const void *psif, bool fp32,
                 const double *uin, const double *base, double *uout, const double *sa,
                 const double *ss, const double *q, double dt, double c0, double c1, int bc,
                 cudaStream_t s);
int launch_flux_update(kitrt_mn *mn, const Tables &T, int C, const double *psi,
                       const float *psi32, double *u, const double *sa, const double *ss,
                       const double *q, double dt, int bc, cudaStream_t s);
