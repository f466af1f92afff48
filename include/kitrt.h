/*
 * kitrt — C ABI of the GB300 minimal-entropy (M_N) step library.
 *
 * The method is the explicit first-order finite-volume M_N scheme of KiT-RT (arXiv 2205.08417):
 *   - entropy closure with the Maxwell-Boltzmann entropy [Sec. 3.1, Eq. entropyOCP], solved per
 *     cell through its dual  f(alpha) = <exp(alpha.m)> - alpha.u  by Newton's method with an
 *     Armijo line search [Sec. 7.2, M_N runs];
 *   - kinetic upwind flux of the closed ansatz [Sec. 4.4, kinetic numerical flux];
 *   - isotropic scattering, absorption and source with a forward-Euler update
 *     [Sec. 3.1 moment equations; Sec. 4.2 explicit first-order iteration].
 * Angular discretisation: real spherical harmonics of degree N, restricted to the functions even
 * in mu for the 2D slab geometry [Sec. 3.1, Sec. 3.2], on the tensorised Gauss-Legendre x
 * uniform-azimuth product rule [Sec. 3.2, Eq. spherical-coordinatesProduct] with `order` Gauss
 * points and 2*order azimuths (Q = 2 order^2 points; the library folds the +-mu pairs, which share
 * a 2D direction, into Q' = Q/2 points of doubled weight).
 *
 * Conventions
 *   - Every function returns a kitrt_status code; nothing is thrown across the ABI.
 *   - "device" pointers are CUDA device memory owned by the caller; "host" pointers are host
 *     memory. State arrays are row-major, one row per cell: u and alpha are [ncells x nmom] FP64.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Calls enqueue
 *     work on it. Calls that must know when every cell's Newton iteration has finished read a
 *     4-byte counter back to the host and therefore synchronise with `stream` (noted below).
 *   - The library owns the handles, the angular tables and its workspace (allocated in
 *     kitrt_mesh_create / kitrt_mn_init, freed by the matching destroy). kitrt_step and
 *     kitrt_closure allocate nothing.
 *   - Device kernels never trap: per-cell failures are reported in `status` arrays and in the
 *     return code.
 */
#ifndef KITRT_H
#define KITRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. Per-cell status values use the same numbers (0 = converged). */
typedef enum {
    KITRT_OK = 0,
    KITRT_EINVAL = 1,          /* bad argument (null pointer, size, unsupported option) */
    KITRT_ENOTREALIZABLE = 2,  /* a moment vector had no finite minimiser (non-finite values) */
    KITRT_ENOCONVERGE = 3,     /* a cell hit max_iter Newton iterations */
    KITRT_ECHOL = 4,           /* Hessian not positive definite in FP64 (Cholesky breakdown) */
    KITRT_ELINESEARCH = 5,     /* Armijo backtracking exhausted max_halvings */
    KITRT_ECUDA = 6,           /* a CUDA runtime call failed */
    KITRT_ENOMEM = 7,          /* device allocation failed */
    KITRT_ETIMEOUT = 8,        /* a bounded device wait expired */
    KITRT_ESCRATCH = 9         /* batch larger than the fixed scratch of kitrt_closure_noalloc */
} kitrt_status;

/* Closure arithmetic. */
enum {
    KITRT_FP64 = 0,        /* every sum, factorisation and line search in FP64 */
    KITRT_MIXED_TF32 = 1,  /* Hessian-only moment sums on tensor cores (TF32 in, FP32 accumulate);
                              exponent, gradient, objective and line search in FP64 (the exp to
                              about 1e-14 relative, its small polynomial term in FP32); the Newton
                              step's Hessian assembly and Cholesky in FP32, in FP64 for cells
                              handed over */
    KITRT_MIXED_BF16 = 2,  /* as MIXED_TF32 with BF16 tensor-core inputs */
    KITRT_LEARNED = 3      /* MLP prediction of alpha, exact mass fix, FP64 residual check, Newton
                              (mixed Hessian) only for cells whose residual exceeds fallback_tol */
};

/* Boundary condition on boundary faces [Sec. 4.4: Neumann and Dirichlet]. */
enum {
    KITRT_BC_NEUMANN = 0,  /* zero-gradient ghost: the outside value is the cell's own psi */
    KITRT_BC_VACUUM = 1    /* Dirichlet psi = 0 outside: boundary faces only let radiation out */
};

typedef struct kitrt_mesh kitrt_mesh;
typedef struct kitrt_mn kitrt_mn;

typedef struct {
    int32_t degree;        /* 1 <= N <= 5; nmom = (N+1)(N+2)/2 */
    int32_t quad_order;    /* Gauss points in mu (>= N+1); Q = 2 order^2 */
    int32_t mode;          /* KITRT_FP64 / KITRT_MIXED_TF32 / KITRT_MIXED_BF16 / KITRT_LEARNED */
    int32_t bc;            /* KITRT_BC_NEUMANN / KITRT_BC_VACUUM */
    double tau;            /* Newton stops when ||g||_2 <= tau ||u||_2 (e.g. 1e-10) */
    int32_t max_iter;      /* Newton iterations per closure (e.g. 100) */
    int32_t max_halvings;  /* Armijo halvings per iteration (e.g. 30) */
    double armijo_c1;      /* Armijo constant (e.g. 1e-4) */
    int32_t polish;        /* 1: one extra full Newton step after the test passes */
    double cfl;            /* dt = cfl * min_i 2 A_i / P_i when kitrt_step gets dt <= 0 */
    double fallback_tol;   /* KITRT_LEARNED: accept the MLP when ||<m psi> - u|| <= tol ||u|| */
    int32_t order;         /* 1: first-order upwind flux and forward Euler [Sec. 4.2];
                              2: second order in space and time [Sec. 4.3]: the ansatz at every
                              quadrature point reconstructed linearly per cell (Green-Gauss
                              gradient, Barth-Jespersen limiter), upwind flux of the
                              reconstructed face values, Heun time stepping (two closures per
                              step) */
    double reg_gamma;      /* (partially) regularized closure [Sec. 3.1, Eq. entropyOCP_reg and
                              Eq. entropyOCP_part_reg] with parameter gamma (0: the entropy
                              closure). Its dual is f(alpha) + gamma/2 |alpha^r|^2: the ansatz no
                              longer reproduces the regularized moments (it has u^r - gamma alpha^r)
                              but a minimiser exists for any u (with u_0 > 0 when it is kept).
                              Not with KITRT_LEARNED or kitrt_adjoint. */
    int32_t reg_keep_mass; /* 1: u_0 is not regularized (r = moments 1..n-1, the paper's partial
                              form); 0: every moment is */
} kitrt_mn_params;

/* Counters of the last call (filled only when a non-null pointer is passed; doing so
 * synchronises with the stream). */
typedef struct {
    int64_t closures;      /* cell closures solved (cells x steps) */
    int64_t evaluations;   /* cell evaluations of the dual (quadrature passes) */
    int32_t max_evals;     /* largest number of evaluations any cell needed in one closure */
    int32_t failed;        /* cells whose last closure ended with a non-zero status */
    int64_t fallbacks;     /* KITRT_LEARNED: cells that needed Newton after the MLP */
    double dt;             /* time step used */
    int64_t launches;      /* CUDA kernels the library launched in this call */
    int64_t restarts;      /* KITRT_LEARNED: fallbacks whose better start was the previous closure's
                              point, stepped from its stored Cholesky factor without a new pass */
    int64_t proposals;     /* KITRT_LEARNED: closures the network was asked for (the rest were
                              already converged from the previous step's state) */
    int64_t handovers;     /* mixed modes: cells sent from the tensor-core Hessian to the FP64
                              Hessian (FP32 factor not positive definite, stalled residual, or
                              line search exhausted), counted once per cell and closure */
} kitrt_stats;

/* Per-kernel-kind trace record (see kitrt_profile_enable). `units` counts what one kind
 * processes: cell evaluations of the dual for the closure sweeps, cells for the other kernels. */
typedef struct {
    char name[32];
    int64_t launches;
    int64_t units;
    double total_ms;       /* device time between CUDA events recorded around each launch */
} kitrt_profile_entry;

/* Human-readable name of a status code (static string). */
const char *kitrt_status_string(int32_t code);

/* Fill `p` with the defaults used by the library's tests: N=2, order 10, FP64, Neumann,
 * tau 1e-10, max_iter 100, 30 halvings, c1 1e-4, polish on, CFL 0.4, fallback_tol 1e-6, first
 * order in space and time, no regularization (reg_gamma 0, reg_keep_mass 1). */
int32_t kitrt_default_params(kitrt_mn_params *p);

/* Build a triangle mesh [Sec. 4.1: cell-centred unstructured grid with centroid, area A_i,
 * neighbours N(i) and face normals n_ij scaled by the face length].
 *   xy  host [nverts x 2] vertex coordinates; tri host [ntri x 3] vertex indices (either
 *       orientation; clockwise triangles are reversed). Face k of cell i is the edge from its
 *       (counter-clockwise) vertex k to vertex k+1.
 *   out receives the handle. The host arrays are copied; geometry is uploaded to the current
 *   CUDA device. EINVAL for null pointers, out-of-range indices, zero-area cells or edges shared
 *   by more than two cells. */
int32_t kitrt_mesh_create(const double *xy, int32_t nverts, const int32_t *tri, int32_t ntri,
                          kitrt_mesh **out);
int32_t kitrt_mesh_destroy(kitrt_mesh *mesh);

/* Copy the mesh geometry to host arrays (any may be NULL): area [C], perimeter [C],
 * centroid [C x 2], neighbour [C x 3] (-1 = boundary), scaled outward normal [C x 3 x 2];
 * ncells and the largest stable step min_i 2 A_i / P_i (to be scaled by the CFL number). */
int32_t kitrt_mesh_geometry(const kitrt_mesh *mesh, int32_t *ncells, double *min_inradius,
                            double *area, double *perim, double *centroid, int32_t *nbr,
                            double *nrm);

/* Create an M_N solver on a mesh: builds the folded quadrature [Sec. 3.2, Eq.
 * spherical-coordinatesProduct: tensorised Gauss-Legendre points in mu times equally spaced
 * azimuths], the real spherical-harmonic basis at its points [Sec. 3.1: the modal basis of the
 * moment system, here the functions even in mu], the Gaunt coefficients <m_a m_b m~_c> with which
 * the closure assembles the Hessian of its dual, and the workspace for every cell of the mesh
 * (device allocations, owned by the handle). The mesh must outlive the solver. EINVAL for a degree
 * outside 1..5, quad_order < degree + 1 or > 64, tau <= 0, max_iter < 1, max_halvings < 0, or an
 * unknown mode or boundary condition; ENOMEM when an allocation fails. */
int32_t kitrt_mn_init(const kitrt_mesh *mesh, const kitrt_mn_params *params, kitrt_mn **out);
int32_t kitrt_mn_destroy(kitrt_mn *mn);

/* Sizes: moments n, quadrature points Q of the full rule and Q' after folding. */
int32_t kitrt_mn_sizes(const kitrt_mn *mn, int32_t *nmom, int32_t *nquad, int32_t *nquad_folded);

/* Work accounting of one cell evaluation of the dual (one quadrature pass) in the solver's mode:
 * moments n, degree-2N moments n2, folded points Q', non-zero Gaunt coefficients, and
 *   sweep_fp64_flops   FP64 flops (FMA = 2) of the quadrature sweep without exp, in its
 *                      sum-factorised form over pairs of mirrored azimuths and rings of equal
 *                      |mu|: per pair (Q'/2 of them) the exponents (2N - 1 operations) and the
 *                      azimuthal sums up to degree L (L = N in the mixed modes, whose higher
 *                      moments run on tensor cores; L = 2N in FP64 mode), per ring the exponent
 *                      coefficients (n FMA) and the moments (nmom(L) FMA);
 *   sweep_fp64_ops     FP64-pipe instructions of the same sweep including the exponentials
 *                      (on the common path of the table-driven method: 8 per exp in FP64
 *                      mode; 2 in the mixed modes, whose exponents are pre-scaled by 2048/ln2
 *                      and whose small polynomial term is formed in FP32);
 *   exps               exponentials per evaluation (Q');
 *   tensor_flops       mixed modes: 3 x 2 (n2 - n) Q' on tensor cores (three split products);
 *   newton_flops       the per-cell Newton step: 2 nnz (Hessian) + n^3/3 + 2n^2 (Cholesky,
 *                      solves);
 *   sweep_grid, sweep_items  launch shape of the sweep on this device. */
typedef struct {
    int32_t nmom, nmom2, nquad_folded, gaunt_nnz;
    double sweep_fp64_flops;
    double exps;
    double tensor_flops;
    double newton_flops;
    double sweep_fp64_ops;
    int32_t sweep_grid;     /* CTAs of the mode's quadrature sweep (persistent grid) */
    int32_t sweep_items;    /* work items (cell tiles x quadrature parts) it aims at per launch */
} kitrt_work;
int32_t kitrt_mn_work(const kitrt_mn *mn, kitrt_work *out);

/* Copy the folded quadrature to host arrays (any may be NULL): weights [Q'], 2D directions
 * [Q' x 2], basis values [Q' x nmom]. */
int32_t kitrt_mn_quadrature(const kitrt_mn *mn, double *w, double *omega, double *m);

/* Isotropic closed form of the closure [Sec. 3.1, Eq. entropyOCP with the Maxwell-Boltzmann
 * entropy, whose minimiser is psi = exp(alpha.m)]: for u = (u_0, 0, ..., 0) the constant
 * psi = u_0 / (4 pi m_0) reproduces u (the other basis functions integrate to zero against a
 * constant), so alpha_0 = ln(u_0 / (4 pi m_0)) / m_0 and the other components are 0
 * (m_0 = 1/sqrt(4 pi)). Only u_0 of each row is read. u, alpha: device [C x n]; asynchronous on
 * `stream`. A row with u_0 <= 0 gets a non-finite alpha_0 (the closure then reports it). */
int32_t kitrt_isotropic_alpha(kitrt_mn *mn, const double *u, double *alpha, void *stream);

/* Entropy closure [Sec. 3.1, Eq. entropyOCP] of every cell: alpha minimises
 * <exp(alpha.m)> - alpha.u on the folded quadrature.
 *   u      device [C x n], read only.
 *   alpha  device [C x n]: warm start on input, solution on output (polished if enabled).
 *   status device [C] int32 per-cell status (0 = converged), or NULL.
 * Uses the solver's mode (FP64 or MIXED_*; LEARNED closes with its MLP first). Synchronises
 * with `stream` once per batch of Newton sweeps to test for completion. Returns the first
 * non-zero per-cell status found, else KITRT_OK. */
int32_t kitrt_closure(kitrt_mn *mn, const double *u, double *alpha, int32_t *status,
                      void *stream, kitrt_stats *stats);

/* Hessian of the dual's entropy part, H = <m m^T exp(alpha.m)> (a regularized solver's Newton
 * step adds reg_gamma on the regularized diagonal), of every cell at the given alpha, computed the
 * way the solver's closure computes it (FP64, or with the degree N+1..2N moments on tensor
 * cores in the mixed modes). alpha device [C x n]; H device [C x n x n] row-major, symmetric.
 * The first call allocates a [C x (2N+1)(2N+2)/2] moments buffer owned by the solver. */
int32_t kitrt_hessian(kitrt_mn *mn, const double *alpha, double *H, void *stream);

/* kitrt_closure for the first `ncells` rows only (ncells <= the mesh's cell count): closes any
 * batch of moment vectors that fits the solver's workspace, e.g. training data for the learned
 * closure. Same arguments and behaviour as kitrt_closure otherwise. */
int32_t kitrt_closure_batch(kitrt_mn *mn, const double *u, double *alpha, int32_t *status,
                            int32_t ncells, void *stream, kitrt_stats *stats);

/* The closed ansatz at the folded quadrature points: psi [C x Q'] FP64 device,
 * psi_cq = exp(alpha_c . m_q). */
int32_t kitrt_ansatz(kitrt_mn *mn, const double *alpha, double *psi, void *stream);

/* Forget the closure state kept for continuation (see kitrt_step): the next kitrt_step starts
 * every cell from the alpha it is given, whatever its contents. */
int32_t kitrt_mn_reset(kitrt_mn *mn);

/* nsteps explicit M_N steps, in place (order 1; with order 2 each step is the Heun scheme of
 * Sec. 4.3 described after the argument list):
 *   u^{n+1}_i = u^n_i - dt/A_i sum_{j in N(i)} F_up(psi_i, psi_j) + dt R_i(u^n_i),
 *   R_i(u) = -sigma_a,i u - sigma_s,i (u - u_0 e_0) + q_i <m>,
 * with F_up the kinetic upwind flux of the closed ansatz [Sec. 4.4] and psi the closure of u^n
 * [Sec. 4.2 explicit iteration; Sec. 3.1: isotropic scattering is diagonal in the moments].
 *   u       device [C x n]: u^0 in, u^{nsteps} out.
 *   alpha   device [C x n]: warm start in; out: closure of u^{nsteps-1} (the last closed state).
 *           Continuation is decided per cell by content: a cell whose given alpha row is, bit for
 *           bit, the alpha this solver returned for it from its last successful closure (and no
 *           kitrt_mn_reset came since) continues from the solver's stored state of that closure
 *           (the Newton predictor starts from the stored factor, as it does between the steps of
 *           one call), so that stepping one call at a time costs what one call of many steps
 *           costs. Every other cell, for instance one whose row the caller overwrote with a new
 *           warm start, starts from its given row. The result does not depend on the start
 *           beyond the closure tolerance: every closure is solved to the same tolerance.
 *   sigma_a, sigma_s, q  device [C] per-cell absorption, scattering, isotropic source.
 *   dt      time step; dt <= 0 selects cfl * min_i 2 A_i / P_i. The step must keep the kinetic
 *           update of every ordinate positive [Sec. 4.4: the updated moments must stay
 *           realizable]: dt (P_i / (2 A_i) + sigma_a,i + sigma_s,i) <= 1 in every cell (the
 *           cell-wise form of dt sigma_t,max <= 1 - CFL). The library tests this on the device
 *           and returns KITRT_EINVAL, before u is touched, when a cell violates it or has a
 *           negative or non-finite coefficient.
 *   status  device [C] or NULL: per-cell status of the last failed closure.
 * Order 2 [Sec. 4.3]: u* = u + dt L(u), u <- (u + u* + dt L(u*)) / 2, where L(v) closes v, builds
 * the ansatz, reconstructs it linearly in every cell at every quadrature point (Green-Gauss
 * gradient from face averages, Barth-Jespersen limiter with the two cells of each face as bounds,
 * so every face value lies between them) and applies the upwind flux of the face values plus
 * R(v); two closures per step (the second continues from the first).
 * Synchronises with `stream` once per step (closure completion test). On a closure failure the
 * step stops before updating u with that closure and returns its status. */
int32_t kitrt_step(kitrt_mn *mn, double *u, double *alpha, const double *sigma_a,
                   const double *sigma_s, const double *q, double dt, int32_t nsteps,
                   int32_t *status, void *stream, kitrt_stats *stats);

/* Heterogeneous density of the transformed CSD equation [Sec. 2, Eq. BoltzmannCSDTrafo]. After
 * the energy transform the CSD equation is a transport equation in the pseudo-time t (the
 * transformed energy) whose flux term is Omega . grad(psi / rho), rho(x) the tissue density, and
 * whose cross sections depend on t only. With a density set, every later first-order kitrt_step
 * of this solver transports psi / rho: the kinetic upwind flux takes psi_up / rho_up across each
 * face (psi_i / rho_i on outflow faces and for the Neumann ghost, 0 for the vacuum ghost); the
 * closure, the source term and the arrays sigma_a, sigma_s, q keep their meaning (for the CSD
 * equation the caller passes this pseudo-time step's Sigma_t - Sigma_s and Sigma_s in every cell).
 * The stability condition of kitrt_step becomes dt (P_i / (2 A_i rho_i) + sigma_a,i + sigma_s,i)
 * <= 1, and dt <= 0 still selects cfl * min_i 2 A_i / P_i, which the test then rejects where
 * rho < 1: pass dt explicitly.
 *   rho   device [C] FP64, every entry positive and finite; the solver keeps 1/rho (FP64 and FP32
 *         copies in its workspace, allocated on the first call). NULL removes the density.
 * KITRT_EINVAL when an entry is not positive and finite (the solver is then left without a
 * density). Synchronises with `stream`. While a density is set, kitrt_step with order 2,
 * kitrt_adjoint and kitrt_sn_step return KITRT_EINVAL. */
int32_t kitrt_mn_set_density(kitrt_mn *mn, const double *rho, void *stream);

/* Dose [Sec. 2: D(x) = 1/rho int int S(E, x) psi dOmega dE with S(E, x) = S_w(E) rho(x)] of one
 * explicit pseudo-time step. In the transformed variables psi~ = S_w rho psi and dE = S_w dE~,
 * so D = 1/rho int Phi~ S_w dE~ with Phi~ = int psi~ dOmega = u_0 / m_0; the step adds
 *   dose_i += dt * S * u_i0 / (m_0 rho_i)
 * (rho = 1 without a density), S the water stopping power S_w at this step's energy (the
 * caller's table: the ICRU data the paper uses are not part of the library).
 *   u     device [C x n] the state at the start of the step; dose device [C] FP64, accumulated.
 * Asynchronous on `stream`. KITRT_EINVAL for NULL pointers or non-finite S or dt. */
int32_t kitrt_dose_accumulate(kitrt_mn *mn, const double *u, double S, double dt, double *dose,
                              void *stream);

/* Entropy closure of a batch of moment vectors without any device allocation. The paper has no
 * counterpart: this entry point exists for callers that cannot let the library allocate device
 * memory at call time, for instance a framework whose pool allocator already owns the free device
 * memory (a cudaMalloc would fail or force the pool to release memory), or a long-running service
 * that must not grow its footprint after start-up, and whose batch is not the solver's mesh. It
 * runs the same FP64 Newton iteration as kitrt_closure with the solver's tables and parameters,
 * but keeps its per-cell Newton state in one static device array of 8 MiB that every GPU loading
 * the library holds until the process exits.
 *   u      device [ncells x nmom], read only; alpha device [ncells x nmom], warm start in,
 *          solution out; status device [ncells] or NULL.
 *   ncells may not exceed floor(8 MiB / per-cell bytes), where a cell needs
 *          8 (3 nmom + 4 + nmom (nmom+1)/2) + 28 bytes plus 256-byte padding of 16 arrays
 *          (about 11,300 cells for N = 3, 3,400 for N = 5); larger batches return
 *          KITRT_ESCRATCH before touching any memory.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture. Every call shares the
 * array and leaves its contents behind (the call clears the counters that must start at zero);
 * calls that overlap on the GPU (other streams or host threads) race on it. The call synchronises
 * with `stream` once every four Newton sweeps to test for completion (a 32-byte device-to-host
 * read of the counters) and, after a failure, to find the first failing cell. */
int32_t kitrt_closure_noalloc(const kitrt_mn *mn, const double *u, double *alpha,
                              int32_t *status, int32_t ncells, void *stream);

/* S_N steps of the nodal (discrete-ordinates) system [Sec. 2, Eq. SNEqns2]: explicit first-order
 * finite volumes [Sec. 4.2] with the upwind flux of Sec. 4.4 applied to every ordinate,
 *   psi'_iq = psi_iq - dt/A_i sum_f (Omega_q . n_if) psi_up - dt (sigma_a,i + sigma_s,i) psi_iq
 *             + dt (O Sigma_i M psi_i)_q + dt q_i,
 * on the solver's folded quadrature (kitrt_mn_quadrature; the +-mu ordinates of the 2D problem
 * are equal). The scattering is the P_N form of Eq. SNEqns2 truncated at the solver's degree N:
 * moment a of the ordinates, sum_q w_q m_a(Omega_q) psi_q, is scaled by sigma_s g_l(a) (l(a) the
 * degree of basis function a) and mapped back through m(Omega_q). Boundary faces take the
 * solver's boundary condition (Neumann: the cell's own ordinate; vacuum: 0). No closure is
 * involved; the solver handle supplies the mesh, the quadrature and the basis.
 *   psi      device [C x Q'] ordinates (Q' = nquad_folded of kitrt_mn_sizes, row-major, no
 *            padding), FP64, or FP32 when fp32 != 0; advanced in place by nsteps steps.
 *   work     device scratch of the same size and type, not overlapping psi.
 *   sigma_a, sigma_s, q  device [C] FP64 per-cell absorption, total scattering, isotropic source.
 *   g        host [N+1] Legendre coefficients of the scattering kernel relative to its total
 *            (g[0] must be 1; g_l = c^l is Henyey-Greenstein with asymmetry c), or NULL for
 *            isotropic scattering.
 *   dt       time step; dt <= 0 selects cfl * (smallest inradius).
 * Asynchronous on `stream` (nsteps launches, plus one device copy when nsteps is odd).
 * KITRT_EINVAL for NULL arguments, nsteps < 0, overlapping buffers, g[0] != 1 or a non-finite
 * g. */
int32_t kitrt_sn_step(kitrt_mn *mn, void *psi, void *work, int32_t fp32, const double *sigma_a,
                      const double *sigma_s, const double *q, const double *g, double dt,
                      int32_t nsteps, void *stream);

/* Discrete adjoint of nsteps FP64 steps (solver in KITRT_FP64 mode): the objective
 *   J = sum_{s=0}^{nsteps-1} dt sum_{i in target} A_i sigma_a,i u^s_i0 / m_0
 * (absorbed energy in the target cells; u_0/m_0 is the scalar flux <psi>) and its gradient with
 * respect to per-block absorption and scattering coefficients, by the exact transpose of the step
 * map (transposed upwind flux; closure derivative d alpha/d u = H^-1 from the implicit-function
 * theorem; source transpose). Not a construct of the paper: it differentiates the paper's step.
 *   u0, alpha0       device [C x n]: initial state and closure warm start (read only).
 *   sigma_a, sigma_s, q  device [C] per-cell coefficients (sigma_a,i = the value of its block).
 *   block_of_cell    device [C] int32 in [0, nblocks).
 *   target           device [C] uint8 (1 = cell in the target region).
 *   dt               time step (<= 0: cfl * min 2A/P); nsteps steps; ckpt_every >= 1 steps per
 *                    checkpoint segment (states are recomputed forward inside a segment).
 *   J                host [1]; dJ_dsa, dJ_dss host [nblocks] (overwritten).
 * The first call (or one needing more than the last) allocates the checkpoint and segment buffers
 * in the solver's workspace (about (nsteps/ckpt_every + 2 ckpt_every + 4) C n doubles + C Q'
 * doubles); later calls reuse them and allocate nothing; kitrt_mn_destroy frees them. Checks the
 * stability condition of kitrt_step (KITRT_EINVAL) and synchronises with `stream` before
 * returning. */
int32_t kitrt_adjoint(kitrt_mn *mn, const double *u0, const double *alpha0, const double *sigma_a,
                      const double *sigma_s, const double *q, const int32_t *block_of_cell,
                      int32_t nblocks, const uint8_t *target, double dt, int32_t nsteps,
                      int32_t ckpt_every, double *J, double *dJ_dsa, double *dJ_dss, void *stream);

/* ---- Halo exchange of a step split over ranks [Sec. 6: the cells are split over parallel
 * workers] ------------------------------------------------------------------------------------
 * A rank steps its own cells plus halo layers of its neighbours' cells (a mesh built from those
 * triangles); before each step the halo rows of u are refreshed from their owners. These two
 * calls pack and unpack the rows (device memory, asynchronous on `stream`); the transport between
 * ranks is the caller's (e.g. point-to-point sends). EINVAL for count < 0, width < 1 or a NULL
 * pointer with count > 0; indices are not range-checked. */
/* dst [count x width] row k = src row idx[k] (src [* x width] row-major, idx device int32). */
int32_t kitrt_gather_rows(const double *src, const int32_t *idx, int32_t count, int32_t width,
                          double *dst, void *stream);
/* dst row idx[k] = src [count x width] row k. */
int32_t kitrt_scatter_rows(const double *src, const int32_t *idx, int32_t count, int32_t width,
                           double *dst, void *stream);
/* dst row idx[k] += src [count x width] row k: the adjoint's reverse halo (the transpose of the
 * halo exchange), adding the contributions other ranks computed for this rank's cells. The
 * indices of one call must be distinct. */
int32_t kitrt_scatter_add_rows(const double *src, const int32_t *idx, int32_t count, int32_t width,
                               double *dst, void *stream);

/* ---- Learned closure [Sec. 3.1: neural entropy closures replace the Newton solve] --------------
 * A plain MLP with three softplus hidden layers maps the normalised moments v = u_{1..n-1}/u_0
 * (standardised) to alpha_{1..n-1} of the normalised problem (also standardised). Parameters are
 * FP32, packed W1[din x H] b1[H] W2[H x H] b2[H] W3[H x H] b3[H] W4[H x dout] b4[dout]
 * (row-major [in x out]). Training runs on the library's own kernels; all pointers are device
 * memory and calls are asynchronous on `stream`. */

/* Number of packed parameters. */
int32_t kitrt_mlp_param_count(int32_t din, int32_t hidden, int32_t dout);
/* Floats of caller-provided workspace that kitrt_mlp_forward / kitrt_mlp_loss_grad need for a
 * batch of B rows: B (8 hidden + 2 dout). */
int32_t kitrt_mlp_work_floats(int32_t B, int32_t hidden, int32_t dout);
/* Y [B x dout] = network(X [B x din]) in FP32. */
int32_t kitrt_mlp_forward(int32_t din, int32_t hidden, int32_t dout, const float *params,
                          const float *X, float *Y, int32_t B, float *work, void *stream);
/* Mean-squared loss 1/(2B) sum ||Y - T||^2 into *loss (device float) and its gradient with
 * respect to the packed parameters into grad [param_count] (both overwritten). */
int32_t kitrt_mlp_loss_grad(int32_t din, int32_t hidden, int32_t dout, const float *params,
                            const float *X, const float *T, int32_t B, float *grad, float *loss,
                            float *work, void *stream);
/* One Adam step (Kingma & Ba) at step count t >= 1 over P parameters; m and v are the moment
 * buffers (zero before the first step). */
int32_t kitrt_mlp_adam(int32_t P, float *params, const float *grad, float *m, float *v, int32_t t,
                       float lr, float beta1, float beta2, float eps, void *stream);
/* Attach a trained network to a KITRT_LEARNED solver (hidden must be 64, din = dout = nmom - 1):
 * params FP32 as above (converted to BF16 for inference), norm [4 (nmom-1)] FP32 =
 * (feature means, feature scales, output means, output scales). Allocates its copy on first use. */
int32_t kitrt_mn_set_mlp(kitrt_mn *mn, const float *params, const float *norm, int32_t hidden,
                         void *stream);
/* Moments u [count x nmom] (FP64) of mixtures of von Mises-Fisher densities on S^2 integrated
 * with the solver's quadrature: centres [count x lobes x 3] (unit vectors, (x, y, mu) order),
 * kappa and weight [count x lobes] (weight 0 = unused lobe). Training data for the network. */
int32_t kitrt_vmf_moments(kitrt_mn *mn, const double *centres, const double *kappa,
                          const double *weight, int32_t lobes, int32_t count, double *u,
                          void *stream);

/* Tracing: on != 0 resets the trace and records a pair of CUDA events on the launching stream
 * around every kernel the solver launches from then on; on == 0 stops recording. */
int32_t kitrt_profile_enable(kitrt_mn *mn, int32_t on);

/* Read the trace (synchronises with the recorded events): up to max_entries records, one per
 * kernel kind that ran, into `out` (host); *n_entries receives the number written. */
int32_t kitrt_profile_read(kitrt_mn *mn, kitrt_profile_entry *out, int32_t max_entries,
                           int32_t *n_entries);

#ifdef __cplusplus
}
#endif

#endif /* KITRT_H */
