/*
 * CPU oracle for the M_N (minimal-entropy moment) step of KiT-RT (arXiv 2205.08417).
 *
 * TEST INFRASTRUCTURE ONLY. This file is a plain, slow, obviously-correct FP64 restatement of the
 * paper's method, used to judge the CUDA path. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it. It shares no code, header, table or constant with the
 * CUDA library, and the CUDA library never calls it.
 *
 * Contents (paper sections in brackets):
 *   - Gauss-Legendre rule and the tensorised Gauss-Legendre x uniform-azimuth quadrature on S^2,
 *     projected to the 2D slab geometry [Sec. 3.2, Eq. spherical-coordinatesProduct].
 *   - Real spherical-harmonic basis m_l^k, normalised on S^2, ordered by l then k [Sec. 3.1];
 *     in 2D only the functions even in mu (l+k even) are kept.
 *   - Cell-centred triangle geometry: areas A_i, neighbours N(i), scaled normals n_ij [Sec. 4.1].
 *   - Entropy closure [Sec. 3.1, Eq. entropyOCP] with the Maxwell-Boltzmann entropy, solved
 *     through its dual f(alpha) = <exp(alpha.m)> - alpha.u by damped Newton with an Armijo line
 *     search [Sec. 7.2 M_N run: "Newton optimizer with line search"]; optionally (partially)
 *     regularized [Sec. 3.1, Eq. entropyOCP_reg, Eq. entropyOCP_part_reg].
 *   - Kinetic upwind flux of the closed ansatz [Sec. 4.4, last flux equation] and the explicit
 *     first-order update [Sec. 4.2, explicit iteration] with isotropic scattering, absorption and
 *     an isotropic source [Sec. 3.1 moment equations: scattering diagonal in moments].
 *   - Discrete adjoint of that step (exact transpose, closure derivative dalpha/du = H^-1), and
 *     the one-step tangent written separately in forward mode (for the transpose test).
 *   - The second-order scheme [Sec. 4.3]: Green-Gauss gradient, Barth-Jespersen limiter,
 *     reconstructed ordinates as the inputs of the kinetic upwind flux, Heun time stepping.
 *   - The S_N step of the nodal system [Sec. 2, Eq. SNEqns2] with the P_N form O Sigma M of the
 *     scattering operator and the same upwind flux applied per ordinate.
 *   - Plain MLP (softplus) forward/backward and Adam, for the learned-closure gradient checks.
 *
 * Quadrature sums here always run over the full, unfolded point set Q; the CUDA path folds the
 * +-mu pairs, so agreement also tests that fold.
 *
 * Build: gcc -O3 -std=c99 -fPIC -shared [-fopenmp] kitrt_oracle.c -lm (ISO C mode: no floating-point
 * contraction, so x86-64 and aarch64 hosts round identically).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------------ */
/* Quadrature [Sec. 3.2]                                                                      */
/* ------------------------------------------------------------------------------------------ */

/* Gauss-Legendre nodes x (ascending) and weights w on [-1,1]: Newton's method on P_n using the
 * three-term Legendre recurrence; w = 2 / ((1 - x^2) P_n'(x)^2). */
void orc_gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            if (n == 0) p1 = 1.0;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_n(z), p0 = P_{n-1}(z) */
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute derivative at the final node */
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Number of quadrature points of the product rule of a given order: order Gauss points in mu
 * times 2*order equally spaced azimuths. */
int orc_quad_count(int order) { return 2 * order * order; }

/* Product rule: mu_k Gauss-Legendre (k = 0..order-1), phi_l = l * 2pi/Nphi (l = 1..Nphi),
 * Nphi = 2*order, w = w^G_k * 2pi / Nphi, index q = k*Nphi + (l-1).
 * Outputs the 2D projected direction Omega = (sqrt(1-mu^2) sin phi, sqrt(1-mu^2) cos phi). */
void orc_quadrature(int order, double *mu, double *phi, double *w, double *ox, double *oy)
{
    int nmu = order, nphi = 2 * order;
    double *gx = (double *)malloc(sizeof(double) * nmu);
    double *gw = (double *)malloc(sizeof(double) * nmu);
    orc_gauss_legendre(nmu, gx, gw);
    for (int k = 0; k < nmu; ++k)
        for (int l = 1; l <= nphi; ++l) {
            int q = k * nphi + (l - 1);
            double p = l * (2.0 * ORC_PI / nphi);
            double s = sqrt(1.0 - gx[k] * gx[k]);
            mu[q] = gx[k];
            phi[q] = p;
            w[q] = gw[k] * 2.0 * ORC_PI / nphi;
            ox[q] = s * sin(p);
            oy[q] = s * cos(p);
        }
    free(gx);
    free(gw);
}

/* ------------------------------------------------------------------------------------------ */
/* Real spherical harmonics [Sec. 3.1]                                                        */
/* ------------------------------------------------------------------------------------------ */

int orc_nmom(int N) { return (N + 1) * (N + 2) / 2; }

/* Associated Legendre function P_l^k(mu), k >= 0, without the Condon-Shortley phase:
 * P_k^k = (2k-1)!! (1-mu^2)^(k/2), P_{k+1}^k = (2k+1) mu P_k^k,
 * (l-k) P_l^k = (2l-1) mu P_{l-1}^k - (l+k-1) P_{l-2}^k. */
static double orc_assoc_legendre(int l, int k, double mu)
{
    double s = sqrt(1.0 - mu * mu);
    double pkk = 1.0;
    for (int i = 1; i <= k; ++i) pkk *= (2.0 * i - 1.0) * s;
    if (l == k) return pkk;
    double pk1 = (2.0 * k + 1.0) * mu * pkk;
    if (l == k + 1) return pk1;
    double a = pkk, b = pk1, c = 0.0;
    for (int ll = k + 2; ll <= l; ++ll) {
        c = ((2.0 * ll - 1.0) * mu * b - (ll + k - 1.0) * a) / (ll - k);
        a = b;
        b = c;
    }
    return c;
}

static double orc_factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

/* Basis vector m(mu,phi) of degree N for the 2D slab: all m_l^k with l <= N and l+k even,
 * ordered by l ascending then k ascending. Normalisation N_l^k = sqrt((2l+1)/(4pi) (l-k)!/(l+k)!):
 *   m_l^0 = N_l^0 P_l, m_l^k = sqrt2 N_l^k P_l^k cos(k phi) (k>0),
 *   m_l^k = sqrt2 N_l^|k| P_l^|k| sin(|k| phi) (k<0). */
void orc_basis(int N, double mu, double phi, double *m)
{
    int idx = 0;
    for (int l = 0; l <= N; ++l)
        for (int k = -l; k <= l; ++k) {
            int ak = k < 0 ? -k : k;
            if (((l + ak) & 1) != 0) continue;
            double nlk = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * orc_factorial(l - ak) /
                              orc_factorial(l + ak));
            double p = orc_assoc_legendre(l, ak, mu);
            double v;
            if (k == 0)
                v = nlk * p;
            else if (k > 0)
                v = sqrt(2.0) * nlk * p * cos(k * phi);
            else
                v = sqrt(2.0) * nlk * p * sin(ak * phi);
            m[idx++] = v;
        }
}

/* Full tables on the product quadrature: M[q*n + a] = m_a(Omega_q), plus w, Omega. */
void orc_tables(int N, int order, double *M, double *w, double *ox, double *oy)
{
    int Q = orc_quad_count(order), n = orc_nmom(N);
    double *mu = (double *)malloc(sizeof(double) * Q);
    double *phi = (double *)malloc(sizeof(double) * Q);
    orc_quadrature(order, mu, phi, w, ox, oy);
    for (int q = 0; q < Q; ++q) orc_basis(N, mu[q], phi[q], M + (size_t)q * n);
    free(mu);
    free(phi);
}

/* ------------------------------------------------------------------------------------------ */
/* Mesh geometry [Sec. 4.1]                                                                   */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int a, b, cell, face;
} orc_edge;

static int orc_edge_cmp(const void *x, const void *y)
{
    const orc_edge *e = (const orc_edge *)x, *f = (const orc_edge *)y;
    if (e->a != f->a) return e->a < f->a ? -1 : 1;
    if (e->b != f->b) return e->b < f->b ? -1 : 1;
    if (e->cell != f->cell) return e->cell < f->cell ? -1 : 1;
    return 0;
}

/* For each triangle (vertices taken counter-clockwise; clockwise input is reversed), face k is the
 * edge from vertex k to vertex k+1. Outputs: area[c], perim[c], cen[2c..], nbr[3c+k] (neighbour
 * cell across face k or -1 on the boundary) and nrm[6c+2k..] = outward normal of face k scaled by
 * the face length. Returns 0, or -1 if a cell has non-positive area or an edge is shared by more
 * than two cells. */
int orc_mesh_geometry(int nv, const double *xy, int nc, const int32_t *tri, double *area,
                      double *perim, double *cen, int32_t *nbr, double *nrm)
{
    (void)nv;
    orc_edge *edges = (orc_edge *)malloc(sizeof(orc_edge) * (size_t)nc * 3);
    int rc = 0;
    for (int c = 0; c < nc; ++c) {
        int v[3] = {tri[3 * c], tri[3 * c + 1], tri[3 * c + 2]};
        double x0 = xy[2 * v[0]], y0 = xy[2 * v[0] + 1];
        double x1 = xy[2 * v[1]], y1 = xy[2 * v[1] + 1];
        double x2 = xy[2 * v[2]], y2 = xy[2 * v[2] + 1];
        double cr = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
        if (cr < 0) {
            int t = v[1];
            v[1] = v[2];
            v[2] = t;
            cr = -cr;
        }
        if (!(cr > 0)) rc = -1;
        area[c] = 0.5 * cr;
        cen[2 * c] = (xy[2 * v[0]] + xy[2 * v[1]] + xy[2 * v[2]]) / 3.0;
        cen[2 * c + 1] = (xy[2 * v[0] + 1] + xy[2 * v[1] + 1] + xy[2 * v[2] + 1]) / 3.0;
        double p = 0.0;
        for (int k = 0; k < 3; ++k) {
            int a = v[k], b = v[(k + 1) % 3];
            double ax = xy[2 * a], ay = xy[2 * a + 1], bx = xy[2 * b], by = xy[2 * b + 1];
            /* edge a->b of a counter-clockwise triangle: outward normal (dy, -dx) */
            nrm[6 * c + 2 * k] = by - ay;
            nrm[6 * c + 2 * k + 1] = ax - bx;
            p += sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
            orc_edge e;
            e.a = a < b ? a : b;
            e.b = a < b ? b : a;
            e.cell = c;
            e.face = k;
            edges[3 * c + k] = e;
            nbr[3 * c + k] = -1;
        }
        perim[c] = p;
    }
    qsort(edges, (size_t)nc * 3, sizeof(orc_edge), orc_edge_cmp);
    size_t ne = (size_t)nc * 3;
    for (size_t i = 0; i < ne;) {
        size_t j = i + 1;
        while (j < ne && edges[j].a == edges[i].a && edges[j].b == edges[i].b) ++j;
        if (j - i == 2) {
            orc_edge e = edges[i], f = edges[i + 1];
            nbr[3 * e.cell + e.face] = f.cell;
            nbr[3 * f.cell + f.face] = e.cell;
        } else if (j - i > 2) {
            rc = -1;
        }
        i = j;
    }
    free(edges);
    return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Entropy closure [Sec. 3.1, Eq. entropyOCP]                                                 */
/* ------------------------------------------------------------------------------------------ */

enum { ORC_OK = 0, ORC_MAXITER = 1, ORC_CHOL = 2, ORC_LINESEARCH = 3, ORC_NONFINITE = 4 };

typedef struct {
    double tau;       /* stop when ||g||_2 <= tau ||u||_2 */
    int max_iter;     /* Newton iterations */
    int max_halvings; /* Armijo backtracking halvings per iteration */
    double c1;        /* Armijo constant */
    int polish;       /* one extra full Newton step after the test passes */
    double gamma;     /* regularization parameter (0: the entropy closure itself) */
    int reg0;         /* first regularized moment: 0 (all, Eq. entropyOCP_reg) or 1 (u_0 kept
                         exact, Eq. entropyOCP_part_reg) */
} orc_newton_opts;

/* Dual objective and its derivatives at alpha over the full quadrature:
 *   f = sum_q w_q exp(alpha.m_q) - alpha.u,  g = sum_q w_q e_q m_q - u,
 *   H = sum_q w_q e_q m_q m_q^T (full n x n). fmag = sum_q w_q e_q + |alpha.u| bounds the size of
 * the terms in f (used as round-off slack). Any pointer may be NULL. */
static void orc_dual_eval(int n, int Q, const double *M, const double *w, const double *u,
                          const double *alpha, double *f, double *g, double *H, double *fmag)
{
    double s = 0.0;
    if (g)
        for (int a = 0; a < n; ++a) g[a] = 0.0;
    if (H)
        for (int a = 0; a < n * n; ++a) H[a] = 0.0;
    for (int q = 0; q < Q; ++q) {
        const double *m = M + (size_t)q * n;
        double z = 0.0;
        for (int a = 0; a < n; ++a) z += alpha[a] * m[a];
        double we = w[q] * exp(z);
        s += we;
        if (g)
            for (int a = 0; a < n; ++a) g[a] += we * m[a];
        if (H)
            for (int a = 0; a < n; ++a)
                for (int b = 0; b < n; ++b) H[a * n + b] += we * m[a] * m[b];
    }
    double au = 0.0;
    for (int a = 0; a < n; ++a) au += alpha[a] * u[a];
    if (g)
        for (int a = 0; a < n; ++a) g[a] -= u[a];
    if (f) *f = s - au;
    if (fmag) *fmag = s + fabs(au);
}

/* The (partially) regularized closure [Sec. 3.1, Eq. entropyOCP_reg and Eq. entropyOCP_part_reg]:
 * the primal adds 1/(2 gamma) ||<m^r g> - u^r||^2 to the entropy (r = the regularized moments)
 * and drops their moment constraints. Eliminating the slack v = <m^r g> - u^r from the
 * Lagrangian, min_v ||v||^2 / (2 gamma) + alpha^r . v = -gamma ||alpha^r||^2 / 2, so the dual to
 * minimise becomes
 *   f(alpha) = <exp(alpha.m)> - alpha.u + gamma/2 ||alpha^r||^2,
 *   g = <m e> - u + gamma alpha^r,   H = <m m^T e> + gamma I_r,
 * and the regularized ansatz exp(alpha.m) has moments <m^r psi> = u^r - gamma alpha^r. Adds the
 * regularization terms to f, g, H, fmag (any may be NULL) at alpha; r = {reg0, ..., n-1}. */
static void orc_dual_regularize(int n, double gamma, int reg0, const double *alpha, double *f,
                                double *g, double *H, double *fmag)
{
    if (gamma == 0.0) return;
    double a2 = 0.0;
    for (int a = reg0; a < n; ++a) a2 += alpha[a] * alpha[a];
    if (f) *f += 0.5 * gamma * a2;
    if (fmag) *fmag += 0.5 * gamma * a2;
    if (g)
        for (int a = reg0; a < n; ++a) g[a] += gamma * alpha[a];
    if (H)
        for (int a = reg0; a < n; ++a) H[a * n + a] += gamma;
}

/* Cholesky H = L L^T (L lower, row-major in L[a*n+b], b <= a). Returns 0 or -1 on a
 * non-positive pivot. */
static int orc_cholesky(int n, const double *H, double *L)
{
    for (int a = 0; a < n * n; ++a) L[a] = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = H[j * n + j];
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (!(d > 0.0)) return -1;
        double ljj = sqrt(d);
        L[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = H[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = s / ljj;
        }
    }
    return 0;
}

/* Solve L L^T x = b. */
static void orc_chol_solve(int n, const double *L, const double *b, double *x)
{
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * x[k];
        x[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
}

static int orc_finite(int n, const double *v)
{
    for (int a = 0; a < n; ++a)
        if (!isfinite(v[a])) return 0;
    return 1;
}

/* Newton's method on the dual with Armijo backtracking:
 *   d = -H^-1 g (Cholesky); accept lambda when
 *   f(alpha + lambda d) <= f(alpha) + c1 lambda g.d + 64 eps fmag   (round-off slack),
 *   halving lambda from 1; stop when ||g|| <= tau ||u||; then optionally one polish step
 *   alpha <- alpha - H^-1 g at the converged point. alpha is the warm start on input.
 * Returns a status code; *iters = Newton iterations taken (polish excluded). */
int orc_closure_solve(int n, int Q, const double *M, const double *w, const double *u,
                      double *alpha, const orc_newton_opts *o, int *iters)
{
    double g[64], H[64 * 64], L[64 * 64], d[64], at[64];
    double f, fmag, ft;
    double un = 0.0;
    for (int a = 0; a < n; ++a) un += u[a] * u[a];
    un = sqrt(un);
    int it = 0;
    if (iters) *iters = 0;
    orc_dual_eval(n, Q, M, w, u, alpha, &f, g, H, &fmag);
    orc_dual_regularize(n, o->gamma, o->reg0, alpha, &f, g, H, &fmag);
    for (;;) {
        if (!isfinite(f) || !orc_finite(n, g)) return ORC_NONFINITE;
        double gn = 0.0;
        for (int a = 0; a < n; ++a) gn += g[a] * g[a];
        gn = sqrt(gn);
        if (orc_cholesky(n, H, L) != 0) return ORC_CHOL;
        orc_chol_solve(n, L, g, d);
        for (int a = 0; a < n; ++a) d[a] = -d[a];
        if (gn <= o->tau * un) {
            if (o->polish)
                for (int a = 0; a < n; ++a) alpha[a] += d[a];
            if (iters) *iters = it;
            return ORC_OK;
        }
        if (it >= o->max_iter) return ORC_MAXITER;
        double gd = 0.0;
        for (int a = 0; a < n; ++a) gd += g[a] * d[a];
        double lam = 1.0;
        int accepted = 0;
        for (int h = 0; h <= o->max_halvings; ++h) {
            for (int a = 0; a < n; ++a) at[a] = alpha[a] + lam * d[a];
            orc_dual_eval(n, Q, M, w, u, at, &ft, NULL, NULL, NULL);
            orc_dual_regularize(n, o->gamma, o->reg0, at, &ft, NULL, NULL, NULL);
            if (isfinite(ft) && ft <= f + o->c1 * lam * gd + 64.0 * 2.220446049250313e-16 * fmag) {
                accepted = 1;
                break;
            }
            lam *= 0.5;
        }
        if (!accepted) return ORC_LINESEARCH;
        for (int a = 0; a < n; ++a) alpha[a] = at[a];
        ++it;
        orc_dual_eval(n, Q, M, w, u, alpha, &f, g, H, &fmag);
        orc_dual_regularize(n, o->gamma, o->reg0, alpha, &f, g, H, &fmag);
    }
}

/* Batch closure over C cells (u, alpha row-major [C x n]), regularized with (gamma, reg0) as in
 * orc_dual_regularize (gamma = 0: the entropy closure). status[c] gets the code; returns the
 * number of failed cells. iters may be NULL. */
int orc_closure_batch_reg(int C, int n, int Q, const double *M, const double *w, const double *u,
                          double *alpha, double tau, int max_iter, int max_halvings, double c1,
                          int polish, double gamma, int reg0, int nthreads, int32_t *status,
                          int32_t *iters)
{
    orc_newton_opts o = {tau, max_iter, max_halvings, c1, polish, gamma, reg0};
    int nfail = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nfail)
#endif
    for (int c = 0; c < C; ++c) {
        int it = 0;
        int st = orc_closure_solve(n, Q, M, w, u + (size_t)c * n, alpha + (size_t)c * n, &o, &it);
        if (status) status[c] = st;
        if (iters) iters[c] = it;
        if (st != ORC_OK) ++nfail;
    }
    (void)nthreads;
    return nfail;
}

/* The entropy closure of every cell (no regularization). */
int orc_closure_batch(int C, int n, int Q, const double *M, const double *w, const double *u,
                      double *alpha, double tau, int max_iter, int max_halvings, double c1,
                      int polish, int nthreads, int32_t *status, int32_t *iters)
{
    return orc_closure_batch_reg(C, n, Q, M, w, u, alpha, tau, max_iter, max_halvings, c1, polish,
                                 0.0, 1, nthreads, status, iters);
}

/* Isotropic closed form of the closure: psi = u_0 / (4 pi m_0) constant, so
 * alpha_0 = ln(u_0 / (4 pi m_0)) / m_0 and all other components vanish. */
void orc_isotropic_alpha(int C, int n, double m0, const double *u, double *alpha)
{
    for (int c = 0; c < C; ++c) {
        for (int a = 0; a < n; ++a) alpha[(size_t)c * n + a] = 0.0;
        alpha[(size_t)c * n] = log(u[(size_t)c * n] / (4.0 * ORC_PI * m0)) / m0;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Kinetic upwind flux and explicit update [Sec. 4.2, Sec. 4.4]                               */
/* ------------------------------------------------------------------------------------------ */

/* psi[c*Q + q] = exp(alpha_c . m_q): the closed ansatz at every quadrature point. */
void orc_ansatz(int C, int n, int Q, const double *M, const double *alpha, double *psi,
                int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int c = 0; c < C; ++c)
        for (int q = 0; q < Q; ++q) {
            double z = 0.0;
            for (int a = 0; a < n; ++a) z += alpha[(size_t)c * n + a] * M[(size_t)q * n + a];
            psi[(size_t)c * Q + q] = exp(z);
        }
    (void)nthreads;
}

/* Kinetic flux sum F_i = sum_{faces k} sum_q w_q m_q (Omega_q . n_ik)
 *                       [psi_iq H(Omega_q . n_ik) + psi_jq (1 - H(Omega_q . n_ik))]
 * with j the neighbour across face k. On a boundary face the outside value is psi_iq (bc = 0,
 * Neumann: zero-gradient ghost) or 0 (bc = 1, Dirichlet vacuum). H(0) = 0.
 * Then u_i <- u_i - dt/A_i F_i + dt R_i with
 *   R_i = -sigma_a u_i - sigma_s (u_i - u_i0 e_0) + qsrc_i <m>   (<m> = sum_q w_q m_q).
 * u is updated in place (the flux reads psi only). sigma_a, sigma_s, qsrc are per cell. */
void orc_flux_update(int C, int n, int Q, const double *M, const double *w, const double *ox,
                     const double *oy, const int32_t *nbr, const double *nrm, const double *area,
                     const double *psi, const double *sigma_a, const double *sigma_s,
                     const double *qsrc, double dt, int bc, double *u, int nthreads)
{
    double mbar[64];
    for (int a = 0; a < n; ++a) {
        mbar[a] = 0.0;
        for (int q = 0; q < Q; ++q) mbar[a] += w[q] * M[(size_t)q * n + a];
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int i = 0; i < C; ++i) {
        double F[64];
        for (int a = 0; a < n; ++a) F[a] = 0.0;
        for (int k = 0; k < 3; ++k) {
            int j = nbr[3 * i + k];
            double nx = nrm[6 * i + 2 * k], ny = nrm[6 * i + 2 * k + 1];
            for (int q = 0; q < Q; ++q) {
                double dot = ox[q] * nx + oy[q] * ny;
                double up;
                if (dot > 0.0)
                    up = psi[(size_t)i * Q + q];
                else if (j >= 0)
                    up = psi[(size_t)j * Q + q];
                else
                    up = (bc == 0) ? psi[(size_t)i * Q + q] : 0.0;
                double s = w[q] * dot * up;
                for (int a = 0; a < n; ++a) F[a] += s * M[(size_t)q * n + a];
            }
        }
        double *ui = u + (size_t)i * n;
        double u0 = ui[0];
        for (int a = 0; a < n; ++a) {
            double R = -sigma_a[i] * ui[a] - sigma_s[i] * (ui[a] - (a == 0 ? u0 : 0.0)) +
                       qsrc[i] * mbar[a];
            ui[a] = ui[a] - dt / area[i] * F[a] + dt * R;
        }
    }
    (void)nthreads;
}

/* ------------------------------------------------------------------------------------------ */
/* Heterogeneous density of the CSD equation in pseudo-time [Sec. 2, Eq. BoltzmannCSDTrafo]      */
/* ------------------------------------------------------------------------------------------ */

/* The transformed CSD equation transports psi / rho(x): its flux term is Omega . grad(psi / rho),
 * with rho the tissue density per cell, and its cross sections depend on the pseudo-time only.
 * So the kinetic flux of the step is orc_flux_update's with the upwind value psi_up / rho_up
 * (the cell's own psi_i / rho_i on an outflow face; across a face the neighbour's psi_j / rho_j;
 * on a boundary face psi_i / rho_i (Neumann) or 0 (vacuum)); the update and source are
 * unchanged (sigma_a, sigma_s per cell carry Sigma_t - Sigma_s and Sigma_s at this pseudo-time). */
void orc_flux_update_rho(int C, int n, int Q, const double *M, const double *w, const double *ox,
                         const double *oy, const int32_t *nbr, const double *nrm,
                         const double *area, const double *rho, const double *psi,
                         const double *sigma_a, const double *sigma_s, const double *qsrc,
                         double dt, int bc, double *u, int nthreads)
{
    double mbar[64];
    for (int a = 0; a < n; ++a) {
        mbar[a] = 0.0;
        for (int q = 0; q < Q; ++q) mbar[a] += w[q] * M[(size_t)q * n + a];
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int i = 0; i < C; ++i) {
        double F[64];
        for (int a = 0; a < n; ++a) F[a] = 0.0;
        for (int k = 0; k < 3; ++k) {
            int j = nbr[3 * i + k];
            double nx = nrm[6 * i + 2 * k], ny = nrm[6 * i + 2 * k + 1];
            for (int q = 0; q < Q; ++q) {
                double dot = ox[q] * nx + oy[q] * ny;
                double up;
                if (dot > 0.0)
                    up = psi[(size_t)i * Q + q] / rho[i];
                else if (j >= 0)
                    up = psi[(size_t)j * Q + q] / rho[j];
                else
                    up = (bc == 0) ? psi[(size_t)i * Q + q] / rho[i] : 0.0;
                double s = w[q] * dot * up;
                for (int a = 0; a < n; ++a) F[a] += s * M[(size_t)q * n + a];
            }
        }
        double *ui = u + (size_t)i * n;
        double u0 = ui[0];
        for (int a = 0; a < n; ++a) {
            double R = -sigma_a[i] * ui[a] - sigma_s[i] * (ui[a] - (a == 0 ? u0 : 0.0)) +
                       qsrc[i] * mbar[a];
            ui[a] = ui[a] - dt / area[i] * F[a] + dt * R;
        }
    }
    (void)nthreads;
}

/* nsteps first-order M_N steps of the transformed CSD equation with density rho per cell. */
int orc_mn_run_rho(int C, int n, int Q, const double *M, const double *w, const double *ox,
                   const double *oy, const int32_t *nbr, const double *nrm, const double *area,
                   const double *rho, const double *sigma_a, const double *sigma_s,
                   const double *qsrc, double dt, int bc, int nsteps, double tau, int max_iter,
                   int polish, int nthreads, double *u, double *alpha, int32_t *status)
{
    double *psi = (double *)malloc(sizeof(double) * (size_t)C * Q);
    int nfail = 0;
    for (int s = 0; s < nsteps; ++s) {
        nfail += orc_closure_batch_reg(C, n, Q, M, w, u, alpha, tau, max_iter, 30, 1e-4, polish,
                                       0.0, 1, nthreads, status, NULL);
        orc_ansatz(C, n, Q, M, alpha, psi, nthreads);
        orc_flux_update_rho(C, n, Q, M, w, ox, oy, nbr, nrm, area, rho, psi, sigma_a, sigma_s,
                            qsrc, dt, bc, u, nthreads);
    }
    free(psi);
    return nfail;
}

/* Dose [Sec. 2]: D(x) = 1/rho int_E int_S2 S(E, x) psi dOmega dE with S(E, x) = S_w(E) rho(x)
 * (water-equivalent tissue). In the transformed variables psi~ = S_w rho psi and
 * dE = S_w(E(E~)) dE~, so D = 1/rho int Phi~(E~) S_w(E(E~)) dE~ with Phi~ = int psi~ dOmega =
 * u_0 / m_0. One explicit pseudo-time step of length dt at stopping power S adds
 * dt S u_i0 / (m_0 rho_i) to cell i (left endpoint rule). */
void orc_dose_accumulate(int C, int n, double m0, const double *u, const double *rho, double S,
                         double dt, double *dose)
{
    for (int i = 0; i < C; ++i) dose[i] += dt * S * (u[(size_t)i * n] / m0) / rho[i];
}

/* ------------------------------------------------------------------------------------------ */
/* Second-order scheme [Sec. 4.3]: linear reconstruction with the Green-Gauss gradient and the   */
/* Barth-Jespersen limiter, second-order upwind (kinetic) flux, Heun time stepping              */
/* ------------------------------------------------------------------------------------------ */

/* Offsets r_ik from the centroid of cell i to the midpoint of its face k (same orientation and
 * face order as orc_mesh_geometry: counter-clockwise, face k from vertex k to vertex k+1). */
void orc_mesh_face_offsets(int nv, const double *xy, int nc, const int32_t *tri, double *r)
{
    (void)nv;
    for (int c = 0; c < nc; ++c) {
        int v[3] = {tri[3 * c], tri[3 * c + 1], tri[3 * c + 2]};
        double cr = (xy[2 * v[1]] - xy[2 * v[0]]) * (xy[2 * v[2] + 1] - xy[2 * v[0] + 1]) -
                    (xy[2 * v[2]] - xy[2 * v[0]]) * (xy[2 * v[1] + 1] - xy[2 * v[0] + 1]);
        if (cr < 0) {
            int t = v[1];
            v[1] = v[2];
            v[2] = t;
        }
        double cx = (xy[2 * v[0]] + xy[2 * v[1]] + xy[2 * v[2]]) / 3.0;
        double cy = (xy[2 * v[0] + 1] + xy[2 * v[1] + 1] + xy[2 * v[2] + 1]) / 3.0;
        for (int k = 0; k < 3; ++k) {
            int a = v[k], b = v[(k + 1) % 3];
            r[6 * c + 2 * k] = 0.5 * (xy[2 * a] + xy[2 * b]) - cx;
            r[6 * c + 2 * k + 1] = 0.5 * (xy[2 * a + 1] + xy[2 * b + 1]) - cy;
        }
    }
}

/* Value of ordinate q of the cell across face k of cell i: the neighbour's cell value, or the
 * boundary ghost (Neumann: the cell's own value; vacuum: 0). */
static double orc_across(const int32_t *nbr, int Q, const double *psi, int bc, int i, int k, int q)
{
    int j = nbr[3 * i + k];
    if (j >= 0) return psi[(size_t)j * Q + q];
    return bc == 0 ? psi[(size_t)i * Q + q] : 0.0;
}

/* Reconstruction of the ordinate values psi [C x Q] (every ordinate separately, the inputs of the
 * kinetic flux) [Sec. 4.3]:
 *   gradient  g_i = 1/A_i sum_k 1/2 (psi_i + psi_j(k)) n_ik            (Green-Gauss, face average)
 *   limiter   Psi_i = min_k { min(1, (max(psi_i, psi_j) - psi_i) / D)   if D > 0
 *                             min(1, (min(psi_i, psi_j) - psi_i) / D)   if D < 0
 *                             1                                          if D = 0 },  D = g_i . r_ik
 *   face value psif_ik = psi_i + Psi_i g_i . r_ik.
 * psi_j(k) across a boundary face is the ghost of orc_across. grad [C x Q x 2] and lim [C x Q]
 * may be NULL; psif is [C x 3 x Q]. */
void orc_reconstruct(int C, int Q, const int32_t *nbr, const double *nrm, const double *area,
                     const double *r, const double *psi, int bc, double *grad, double *lim,
                     double *psif)
{
    for (int i = 0; i < C; ++i)
        for (int q = 0; q < Q; ++q) {
            double pi = psi[(size_t)i * Q + q];
            double gx = 0.0, gy = 0.0;
            for (int k = 0; k < 3; ++k) {
                double avg = 0.5 * (pi + orc_across(nbr, Q, psi, bc, i, k, q));
                gx += avg * nrm[6 * i + 2 * k];
                gy += avg * nrm[6 * i + 2 * k + 1];
            }
            gx /= area[i];
            gy /= area[i];
            double L = 1.0;
            for (int k = 0; k < 3; ++k) {
                double pj = orc_across(nbr, Q, psi, bc, i, k, q);
                double D = gx * r[6 * i + 2 * k] + gy * r[6 * i + 2 * k + 1];
                double lk = 1.0;
                if (D > 0.0) {
                    double hi = pi > pj ? pi : pj;
                    lk = (hi - pi) / D;
                } else if (D < 0.0) {
                    double lo = pi < pj ? pi : pj;
                    lk = (lo - pi) / D;
                }
                if (lk > 1.0) lk = 1.0;
                if (lk < L) L = lk;
            }
            if (grad) {
                grad[((size_t)i * Q + q) * 2] = gx;
                grad[((size_t)i * Q + q) * 2 + 1] = gy;
            }
            if (lim) lim[(size_t)i * Q + q] = L;
            for (int k = 0; k < 3; ++k)
                psif[((size_t)i * 3 + k) * Q + q] =
                    pi + L * (gx * r[6 * i + 2 * k] + gy * r[6 * i + 2 * k + 1]);
        }
}

/* Explicit update with the second-order kinetic flux [Sec. 4.3, Sec. 4.4]: the upwind flux of
 * Eq. upwind1stOrder at every quadrature point with the reconstructed face values as its inputs,
 *   F_i = sum_k sum_q w_q m_q (Omega_q . n_ik) [psif_ik,q H(Omega_q . n_ik)
 *                                               + psif_j(k)k',q (1 - H(Omega_q . n_ik))],
 * k' the face of the neighbour j shared with cell i; across a boundary face the outside value is
 * psif_ik,q (Neumann) or 0 (vacuum). Then uout_i = uin_i - dt/A_i F_i + dt R_i(uin_i) with the
 * source of orc_flux_update. */
void orc_flux_update2(int C, int n, int Q, const double *M, const double *w, const double *ox,
                      const double *oy, const int32_t *nbr, const double *nrm, const double *area,
                      const double *psif, const double *sigma_a, const double *sigma_s,
                      const double *qsrc, double dt, int bc, const double *uin, double *uout)
{
    double mbar[64];
    for (int a = 0; a < n; ++a) {
        mbar[a] = 0.0;
        for (int q = 0; q < Q; ++q) mbar[a] += w[q] * M[(size_t)q * n + a];
    }
    for (int i = 0; i < C; ++i) {
        double F[64];
        for (int a = 0; a < n; ++a) F[a] = 0.0;
        for (int k = 0; k < 3; ++k) {
            int j = nbr[3 * i + k];
            int kk = -1;
            if (j >= 0)
                for (int t = 0; t < 3; ++t)
                    if (nbr[3 * j + t] == i) kk = t;
            double nx = nrm[6 * i + 2 * k], ny = nrm[6 * i + 2 * k + 1];
            for (int q = 0; q < Q; ++q) {
                double dot = ox[q] * nx + oy[q] * ny;
                double own = psif[((size_t)i * 3 + k) * Q + q];
                double up;
                if (dot > 0.0)
                    up = own;
                else if (j >= 0)
                    up = psif[((size_t)j * 3 + kk) * Q + q];
                else
                    up = (bc == 0) ? own : 0.0;
                double s = w[q] * dot * up;
                for (int a = 0; a < n; ++a) F[a] += s * M[(size_t)q * n + a];
            }
        }
        const double *ui = uin + (size_t)i * n;
        double u0 = ui[0];
        for (int a = 0; a < n; ++a) {
            double R = -sigma_a[i] * ui[a] - sigma_s[i] * (ui[a] - (a == 0 ? u0 : 0.0)) +
                       qsrc[i] * mbar[a];
            uout[(size_t)i * n + a] = ui[a] - dt / area[i] * F[a] + dt * R;
        }
    }
}

/* nsteps second-order M_N steps [Sec. 4.3, Heun]: with L(u) = -F(psif(alpha(u)))/A + R(u),
 *   u* = u^n + dt L(u^n),  u** = u* + dt L(u*),  u^{n+1} = (u^n + u**) / 2
 * (the paper's Delta t / A_i R in the Heun stages reads as Delta t R, as in the first-order
 * iteration). Each stage closes its moments (warm start: the previous closure), builds the
 * ansatz, reconstructs it and applies the second-order flux. Returns the number of failed
 * closures. */
int orc_mn_run2(int C, int n, int Q, const double *M, const double *w, const double *ox,
                const double *oy, const int32_t *nbr, const double *nrm, const double *area,
                const double *r, const double *sigma_a, const double *sigma_s, const double *qsrc,
                double dt, int bc, int nsteps, double tau, int max_iter, int polish, int nthreads,
                double *u, double *alpha, int32_t *status)
{
    size_t Cn = (size_t)C * n;
    double *psi = (double *)malloc(sizeof(double) * (size_t)C * Q);
    double *psif = (double *)malloc(sizeof(double) * (size_t)C * 3 * Q);
    double *u0 = (double *)malloc(sizeof(double) * Cn);
    double *us = (double *)malloc(sizeof(double) * Cn);
    double *uss = (double *)malloc(sizeof(double) * Cn);
    int nfail = 0;
    for (int s = 0; s < nsteps; ++s) {
        memcpy(u0, u, sizeof(double) * Cn);
        nfail += orc_closure_batch(C, n, Q, M, w, u0, alpha, tau, max_iter, 30, 1e-4, polish,
                                   nthreads, status, NULL);
        orc_ansatz(C, n, Q, M, alpha, psi, nthreads);
        orc_reconstruct(C, Q, nbr, nrm, area, r, psi, bc, NULL, NULL, psif);
        orc_flux_update2(C, n, Q, M, w, ox, oy, nbr, nrm, area, psif, sigma_a, sigma_s, qsrc, dt,
                         bc, u0, us);
        nfail += orc_closure_batch(C, n, Q, M, w, us, alpha, tau, max_iter, 30, 1e-4, polish,
                                   nthreads, status, NULL);
        orc_ansatz(C, n, Q, M, alpha, psi, nthreads);
        orc_reconstruct(C, Q, nbr, nrm, area, r, psi, bc, NULL, NULL, psif);
        orc_flux_update2(C, n, Q, M, w, ox, oy, nbr, nrm, area, psif, sigma_a, sigma_s, qsrc, dt,
                         bc, us, uss);
        for (size_t k = 0; k < Cn; ++k) u[k] = 0.5 * (u0[k] + uss[k]);
    }
    free(psi);
    free(psif);
    free(u0);
    free(us);
    free(uss);
    return nfail;
}

/* ------------------------------------------------------------------------------------------ */
/* S_N step [Sec. 2, Eq. SNEqns2; Sec. 4.2 explicit iteration; Sec. 4.4 upwind flux per         */
/* ordinate]                                                                                  */
/* ------------------------------------------------------------------------------------------ */

/* Degree l of each basis function, in the order of orc_basis. */
static void orc_basis_degrees(int N, int *deg)
{
    int idx = 0;
    for (int l = 0; l <= N; ++l)
        for (int k = -l; k <= l; ++k) {
            int ak = k < 0 ? -k : k;
            if (((l + ak) & 1) != 0) continue;
            deg[idx++] = l;
        }
}

/* One explicit S_N step of the nodal system (the ordinates psi_q of the full quadrature):
 *   psi'_iq = psi_iq - dt/A_i sum_f (Omega_q . n_if) [upwind psi]
 *             - dt (sigma_a,i + sigma_s,i) psi_iq + dt (O Sigma_i M psi_i)_q + dt q_i,
 * with the scattering in its P_N form O Sigma M of Eq. SNEqns2: M = (w_q m(Omega_q)) maps the
 * ordinates to the n moments of degree <= N, Sigma_i = sigma_s,i diag(g_l(a)) scales moment a by
 * the kernel's coefficient of its degree l(a) (g_0 = 1: sigma_s is the total scattering
 * cross-section; isotropic scattering is g = (1, 0, ..., 0)), and O = (m(Omega_q)) maps back.
 * The upwind value on face f is psi_iq when Omega_q . n_if > 0, else the neighbour's psi_jq,
 * or at the boundary the cell's own value (bc 0) or 0 (bc 1, vacuum). psi and psi_out are
 * [C x Q], distinct arrays. */
void orc_sn_step(int C, int n, int N, int Q, const double *M, const double *w, const double *ox,
                 const double *oy, const int32_t *nbr, const double *nrm, const double *area,
                 const double *sigma_a, const double *sigma_s, const double *qsrc,
                 const double *g, double dt, int bc, const double *psi, double *psi_out,
                 int nthreads)
{
    int deg[64];
    orc_basis_degrees(N, deg);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int i = 0; i < C; ++i) {
        const double *pi = psi + (size_t)i * Q;
        /* moments of the cell's ordinates, then the scattered moments */
        double s[64];
        for (int a = 0; a < n; ++a) {
            double v = 0.0;
            for (int q = 0; q < Q; ++q) v += w[q] * M[(size_t)q * n + a] * pi[q];
            s[a] = sigma_s[i] * g[deg[a]] * v;
        }
        for (int q = 0; q < Q; ++q) {
            double tr = 0.0;
            for (int k = 0; k < 3; ++k) {
                int j = nbr[3 * i + k];
                double dot = ox[q] * nrm[6 * i + 2 * k] + oy[q] * nrm[6 * i + 2 * k + 1];
                double up;
                if (dot > 0.0)
                    up = pi[q];
                else if (j >= 0)
                    up = psi[(size_t)j * Q + q];
                else
                    up = bc == 0 ? pi[q] : 0.0;
                tr += dot * up;
            }
            double sc = 0.0;
            for (int a = 0; a < n; ++a) sc += M[(size_t)q * n + a] * s[a];
            psi_out[(size_t)i * Q + q] = pi[q] - dt / area[i] * tr -
                                         dt * (sigma_a[i] + sigma_s[i]) * pi[q] + dt * sc +
                                         dt * qsrc[i];
        }
    }
    (void)nthreads;
}

/* nsteps S_N steps; psi [C x Q] is advanced in place (tmp is scratch of the same size). */
void orc_sn_run(int C, int n, int N, int Q, const double *M, const double *w, const double *ox,
                const double *oy, const int32_t *nbr, const double *nrm, const double *area,
                const double *sigma_a, const double *sigma_s, const double *qsrc, const double *g,
                double dt, int bc, int nsteps, double *psi, double *tmp, int nthreads)
{
    for (int s = 0; s < nsteps; ++s) {
        orc_sn_step(C, n, N, Q, M, w, ox, oy, nbr, nrm, area, sigma_a, sigma_s, qsrc, g, dt, bc,
                    psi, tmp, nthreads);
        memcpy(psi, tmp, sizeof(double) * (size_t)C * Q);
    }
}

/* nsteps explicit M_N steps. Each step: closure of every cell (warm start alpha), ansatz psi,
 * kinetic flux + update. alpha holds the closure of the last u that was closed. Returns the
 * number of failed closures summed over steps (0 on success); status gets the last failure
 * code per cell. */
int orc_mn_run_reg(int C, int n, int Q, const double *M, const double *w, const double *ox,
                   const double *oy, const int32_t *nbr, const double *nrm, const double *area,
                   const double *sigma_a, const double *sigma_s, const double *qsrc, double dt,
                   int bc, int nsteps, double tau, int max_iter, int polish, double gamma,
                   int reg0, int nthreads, double *u, double *alpha, int32_t *status)
{
    double *psi = (double *)malloc(sizeof(double) * (size_t)C * Q);
    int nfail = 0;
    for (int s = 0; s < nsteps; ++s) {
        nfail += orc_closure_batch_reg(C, n, Q, M, w, u, alpha, tau, max_iter, 30, 1e-4, polish,
                                       gamma, reg0, nthreads, status, NULL);
        orc_ansatz(C, n, Q, M, alpha, psi, nthreads);
        orc_flux_update(C, n, Q, M, w, ox, oy, nbr, nrm, area, psi, sigma_a, sigma_s, qsrc, dt,
                        bc, u, nthreads);
    }
    free(psi);
    return nfail;
}

/* nsteps first-order M_N steps with the entropy closure (no regularization). */
int orc_mn_run(int C, int n, int Q, const double *M, const double *w, const double *ox,
               const double *oy, const int32_t *nbr, const double *nrm, const double *area,
               const double *sigma_a, const double *sigma_s, const double *qsrc, double dt, int bc,
               int nsteps, double tau, int max_iter, int polish, int nthreads, double *u,
               double *alpha, int32_t *status)
{
    return orc_mn_run_reg(C, n, Q, M, w, ox, oy, nbr, nrm, area, sigma_a, sigma_s, qsrc, dt, bc,
                          nsteps, tau, max_iter, polish, 0.0, 1, nthreads, u, alpha, status);
}

/* ------------------------------------------------------------------------------------------ */
/* Discrete adjoint of the step                                                               */
/* ------------------------------------------------------------------------------------------ */

/* Transpose of the one-step map u^s -> u^{s+1} = u^s - dt/A F(psi(alpha(u^s))) + dt R(u^s),
 * linearised at (u, alpha) with alpha the converged closure of u and psi its ansatz:
 *   lamn = (du^{s+1}/du^s)^T lam.
 * The flux term gives mu_cq = d(sum_c lam_c . u_c^{s+1}) / d psi_cq (transposed upwind gather);
 * the closure term maps it back through d psi_iq / d u_i = psi_iq m_q^T H_i^-1 (implicit-function
 * theorem on g(alpha, u) = <m exp(alpha.m)> - u = 0); the source Jacobian -sigma_t I + sigma_s
 * e0 e0^T is symmetric. mu [C x Q] is scratch. Returns the number of Cholesky failures. */
static int orc_step_transpose(int C, int n, int Q, const double *M, const double *w,
                              const double *ox, const double *oy, const int32_t *nbr,
                              const double *nrm, const double *area, const double *sa,
                              const double *ss, double dt, int bc, const double *u,
                              const double *al, const double *psi, const double *lam, double *mu,
                              double *lamn)
{
    int nfail = 0;
    /* mu_cq = d(sum_c lambda_c . u_c^{s+1}) / d psi_cq through the flux term */
    for (size_t k = 0; k < (size_t)C * Q; ++k) mu[k] = 0.0;
    for (int c = 0; c < C; ++c) {
        const double *lc = lam + (size_t)c * n;
        for (int k = 0; k < 3; ++k) {
            int j = nbr[3 * c + k];
            double nx = nrm[6 * c + 2 * k], ny = nrm[6 * c + 2 * k + 1];
            for (int q = 0; q < Q; ++q) {
                double dot = ox[q] * nx + oy[q] * ny;
                double Lq = 0.0;
                for (int a = 0; a < n; ++a) Lq += lc[a] * M[(size_t)q * n + a];
                double coef = -dt / area[c] * w[q] * dot * Lq;
                if (dot > 0.0)
                    mu[(size_t)c * Q + q] += coef;
                else if (j >= 0)
                    mu[(size_t)j * Q + q] += coef;
                else if (bc == 0)
                    mu[(size_t)c * Q + q] += coef;
            }
        }
    }
    /* (du^{s+1}/du^s)^T lambda^{s+1} */
    for (int i = 0; i < C; ++i) {
        const double *li = lam + (size_t)i * n;
        double *ln = lamn + (size_t)i * n;
        /* identity + source Jacobian (-sigma_t I + sigma_s e0 e0^T, symmetric) */
        for (int a = 0; a < n; ++a)
            ln[a] = li[a] + dt * (-(sa[i] + ss[i]) * li[a] + (a == 0 ? ss[i] * li[0] : 0.0));
        /* closure: H_i^-1 sum_q mu_iq psi_iq m_q */
        double H[64 * 64], L[64 * 64], r[64], x[64];
        orc_dual_eval(n, Q, M, w, u + (size_t)i * n, al + (size_t)i * n, NULL, NULL, H, NULL);
        for (int a = 0; a < n; ++a) r[a] = 0.0;
        for (int q = 0; q < Q; ++q) {
            double t = mu[(size_t)i * Q + q] * psi[(size_t)i * Q + q];
            for (int a = 0; a < n; ++a) r[a] += t * M[(size_t)q * n + a];
        }
        if (orc_cholesky(n, H, L) != 0) {
            ++nfail;
            continue;
        }
        orc_chol_solve(n, L, r, x);
        for (int a = 0; a < n; ++a) ln[a] += x[a];
    }
    return nfail;
}

/* Objective: absorbed energy in the target cells,
 *   J = sum_{s=0}^{nsteps-1} dt sum_{i in T} A_i sigma_a,i <psi_i>,  <psi_i> = u_i0 / m_0.
 * Parameters: per-block sigma_a and sigma_s (block_of_cell). The reverse sweep applies the exact
 * transpose of u^{s+1} = u^s - dt/A F(psi(alpha(u^s))) + dt R(u^s), with
 * d psi_iq / d u_i = psi_iq m_q^T H_i^-1 (implicit-function theorem on g(alpha,u) = 0).
 * Stores every forward state (this is the plain version; no checkpointing).
 * Outputs J and dJ/dsigma_a[nb], dJ/dsigma_s[nb]. u0 is the initial state, alpha0 the warm start.
 * Returns the number of failed closures. */
int orc_mn_adjoint(int C, int n, int Q, const double *M, const double *w, const double *ox,
                   const double *oy, const int32_t *nbr, const double *nrm, const double *area,
                   const int32_t *block_of_cell, int nb, const double *sa_blk,
                   const double *ss_blk, const double *qsrc, const uint8_t *target, double dt,
                   int bc, int nsteps, double tau, int max_iter, int nthreads, const double *u0,
                   const double *alpha0, double *J, double *dJ_dsa, double *dJ_dss)
{
    size_t Cn = (size_t)C * n;
    double *us = (double *)malloc(sizeof(double) * Cn * (nsteps + 1));
    double *als = (double *)malloc(sizeof(double) * Cn * nsteps);
    double *sa = (double *)malloc(sizeof(double) * C);
    double *ss = (double *)malloc(sizeof(double) * C);
    double *psi = (double *)malloc(sizeof(double) * (size_t)C * Q);
    double *mu = (double *)malloc(sizeof(double) * (size_t)C * Q);
    double *lam = (double *)malloc(sizeof(double) * Cn);
    double *lamn = (double *)malloc(sizeof(double) * Cn);
    double *alpha = (double *)malloc(sizeof(double) * Cn);
    int32_t *st = (int32_t *)malloc(sizeof(int32_t) * C);
    double m0 = 1.0 / sqrt(4.0 * ORC_PI);
    for (int i = 0; i < C; ++i) {
        sa[i] = sa_blk[block_of_cell[i]];
        ss[i] = ss_blk[block_of_cell[i]];
    }
    memcpy(us, u0, sizeof(double) * Cn);
    memcpy(alpha, alpha0, sizeof(double) * Cn);
    int nfail = 0;
    double Jv = 0.0;
    for (int s = 0; s < nsteps; ++s) {
        double *u = us + Cn * s;
        for (int i = 0; i < C; ++i)
            if (target[i]) Jv += dt * area[i] * sa[i] * u[(size_t)i * n] / m0;
        nfail += orc_closure_batch(C, n, Q, M, w, u, alpha, tau, max_iter, 30, 1e-4, 1, nthreads,
                                   st, NULL);
        memcpy(als + Cn * s, alpha, sizeof(double) * Cn);
        orc_ansatz(C, n, Q, M, alpha, psi, nthreads);
        memcpy(us + Cn * (s + 1), u, sizeof(double) * Cn);
        orc_flux_update(C, n, Q, M, w, ox, oy, nbr, nrm, area, psi, sa, ss, qsrc, dt, bc,
                        us + Cn * (s + 1), nthreads);
    }
    *J = Jv;
    for (int b = 0; b < nb; ++b) dJ_dsa[b] = dJ_dss[b] = 0.0;
    for (size_t k = 0; k < Cn; ++k) lam[k] = 0.0; /* lambda^{nsteps} */
    for (int s = nsteps - 1; s >= 0; --s) {
        const double *u = us + Cn * s;
        const double *al = als + Cn * s;
        orc_ansatz(C, n, Q, M, al, psi, nthreads);
        /* parameter gradients from this step, with lambda^{s+1} */
        for (int i = 0; i < C; ++i) {
            const double *ui = u + (size_t)i * n, *li = lam + (size_t)i * n;
            double lu = 0.0, lus = 0.0;
            for (int a = 0; a < n; ++a) {
                lu += li[a] * ui[a];
                lus += li[a] * (ui[a] - (a == 0 ? ui[0] : 0.0));
            }
            dJ_dsa[block_of_cell[i]] += -dt * lu;
            dJ_dss[block_of_cell[i]] += -dt * lus;
            if (target[i]) dJ_dsa[block_of_cell[i]] += dt * area[i] * ui[0] / m0;
        }
        nfail += orc_step_transpose(C, n, Q, M, w, ox, oy, nbr, nrm, area, sa, ss, dt, bc, u, al,
                                    psi, lam, mu, lamn);
        for (int i = 0; i < C; ++i)
            if (target[i]) lamn[(size_t)i * n] += dt * area[i] * sa[i] / m0;
        memcpy(lam, lamn, sizeof(double) * Cn);
    }
    free(us);
    free(als);
    free(sa);
    free(ss);
    free(psi);
    free(mu);
    free(lam);
    free(lamn);
    free(alpha);
    free(st);
    return nfail;
}

/* One-step transpose (vector-Jacobian product) at (u, alpha), alpha the converged closure of u:
 * out = (du^{s+1}/du^s)^T lam, the reverse step of orc_mn_adjoint without the objective's terms.
 * Returns the number of Cholesky failures. */
int orc_step_vjp(int C, int n, int Q, const double *M, const double *w, const double *ox,
                 const double *oy, const int32_t *nbr, const double *nrm, const double *area,
                 const double *sa, const double *ss, double dt, int bc, const double *u,
                 const double *alpha, const double *lam, double *out)
{
    double *psi = (double *)malloc(sizeof(double) * (size_t)C * Q);
    double *mu = (double *)malloc(sizeof(double) * (size_t)C * Q);
    orc_ansatz(C, n, Q, M, alpha, psi, 0);
    int nf = orc_step_transpose(C, n, Q, M, w, ox, oy, nbr, nrm, area, sa, ss, dt, bc, u, alpha, psi,
                                lam, mu, out);
    free(psi);
    free(mu);
    return nf;
}

/* One-step tangent (Jacobian-vector product) at (u, alpha), written in forward mode and
 * independently of the transpose above: the closure's tangent d alpha_i = H_i^-1 du_i (from
 * g(alpha, u) = 0), the ansatz's d psi_iq = psi_iq m_q . d alpha_i, then the step itself, which is
 * linear in (psi, u) once the source q is zero:
 *   out = du - dt/A F(d psi) + dt (-sigma_a du - sigma_s (du - du_0 e_0)).
 * Returns the number of Cholesky failures. */
int orc_step_jvp(int C, int n, int Q, const double *M, const double *w, const double *ox,
                 const double *oy, const int32_t *nbr, const double *nrm, const double *area,
                 const double *sa, const double *ss, double dt, int bc, const double *u,
                 const double *alpha, const double *du, double *out)
{
    double *dpsi = (double *)malloc(sizeof(double) * (size_t)C * Q);
    double *zero = (double *)calloc((size_t)C, sizeof(double));
    int nf = 0;
    for (int i = 0; i < C; ++i) {
        double H[64 * 64], L[64 * 64], da[64];
        orc_dual_eval(n, Q, M, w, u + (size_t)i * n, alpha + (size_t)i * n, NULL, NULL, H, NULL);
        if (orc_cholesky(n, H, L) != 0) {
            ++nf;
            for (int a = 0; a < n; ++a) da[a] = 0.0;
        } else {
            orc_chol_solve(n, L, du + (size_t)i * n, da);
        }
        for (int q = 0; q < Q; ++q) {
            double z = 0.0, dz = 0.0;
            for (int a = 0; a < n; ++a) {
                z += alpha[(size_t)i * n + a] * M[(size_t)q * n + a];
                dz += da[a] * M[(size_t)q * n + a];
            }
            dpsi[(size_t)i * Q + q] = exp(z) * dz;
        }
    }
    memcpy(out, du, sizeof(double) * (size_t)C * n);
    orc_flux_update(C, n, Q, M, w, ox, oy, nbr, nrm, area, dpsi, sa, ss, zero, dt, bc, out, 0);
    free(dpsi);
    free(zero);
    return nf;
}

/* Forward value only of the same objective (for finite differences). */
int orc_mn_objective(int C, int n, int Q, const double *M, const double *w, const double *ox,
                     const double *oy, const int32_t *nbr, const double *nrm, const double *area,
                     const int32_t *block_of_cell, const double *sa_blk, const double *ss_blk,
                     const double *qsrc, const uint8_t *target, double dt, int bc, int nsteps,
                     double tau, int max_iter, int nthreads, const double *u0,
                     const double *alpha0, double *J)
{
    size_t Cn = (size_t)C * n;
    double *u = (double *)malloc(sizeof(double) * Cn);
    double *alpha = (double *)malloc(sizeof(double) * Cn);
    double *sa = (double *)malloc(sizeof(double) * C);
    double *ss = (double *)malloc(sizeof(double) * C);
    double *psi = (double *)malloc(sizeof(double) * (size_t)C * Q);
    int32_t *st = (int32_t *)malloc(sizeof(int32_t) * C);
    double m0 = 1.0 / sqrt(4.0 * ORC_PI);
    for (int i = 0; i < C; ++i) {
        sa[i] = sa_blk[block_of_cell[i]];
        ss[i] = ss_blk[block_of_cell[i]];
    }
    memcpy(u, u0, sizeof(double) * Cn);
    memcpy(alpha, alpha0, sizeof(double) * Cn);
    int nfail = 0;
    double Jv = 0.0;
    for (int s = 0; s < nsteps; ++s) {
        for (int i = 0; i < C; ++i)
            if (target[i]) Jv += dt * area[i] * sa[i] * u[(size_t)i * n] / m0;
        nfail += orc_closure_batch(C, n, Q, M, w, u, alpha, tau, max_iter, 30, 1e-4, 1, nthreads,
                                   st, NULL);
        orc_ansatz(C, n, Q, M, alpha, psi, nthreads);
        orc_flux_update(C, n, Q, M, w, ox, oy, nbr, nrm, area, psi, sa, ss, qsrc, dt, bc, u,
                        nthreads);
    }
    *J = Jv;
    free(u);
    free(alpha);
    free(sa);
    free(ss);
    free(psi);
    free(st);
    return nfail;
}

/* ------------------------------------------------------------------------------------------ */
/* MLP (learned closure): y = W4 s(W3 s(W2 s(W1 x + b1) + b2) + b3) + b4, s = softplus.       */
/* Weights row-major [in x out]; loss = 1/(2B) sum_b ||y_b - t_b||^2.                        */
/* ------------------------------------------------------------------------------------------ */

static double orc_softplus(double x) { return x > 0 ? x + log1p(exp(-x)) : log1p(exp(x)); }
static double orc_sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

static void orc_dense(int B, int din, int dout, const double *X, const double *W, const double *b,
                      double *Y)
{
    for (int r = 0; r < B; ++r)
        for (int o = 0; o < dout; ++o) {
            double s = b[o];
            for (int i = 0; i < din; ++i) s += X[(size_t)r * din + i] * W[(size_t)i * dout + o];
            Y[(size_t)r * dout + o] = s;
        }
}

/* params: W1[din*H] b1[H] W2[H*H] b2[H] W3[H*H] b3[H] W4[H*dout] b4[dout], packed in that order. */
void orc_mlp_forward(int B, int din, int H, int dout, const double *params, const double *X,
                     double *Y)
{
    const double *W1 = params, *b1 = W1 + din * H, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H,
                 *b3 = W3 + H * H, *W4 = b3 + H, *b4 = W4 + H * dout;
    double *a = (double *)malloc(sizeof(double) * (size_t)B * H);
    double *c = (double *)malloc(sizeof(double) * (size_t)B * H);
    orc_dense(B, din, H, X, W1, b1, a);
    for (size_t k = 0; k < (size_t)B * H; ++k) a[k] = orc_softplus(a[k]);
    orc_dense(B, H, H, a, W2, b2, c);
    for (size_t k = 0; k < (size_t)B * H; ++k) c[k] = orc_softplus(c[k]);
    orc_dense(B, H, H, c, W3, b3, a);
    for (size_t k = 0; k < (size_t)B * H; ++k) a[k] = orc_softplus(a[k]);
    orc_dense(B, H, dout, a, W4, b4, Y);
    free(a);
    free(c);
}

/* Loss and gradient w.r.t. the packed parameters (same packing). Returns the loss. */
double orc_mlp_loss_grad(int B, int din, int H, int dout, const double *params, const double *X,
                         const double *T, double *grad)
{
    const double *W1 = params, *b1 = W1 + din * H, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H,
                 *b3 = W3 + H * H, *W4 = b3 + H, *b4 = W4 + H * dout;
    double *gW1 = grad, *gb1 = gW1 + din * H, *gW2 = gb1 + H, *gb2 = gW2 + H * H,
           *gW3 = gb2 + H, *gb3 = gW3 + H * H, *gW4 = gb3 + H, *gb4 = gW4 + H * dout;
    size_t BH = (size_t)B * H;
    double *z1 = malloc(sizeof(double) * BH), *h1 = malloc(sizeof(double) * BH);
    double *z2 = malloc(sizeof(double) * BH), *h2 = malloc(sizeof(double) * BH);
    double *z3 = malloc(sizeof(double) * BH), *h3 = malloc(sizeof(double) * BH);
    double *y = malloc(sizeof(double) * (size_t)B * dout);
    double *dy = malloc(sizeof(double) * (size_t)B * dout);
    double *dh = malloc(sizeof(double) * BH), *dz = malloc(sizeof(double) * BH);
    orc_dense(B, din, H, X, W1, b1, z1);
    for (size_t k = 0; k < BH; ++k) h1[k] = orc_softplus(z1[k]);
    orc_dense(B, H, H, h1, W2, b2, z2);
    for (size_t k = 0; k < BH; ++k) h2[k] = orc_softplus(z2[k]);
    orc_dense(B, H, H, h2, W3, b3, z3);
    for (size_t k = 0; k < BH; ++k) h3[k] = orc_softplus(z3[k]);
    orc_dense(B, H, dout, h3, W4, b4, y);
    double loss = 0.0;
    for (size_t k = 0; k < (size_t)B * dout; ++k) {
        double r = y[k] - T[k];
        loss += 0.5 * r * r / B;
        dy[k] = r / B;
    }
    /* layer 4 */
    for (int i = 0; i < H; ++i)
        for (int o = 0; o < dout; ++o) {
            double s = 0.0;
            for (int r = 0; r < B; ++r) s += h3[(size_t)r * H + i] * dy[(size_t)r * dout + o];
            gW4[i * dout + o] = s;
        }
    for (int o = 0; o < dout; ++o) {
        double s = 0.0;
        for (int r = 0; r < B; ++r) s += dy[(size_t)r * dout + o];
        gb4[o] = s;
    }
    for (int r = 0; r < B; ++r)
        for (int i = 0; i < H; ++i) {
            double s = 0.0;
            for (int o = 0; o < dout; ++o) s += dy[(size_t)r * dout + o] * W4[i * dout + o];
            dh[(size_t)r * H + i] = s;
        }
    /* layers 3, 2, 1 */
    const double *Ws[3] = {W3, W2, W1};
    double *gWs[3] = {gW3, gW2, gW1}, *gbs[3] = {gb3, gb2, gb1};
    double *zs[3] = {z3, z2, z1};
    const double *ins[3] = {h2, h1, X};
    int dins[3] = {H, H, din};
    for (int l = 0; l < 3; ++l) {
        for (size_t k = 0; k < BH; ++k) dz[k] = dh[k] * orc_sigmoid(zs[l][k]);
        int di = dins[l];
        for (int i = 0; i < di; ++i)
            for (int o = 0; o < H; ++o) {
                double s = 0.0;
                for (int r = 0; r < B; ++r) s += ins[l][(size_t)r * di + i] * dz[(size_t)r * H + o];
                gWs[l][i * H + o] = s;
            }
        for (int o = 0; o < H; ++o) {
            double s = 0.0;
            for (int r = 0; r < B; ++r) s += dz[(size_t)r * H + o];
            gbs[l][o] = s;
        }
        if (l < 2) {
            for (int r = 0; r < B; ++r)
                for (int i = 0; i < H; ++i) {
                    double s = 0.0;
                    for (int o = 0; o < H; ++o) s += dz[(size_t)r * H + o] * Ws[l][i * H + o];
                    dh[(size_t)r * H + i] = s;
                }
        }
    }
    free(z1); free(h1); free(z2); free(h2); free(z3); free(h3);
    free(y); free(dy); free(dh); free(dz);
    return loss;
}

/* One Adam step (Kingma & Ba 2015) at step count t >= 1 over P parameters. */
void orc_adam(int P, double *p, const double *g, double *m, double *v, int t, double lr,
              double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int k = 0; k < P; ++k) {
        m[k] = b1 * m[k] + (1.0 - b1) * g[k];
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
        p[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
    }
}
