// Body of the thread-per-cell Newton step, included twice by newton_common.cuh: once with every
// loop fully unrolled (N <= 3: the packed Cholesky factor lives in registers) and once with the
// loops rolled (N >= 4: the 120 or 231 factor entries live in local memory; full unrolling
// would spill anyway and takes the compiler minutes). The includer defines KITRT_PT_NAME and
// KITRT_PT_UNROLL. No include guard on purpose.
// One-thread version of newton_post for the scalar Newton logic after an evaluation: V points to
// the cell's n2 degree-2N moments (the post kernel's shared-memory copy), entry c at V[c vs];
// for a tensor-core cell of the mixed modes the moments c >= n are instead FP32 numbers in Vf
// (same stride), and the body adds the FP32 copies of the first n there.
// Every instruction of this logic keeps all 32 lanes busy (32 cells per warp).
//
// Precision: the dual, its gradient, the Armijo and convergence tests and the iterate are FP64.
// The Hessian, its Cholesky factor and the Newton direction are FP64 in the FP64 mode and for
// cells handed to the FP64 Hessian (S.h64); in the mixed modes they are otherwise FP32: those
// Hessian moments come from TF32/BF16 tensor-core products, so FP64 arithmetic on them buys no
// accuracy, and on this GPU an FP64 instruction costs as much issue time as 64 FP32 ones. The
// direction only steers Newton; the accepted alpha is judged by the FP64 gradient. A factor that
// is not positive definite in FP32 sends the cell to the FP64 Hessian, as a TF32 one does.
// Returns true when the cell continues (must be appended to the next list).
template <int NN>
__device__ bool KITRT_PT_NAME(const Tables &T, const NewtonState &S, const NewtonParams &np,
                                   int cell, const double *__restrict__ V, float *__restrict__ Vf,
                                   int vs, const double *__restrict__ u, bool mixed, int &evals_out)
{
    constexpr int n = Dims<NN>::n, n2 = Dims<NN>::n2, npairs = Dims<NN>::npairs;
    const size_t off = (size_t)cell * n;
    const int ph = S.phase[cell];
    const double lam = ph == PH_NEWTON ? S.lam[cell] : 0.0;
    const bool reg = np.gamma != 0.0;  // uniform: regularized closure
    double at[n], ua[n];
    double au = 0.0, ar2 = 0.0;
KITRT_PT_UNROLL
    for (int a = 0; a < n; ++a) {
        const double al = S.alpha[off + a];
        at[a] = ph == PH_NEWTON ? fma(lam, S.dir[off + a], al) : al;
        ua[a] = u[off + a];
        au = fma(at[a], ua[a], au);
    }
    if (reg) {
KITRT_PT_UNROLL
        for (int a = 0; a < n; ++a)
            if (a >= np.reg0) ar2 = fma(at[a], at[a], ar2);
    }
    // in the mixed modes a tensor-core cell's Hessian-only moments (c >= n) are in Vf (FP32)
    const bool h32 = mixed && !S.h64[cell];
    bool finite = true;
KITRT_PT_UNROLL
    for (int c = 0; c < n2; ++c)
        finite = finite && (c < n || !h32 ? finite_bits(V[(size_t)c * vs])
                                          : (__float_as_uint(Vf[(size_t)c * vs]) & 0x7f800000u) != 0x7f800000u);
    const double fs = V[0] * T.rm0;
    // the dual at the trial point (plus the regularization gamma/2 |alpha^r|^2)
    const double ft = reg ? fma(0.5 * np.gamma, ar2, fs - au) : fs - au;
    const int ev = S.evals[cell] + 1;
    S.evals[cell] = ev;
    evals_out = ev;
    auto fail_t = [&](int code) {
        S.status[cell] = code;
        S.phase[cell] = PH_DONE;
        atomicAdd(&S.cnt[3], 1);
    };
    bool accept;
    if (ph == PH_INIT) {
        if (!finite) {
            fail_t(KITRT_ENOTREALIZABLE);
            return false;
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
            if (mixed && !S.h64[cell]) {
                // the line search could not follow the direction from the tensor-core Hessian:
                // restart from the accepted point with the FP64 Hessian
                hand_over(S, cell);
                S.halv[cell] = 0;
                S.phase[cell] = PH_INIT;
                return true;
            }
            fail_t(KITRT_ELINESEARCH);
            return false;
        }
        S.halv[cell] = h;
        S.lam[cell] = 0.5 * lam;
        return true;
    }
    // gradient g = <m e> - u (+ gamma alpha^r), FP64
    double g[n];
KITRT_PT_UNROLL
    for (int a = 0; a < n; ++a) {
        g[a] = V[(size_t)a * vs] - ua[a];
        if (reg && a >= np.reg0) g[a] = fma(np.gamma, at[a], g[a]);
    }
    double y[n];  // the Newton direction -H^-1 g
    if (h32) {
        // Hessian (packed lower) from the Gaunt coefficients, Cholesky with 1/L_jj on the
        // diagonal, and the two triangular solves, in FP32
KITRT_PT_UNROLL
        for (int c = 0; c < n; ++c) Vf[(size_t)c * vs] = d2f_bits(V[(size_t)c * vs]);
        float Lf[npairs];
KITRT_PT_UNROLL
        for (int p = 0; p < npairs; ++p) {
            float h = 0.0f;
            for (int t = T.gstart[p]; t < T.gstart[p + 1]; ++t)
                h = fmaf(T.gcoef32[t], Vf[(size_t)T.gidx[t] * vs], h);
            Lf[p] = h;
        }
        if (reg) {
            const float gam = d2f_bits(np.gamma);
KITRT_PT_UNROLL
            for (int j = 0; j < n; ++j)
                if (j >= np.reg0) Lf[tri_idx(j, j)] += gam;
        }
        bool spd = true;
KITRT_PT_UNROLL
        for (int j = 0; j < n; ++j) {
            float d = Lf[tri_idx(j, j)];
KITRT_PT_UNROLL
            for (int k = 0; k < j; ++k) d = fmaf(-Lf[tri_idx(j, k)], Lf[tri_idx(j, k)], d);
            spd = spd && d > 0.0f && d < 3.0e38f;
            const float rinv = rsqrtf(d > 0.0f ? d : 1.0f);
            Lf[tri_idx(j, j)] = rinv;
KITRT_PT_UNROLL
            for (int i = j + 1; i < n; ++i) {
                float s = Lf[tri_idx(i, j)];
KITRT_PT_UNROLL
                for (int k = 0; k < j; ++k) s = fmaf(-Lf[tri_idx(i, k)], Lf[tri_idx(j, k)], s);
                Lf[tri_idx(i, j)] = s * rinv;
            }
        }
        if (!spd) {
            hand_over(S, cell);  // rounding broke positive definiteness: redo this point in FP64
            return true;
        }
        float yf[n];
KITRT_PT_UNROLL
        for (int i = 0; i < n; ++i) {
            float s = -d2f_bits(g[i]);
KITRT_PT_UNROLL
            for (int k = 0; k < i; ++k) s = fmaf(-Lf[tri_idx(i, k)], yf[k], s);
            yf[i] = s * Lf[tri_idx(i, i)];
        }
KITRT_PT_UNROLL
        for (int i = n - 1; i >= 0; --i) {
            float s = yf[i];
KITRT_PT_UNROLL
            for (int k = i + 1; k < n; ++k) s = fmaf(-Lf[tri_idx(k, i)], yf[k], s);
            yf[i] = s * Lf[tri_idx(i, i)];
        }
KITRT_PT_UNROLL
        for (int a = 0; a < n; ++a) y[a] = f2d_bits(yf[a]);
KITRT_PT_UNROLL
        for (int p = 0; p < npairs; ++p) S.L[(size_t)cell * npairs + p] = f2d_bits(Lf[p]);
    } else {
        double Lp[npairs];
KITRT_PT_UNROLL
        for (int p = 0; p < npairs; ++p) {
            double h = 0.0;
            for (int t = T.gstart[p]; t < T.gstart[p + 1]; ++t) h = fma(T.gcoef[t], V[(size_t)T.gidx[t] * vs], h);
            Lp[p] = h;
        }
        // regularized moments: the Hessian gains gamma on their diagonal
        if (reg) {
KITRT_PT_UNROLL
            for (int j = 0; j < n; ++j)
                if (j >= np.reg0) Lp[tri_idx(j, j)] += np.gamma;
        }
        bool spd = true;
KITRT_PT_UNROLL
        for (int j = 0; j < n; ++j) {
            double d = Lp[tri_idx(j, j)];
KITRT_PT_UNROLL
            for (int k = 0; k < j; ++k) d = fma(-Lp[tri_idx(j, k)], Lp[tri_idx(j, k)], d);
            spd = spd && d > 0.0;
            const double rinv = rsqrt(d > 0.0 ? d : 1.0);
            Lp[tri_idx(j, j)] = rinv;
KITRT_PT_UNROLL
            for (int i = j + 1; i < n; ++i) {
                double s = Lp[tri_idx(i, j)];
KITRT_PT_UNROLL
                for (int k = 0; k < j; ++k) s = fma(-Lp[tri_idx(i, k)], Lp[tri_idx(j, k)], s);
                Lp[tri_idx(i, j)] = s * rinv;
            }
        }
        if (!spd) {
            // FP64 mode, or the FP64 Hessian of a handed-over cell: no further fallback
            fail_t(KITRT_ECHOL);
            return false;
        }
KITRT_PT_UNROLL
        for (int i = 0; i < n; ++i) {
            double s = -g[i];
KITRT_PT_UNROLL
            for (int k = 0; k < i; ++k) s = fma(-Lp[tri_idx(i, k)], y[k], s);
            y[i] = s * Lp[tri_idx(i, i)];
        }
KITRT_PT_UNROLL
        for (int i = n - 1; i >= 0; --i) {
            double s = y[i];
KITRT_PT_UNROLL
            for (int k = i + 1; k < n; ++k) s = fma(-Lp[tri_idx(k, i)], y[k], s);
            y[i] = s * Lp[tri_idx(i, i)];
        }
KITRT_PT_UNROLL
        for (int p = 0; p < npairs; ++p) S.L[(size_t)cell * npairs + p] = Lp[p];
    }
    // accepted: store the point, its moments and (above) the factor of H
KITRT_PT_UNROLL
    for (int a = 0; a < n; ++a) {
        S.alpha[off + a] = at[a];
        S.U[off + a] = V[(size_t)a * vs];
    }
    S.fsum[cell] = fs;
    S.f0[cell] = ft;
    if (S.lfac) S.lfac[cell] = 1;
    double gn2 = 0.0, un2 = 0.0, gd = 0.0;
KITRT_PT_UNROLL
    for (int a = 0; a < n; ++a) {
        gn2 = fma(g[a], g[a], gn2);
        un2 = fma(ua[a], ua[a], un2);
        gd = fma(g[a], y[a], gd);
        S.dir[off + a] = y[a];
    }
    int iters = S.iters[cell];
    if (ph == PH_NEWTON) ++iters;
    S.iters[cell] = iters;
    const double gn = sqrt(gn2);
    if (gn <= np.tau * sqrt(un2)) {
        S.phase[cell] = PH_DONE;
        return false;
    }
    if (iters >= np.max_iter) {
        fail_t(KITRT_ENOCONVERGE);
        return false;
    }
    if (mixed && ph == PH_NEWTON && gn > kStallRatio * S.gnorm[cell]) hand_over(S, cell);
    if (S.gnorm) S.gnorm[cell] = gn;
    S.gd[cell] = gd;
    S.lam[cell] = 1.0;
    S.halv[cell] = 0;
    S.phase[cell] = PH_NEWTON;
    return true;
}
