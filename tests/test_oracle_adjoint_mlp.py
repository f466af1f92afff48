"""Pins for the oracle's discrete adjoint (checked against central finite differences of its own
forward objective, which is a different code path, and against the mirror image of the same
problem) and for its MLP backward pass and Adam step (finite differences; Adam's first step has
the closed form -lr * sign(g))."""
import numpy as np
import pytest

import oracle as O
from paper_2205_08417_gb300 import synth


def _blocks_problem(k=13, nb=7, seed=3, N=2, order=4):
    T = O.Tables(N, order)
    m = synth.jittered_mesh(k, 0.0, 7.0, seed=seed)
    G = O.Geometry(m.xy, m.tri)
    blk, sa, ss = synth.block_coefficients(G.cen, 0.0, 7.0, nb, seed)
    q = np.where(blk == (nb // 2) * nb + nb // 2, 1.0, 0.0)
    tgt = np.zeros(G.C, dtype=np.uint8)
    bx, by = blk // nb, blk % nb
    tgt[(bx >= 2) & (bx <= 4) & (by >= 2) & (by <= 4)] = 1
    u0 = np.zeros((G.C, T.n))
    u0[:, 0] = 1e-4 / np.sqrt(4 * np.pi)
    a0 = O.isotropic_alpha(T, u0)
    return T, G, blk, sa, ss, q, tgt, u0, a0


def test_adjoint_matches_central_differences():
    T, G, blk, sa, ss, q, tgt, u0, a0 = _blocks_problem()
    dt = G.cfl_dt(0.4)
    assert dt * (sa.max() + ss.max()) <= 0.6
    nsteps = 12
    J, gsa, gss = O.mn_adjoint(T, G, blk, sa, ss, q, tgt, dt, nsteps, u0, a0, bc=1, tau=1e-13)
    J2 = O.mn_objective(T, G, blk, sa, ss, q, tgt, dt, nsteps, u0, a0, bc=1, tau=1e-13)
    assert abs(J - J2) <= 1e-14 * abs(J)
    h = 1e-6
    rng = np.random.default_rng(0)
    for which, grad, base in [("sa", gsa, sa), ("ss", gss, ss)]:
        for b in list(rng.choice(len(base), 5, replace=False)) + [24, 16]:
            p, m = base.copy(), base.copy()
            p[b] += h
            m[b] -= h
            args_p = (p, ss) if which == "sa" else (sa, p)
            args_m = (m, ss) if which == "sa" else (sa, m)
            Jp = O.mn_objective(T, G, blk, *args_p, q, tgt, dt, nsteps, u0, a0, bc=1, tau=1e-13)
            Jm = O.mn_objective(T, G, blk, *args_m, q, tgt, dt, nsteps, u0, a0, bc=1, tau=1e-13)
            fd = (Jp - Jm) / (2 * h)
            assert abs(fd - grad[b]) <= 1e-6 * max(np.abs(gsa).max(), np.abs(gss).max()), \
                (which, b, fd, grad[b])


def test_adjoint_neumann_variant():
    T, G, blk, sa, ss, q, tgt, u0, a0 = _blocks_problem(k=9, N=1, order=3)
    dt = G.cfl_dt(0.4)
    J, gsa, gss = O.mn_adjoint(T, G, blk, sa, ss, q, tgt, dt, 6, u0, a0, bc=0, tau=1e-13)
    h = 1e-6
    b = 24
    p, m = sa.copy(), sa.copy()
    p[b] += h
    m[b] -= h
    fd = (O.mn_objective(T, G, blk, p, ss, q, tgt, dt, 6, u0, a0, bc=0, tau=1e-13) -
          O.mn_objective(T, G, blk, m, ss, q, tgt, dt, 6, u0, a0, bc=0, tau=1e-13)) / (2 * h)
    assert abs(fd - gsa[b]) <= 1e-6 * np.abs(gsa).max()


def _mlp_setup(seed=0, din=5, H=8, dout=5, B=7):
    rng = np.random.default_rng(seed)
    P = O.mlp_param_count(din, H, dout)
    p = rng.normal(scale=0.4, size=P)
    X = rng.normal(size=(B, din))
    Tt = rng.normal(size=(B, dout))
    return p, X, Tt, din, H, dout


def test_mlp_gradient_matches_finite_differences():
    p, X, Tt, din, H, dout = _mlp_setup()
    loss, g = O.mlp_loss_grad(p, X, Tt, din, H, dout)
    h = 1e-6
    for k in range(p.shape[0]):
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (O.mlp_loss_grad(pp, X, Tt, din, H, dout)[0] - O.mlp_loss_grad(pm, X, Tt, din, H, dout)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k]))
    # loss is consistent with the forward pass
    Y = O.mlp_forward(p, X, din, H, dout)
    assert abs(loss - 0.5 * ((Y - Tt) ** 2).sum() / X.shape[0]) < 1e-14


def test_mlp_softplus_layer_by_hand():
    # din = H = dout = 1 with zero biases: y = w4 s(w3 s(w2 s(w1 x))), s(z) = log(1 + e^z)
    sp = lambda z: np.log1p(np.exp(z))
    w1, w2, w3, w4 = 0.7, -1.3, 0.4, 2.0
    p = np.array([w1, 0.0, w2, 0.0, w3, 0.0, w4, 0.0])
    x = 0.9
    y = w4 * sp(w3 * sp(w2 * sp(w1 * x)))
    assert abs(O.mlp_forward(p, np.array([[x]]), 1, 1, 1)[0, 0] - y) < 1e-15


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    p = rng.normal(size=10)
    g = rng.normal(size=10)
    p0 = p.copy()
    m = np.zeros(10)
    v = np.zeros(10)
    O.adam(p, g, m, v, 1, lr=1e-2, eps=0.0)
    np.testing.assert_allclose(p, p0 - 1e-2 * np.sign(g), rtol=0, atol=1e-15)


@pytest.mark.parametrize("bc", [0, 1])
def test_one_step_transpose_dot_product(bc):
    """<J du, lam> = <du, J^T lam> for the one-step map u^s -> u^{s+1} at a converged closure, with
    J du from the oracle's forward-mode tangent and J^T lam from the reverse step its adjoint
    uses (two separately written code paths), to 1e-12 of |J du| |lam|; the tangent itself
    agrees with central differences of the forward step."""
    N, order = 2, 6
    T = O.Tables(N, order)
    m = synth.jittered_mesh(9, 0.0, 1.0, seed=5)
    G = O.Geometry(m.xy, m.tri)
    C = G.C
    rng = np.random.default_rng(8)
    mu, phi, w, ox, oy = O.quadrature(order)
    c, k, wt = synth.vmf_mixtures(C, 12, kappa_hi=5.0)
    u = synth.vmf_density(np.stack([ox, oy, mu], axis=1), c, k, wt) @ (T.w[:, None] * T.M)
    alpha = O.isotropic_alpha(T, u)
    st, _ = O.closure(T, u, alpha, tau=1e-13)
    assert (st == 0).all()
    sa, ss = rng.uniform(0, 1, C), rng.uniform(0, 1, C)
    dt = G.cfl_dt(0.4)
    du = rng.normal(size=u.shape) * np.abs(u).max() * 1e-2
    lam = rng.normal(size=u.shape)
    Jdu = O.step_jvp(T, G, u, alpha, sa, ss, dt, du, bc=bc)
    JTl = O.step_vjp(T, G, u, alpha, sa, ss, dt, lam, bc=bc)
    lhs, rhs = float(np.sum(Jdu * lam)), float(np.sum(du * JTl))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Jdu) * np.linalg.norm(lam), (lhs, rhs)
    # the tangent is the derivative of the forward step
    h = 1e-4

    def step(uu):
        uu = uu.copy()
        aa = alpha.copy()
        nf, _ = O.mn_run(T, G, uu, aa, sa, ss, np.zeros(C), dt, 1, bc=bc, tau=1e-13)
        assert nf == 0
        return uu

    fd = (step(u + h * du) - step(u - h * du)) / (2 * h)
    assert np.linalg.norm(fd - Jdu) <= 1e-6 * np.linalg.norm(Jdu)


def test_adam_second_step_closed_forms():
    """Adam at t = 2 (Kingma & Ba): with the same gradient twice the bias-corrected moments are
    exactly g and g^2, so each step is -lr sign(g); with the gradient reversed, m^_2 =
    -(1 - b1)/(1 + b1) g and v^_2 = g^2, so the second step is +lr (1 - b1)/(1 + b1) sign(g).
    A bias correction with the wrong power of beta at t >= 2 fails both."""
    rng = np.random.default_rng(4)
    lr, b1, b2 = 1e-2, 0.9, 0.999
    g = rng.normal(size=12)
    p0 = rng.normal(size=12)
    for g2, expect in [(g, p0 - 2 * lr * np.sign(g)),
                       (-g, p0 - lr * np.sign(g) + lr * (1 - b1) / (1 + b1) * np.sign(g))]:
        p, m, v = p0.copy(), np.zeros(12), np.zeros(12)
        O.adam(p, g, m, v, 1, lr=lr, b1=b1, b2=b2, eps=0.0)
        O.adam(p, g2, m, v, 2, lr=lr, b1=b1, b2=b2, eps=0.0)
        np.testing.assert_allclose(p, expect, rtol=0, atol=1e-15)


@pytest.mark.parametrize("axis", [0, 1])
def test_adjoint_is_unchanged_by_mirroring_the_mesh(axis):
    """The same block problem on the mesh mirrored in x or y (every triangle clockwise, each cell
    keeping its block, source and target flag) is the mirror image of the original: the
    isotropic start is its own mirror, so the objective and every block gradient of the adjoint
    (transposed flux, closure backward) must be unchanged."""
    from mirror_map import mirror_xy
    T, G, blk, sa, ss, q, tgt, u0, a0 = _blocks_problem()
    m = synth.jittered_mesh(13, 0.0, 7.0, seed=3)
    Gr = O.Geometry(mirror_xy(m.xy, axis), m.tri)
    dt = G.cfl_dt(0.4)
    J, gsa, gss = O.mn_adjoint(T, G, blk, sa, ss, q, tgt, dt, 8, u0, a0.copy(), bc=1, tau=1e-13)
    Jr, gsar, gssr = O.mn_adjoint(T, Gr, blk, sa, ss, q, tgt, dt, 8, u0, a0.copy(), bc=1, tau=1e-13)
    scale = max(np.abs(gsa).max(), np.abs(gss).max())
    print("adjoint mirror: J", abs(Jr - J) / abs(J), "grad", max(np.abs(gsar - gsa).max(), np.abs(gssr - gss).max()) / scale)
    assert abs(Jr - J) <= 1e-13 * abs(J)
    assert np.abs(gsar - gsa).max() <= 1e-12 * scale and np.abs(gssr - gss).max() <= 1e-12 * scale
