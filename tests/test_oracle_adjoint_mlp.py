"""Pins for the oracle's discrete adjoint (checked against central finite differences of its own
forward objective, which is a different code path) and for its MLP backward pass and Adam step
(finite differences; Adam's first step has the closed form -lr * sign(g))."""
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
