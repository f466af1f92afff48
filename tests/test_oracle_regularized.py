"""Pins for the oracle's (partially) regularized closure (Sec. 3.1, Eq. entropyOCP_reg and
Eq. entropyOCP_part_reg), checked against closed forms and convex duality rather than against
the closure code itself:
- M_1 with regularization: for a chosen alpha the regularized problem's moments are the exact
  sphere integrals (Langevin function) shifted by gamma alpha^r; the closure must recover alpha;
- strong duality: the primal objective (entropy plus the quadratic penalty) at the ansatz equals
  minus the dual minimum, and the ansatz keeps u_0 exactly (partial form) while its regularized
  moments fall short of u^r by gamma alpha^r;
- the regularized closure tends to the entropy closure linearly in gamma;
- it is solvable outside the realizable set, where the entropy closure has no minimiser;
- the isotropic closed form is unchanged (alpha^r = 0 is optimal for u^r = 0)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_08417_gb300 import synth


def _vmf_u(T, count, seed, kappa_hi=20.0):
    mu, phi, w, ox, oy = O.quadrature(T.order)
    c, k, wt = synth.vmf_mixtures(count, seed, kappa_hi=kappa_hi)
    psi = synth.vmf_density(np.stack([ox, oy, mu], axis=1), c, k, wt)
    return psi @ (T.w[:, None] * T.M)


@pytest.mark.parametrize("reg0", [0, 1])
def test_m1_regularized_closed_form(reg0):
    """N = 1, ansatz exp(A + B.Omega): <e> = 4 pi e^A sinh|B|/|B|, <Omega e> = L(|B|) B/|B| <e>.
    The regularized problem with data u = <m e> + gamma alpha^r has the minimiser alpha."""
    gamma = 1e-2
    T = O.Tables(1, 40)
    c = math.sqrt(3 / (4 * math.pi))
    m0 = 1 / math.sqrt(4 * math.pi)
    rng = np.random.default_rng(12)
    alphas, us = [], []
    for _ in range(10):
        alpha = np.array([rng.uniform(-3, 3), *rng.uniform(-4, 4, size=2)])
        A, B = alpha[0] * m0, c * alpha[1:]
        b = np.linalg.norm(B)
        mass = 4 * math.pi * math.exp(A) * math.sinh(b) / b
        L = 1 / math.tanh(b) - 1 / b
        u = np.array([m0 * mass, c * L * B[0] / b * mass, c * L * B[1] / b * mass])
        u[reg0:] += gamma * alpha[reg0:]
        alphas.append(alpha)
        us.append(u)
    u = np.array(us)
    a = O.isotropic_alpha(T, u)
    st, _ = O.closure_reg(T, u, a, gamma, reg0, tau=1e-13)
    assert (st == 0).all()
    np.testing.assert_allclose(a, np.array(alphas), rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("N,order", [(2, 10), (3, 10)])
def test_strong_duality_and_the_moments_of_the_regularized_ansatz(N, order):
    gamma = 1e-3
    T = O.Tables(N, order)
    u = _vmf_u(T, 40, seed=3)
    a = O.isotropic_alpha(T, u)
    st, _ = O.closure_reg(T, u, a, gamma, 1, tau=1e-13)
    assert (st == 0).all()
    for i in range(u.shape[0]):
        psi = np.exp(T.M @ a[i])
        mom = T.M.T @ (T.w * psi)
        # u_0 kept exactly, the regularized moments short by gamma alpha^r
        assert abs(mom[0] - u[i, 0]) <= 1e-11 * abs(u[i, 0])
        np.testing.assert_allclose(mom[1:], u[i, 1:] - gamma * a[i, 1:], atol=1e-11 * np.abs(u[i]).max())
        # primal: entropy psi ln psi - psi plus the penalty; dual: <e> - alpha.u + gamma/2 |alpha^r|^2
        primal = np.dot(T.w, psi * np.log(psi) - psi) + np.sum((mom[1:] - u[i, 1:]) ** 2) / (2 * gamma)
        dual_min = np.dot(T.w, psi) - np.dot(a[i], u[i]) + 0.5 * gamma * np.sum(a[i, 1:] ** 2)
        scale = np.dot(T.w, psi) + abs(np.dot(a[i], u[i]))
        assert abs(primal + dual_min) <= 1e-11 * scale


def test_regularized_closure_tends_to_the_entropy_closure_linearly():
    """alpha_gamma - alpha_0 = -gamma H^-1 alpha_0^r + O(gamma^2): linear once gamma is well below
    the smallest eigenvalue of the dual Hessian (smooth densities keep it away from zero)."""
    T = O.Tables(2, 10)
    u = _vmf_u(T, 20, seed=5, kappa_hi=2.0)
    a0 = O.isotropic_alpha(T, u)
    assert (O.closure(T, u, a0, tau=1e-13)[0] == 0).all()
    diffs = []
    for gamma in (1e-8, 1e-7, 1e-6):
        a = O.isotropic_alpha(T, u)
        assert (O.closure_reg(T, u, a, gamma, 1, tau=1e-13)[0] == 0).all()
        diffs.append(np.linalg.norm(a - a0))
    r1, r2 = diffs[1] / diffs[0], diffs[2] / diffs[1]
    assert 9.0 < r1 < 11.0 and 9.0 < r2 < 11.0, diffs


def test_regularized_closure_is_solvable_outside_the_realizable_set():
    """|u_1| too large for u_0: no minimiser of the entropy closure; the partially regularized
    problem (gamma = 1e-3, u_0 exact, as in the paper's regularized M_3 run) has one."""
    T = O.Tables(1, 10)
    u = np.array([[1.0, 5.0, 0.0]])
    a = O.isotropic_alpha(T, u)
    assert O.closure(T, u, a.copy())[0][0] != 0
    st, _ = O.closure_reg(T, u, a, 1e-3, 1, tau=1e-12)
    assert st[0] == 0
    mom = T.M.T @ (T.w * np.exp(T.M @ a[0]))
    assert abs(mom[0] - 1.0) < 1e-12


def test_isotropic_closed_form_is_unchanged_by_regularization():
    T = O.Tables(3, 10)
    u = np.zeros((5, T.n))
    u[:, 0] = np.linspace(0.1, 3.0, 5)
    a = O.isotropic_alpha(T, u)
    ref = a.copy()
    st, _ = O.closure_reg(T, u, a, 1e-3, 1, tau=1e-13, polish=False)
    assert (st == 0).all()
    np.testing.assert_allclose(a, ref, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("reg0", [0, 1])
def test_regularized_closure_commutes_with_the_rules_mirrors(reg0):
    """The penalty gamma/2 |alpha_reg|^2 of Eq. entropyOCP_reg / _part_reg is invariant under the
    product rule's mirrors, which act on the basis as an orthogonal D that keeps m_0, so the
    regularized minimiser moves with the state: alpha(D u) = D alpha(u)."""
    from mirror_map import mirror_basis, mirror_points
    N, order = 3, 12
    T = O.Tables(N, order)
    mu, phi, w, ox, oy = O.quadrature(order)
    c, k, wt = synth.vmf_mixtures(32, 5)
    u = synth.vmf_density(np.stack([ox, oy, mu], axis=1), c, k, wt) @ (T.w[:, None] * T.M)
    a = O.isotropic_alpha(T, u)
    st, _ = O.closure_reg(T, u, a, 1e-2, reg0=reg0)
    for axis in (0, 1):
        D = mirror_basis(T.M, mirror_points(ox, oy, mu, axis))
        assert abs(D[0, 0] - 1.0) < 1e-12
        ur = u @ D.T
        ar = O.isotropic_alpha(T, ur)
        st_r, _ = O.closure_reg(T, ur, ar, 1e-2, reg0=reg0)
        ok = (st == 0) & (st_r == 0)
        assert ok.mean() > 0.9
        err = np.linalg.norm(ar[ok] - a[ok] @ D.T, axis=1) / np.linalg.norm(a[ok], axis=1)
        print("regularized mirror diff", err.max())
        assert err.max() <= 1e-10
