"""Pins for the oracle's entropy closure (Sec. 3.1, Eq. entropyOCP, Maxwell-Boltzmann entropy).

Checked against: the isotropic closed form, the exact M_1 (Langevin) moments of exp(a + b.Omega)
on S^2, moment reproduction for random realizable moments, uniqueness of the minimiser (strict
convexity), and equivariance under the product rule's azimuthal rotations and reflection (a 0.1%
error in one quadrature weight moves alpha by about 4e-6 there, against a 1e-10 bar)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_08417_gb300 import synth


def vmf_moments(T, count, seed):
    mu, phi, w, ox, oy = O.quadrature(T.order)
    dirs = np.stack([ox, oy, mu], axis=1)
    c, k, wt = synth.vmf_mixtures(count, seed)
    psi = synth.vmf_density(dirs, c, k, wt)          # [count, Q]
    scale = np.exp(np.random.default_rng(seed + 1).uniform(-3, 3, size=count))
    return (psi * scale[:, None]) @ (T.w[:, None] * T.M)


@pytest.mark.parametrize("N,order", [(2, 10), (3, 20), (5, 12)])
def test_isotropic_closed_form(N, order):
    T = O.Tables(N, order)
    rng = np.random.default_rng(0)
    u = np.zeros((16, T.n))
    u[:, 0] = np.exp(rng.uniform(-8, 4, size=16))
    exact = O.isotropic_alpha(T, u)
    # closed form alpha_0 = sqrt(4 pi) ln(u_0 / sqrt(4 pi)) when m_0 = 1/sqrt(4 pi)
    np.testing.assert_allclose(exact[:, 0], math.sqrt(4 * math.pi) * np.log(u[:, 0] / math.sqrt(4 * math.pi)),
                               rtol=1e-14)
    # Newton from a perturbed start converges to it
    a = exact + rng.normal(scale=0.3, size=exact.shape)
    st, it = O.closure(T, u, a)
    assert (st == 0).all()
    np.testing.assert_allclose(a, exact, atol=1e-12 * np.abs(exact).max())


@pytest.mark.parametrize("N,order,tol", [(2, 10, 1e-10), (3, 20, 1e-10), (5, 30, 1e-10)])
def test_moment_reproduction_and_uniqueness(N, order, tol):
    T = O.Tables(N, order)
    u = vmf_moments(T, 64, seed=7)
    a1 = O.isotropic_alpha(T, u)
    st, it = O.closure(T, u, a1, tau=tol, polish=False)
    ok = st == 0
    assert ok.mean() > 0.9, st
    rec = np.exp(a1 @ T.M.T) @ (T.w[:, None] * T.M)
    rel = np.linalg.norm(rec - u, axis=1) / np.linalg.norm(u, axis=1)
    assert rel[ok].max() <= tol
    # a second, unrelated start reaches the same minimiser (strict convexity): the two answers
    # differ by no more than ||H^-1|| (||g_1|| + ||g_2||), with H the Hessian of the dual
    a2 = O.isotropic_alpha(T, u) + np.random.default_rng(3).normal(scale=0.05, size=u.shape)
    st2, _ = O.closure(T, u, a2, tau=tol, polish=False)
    both = np.flatnonzero(ok & (st2 == 0))
    assert both.size > 0.9 * u.shape[0]
    for i in both:
        e1 = T.w * np.exp(T.M @ a1[i])
        e2 = T.w * np.exp(T.M @ a2[i])
        H = T.M.T @ (e1[:, None] * T.M)
        g1 = np.linalg.norm(T.M.T @ e1 - u[i])
        g2 = np.linalg.norm(T.M.T @ e2 - u[i])
        bound = (g1 + g2) / np.linalg.eigvalsh(H)[0]
        assert np.linalg.norm(a1[i] - a2[i]) <= 2.0 * bound + 1e-13 * np.linalg.norm(a1[i])


def test_m1_langevin_closed_form():
    """N = 1: the ansatz is exp(A + B.Omega) with B in the x-y plane. On S^2,
    <e> = 4 pi e^A sinh|B|/|B| and <Omega e> = L(|B|) B/|B| <e>, L(x) = coth x - 1/x."""
    T = O.Tables(1, 40)
    c = math.sqrt(3 / (4 * math.pi))
    m0 = 1 / math.sqrt(4 * math.pi)
    rng = np.random.default_rng(11)
    cases = []
    for _ in range(12):
        alpha = np.array([rng.uniform(-3, 3), *rng.uniform(-4, 4, size=2)])
        A = alpha[0] * m0
        B = c * alpha[1:]
        b = np.linalg.norm(B)
        mass = 4 * math.pi * math.exp(A) * math.sinh(b) / b
        L = 1 / math.tanh(b) - 1 / b
        u = np.array([m0 * mass, c * L * B[0] / b * mass, c * L * B[1] / b * mass])
        cases.append((alpha, u))
    u = np.array([cu for _, cu in cases])
    a = O.isotropic_alpha(T, u)
    st, _ = O.closure(T, u, a, tau=1e-13)
    assert (st == 0).all()
    np.testing.assert_allclose(a, np.array([ca for ca, _ in cases]), rtol=1e-11, atol=1e-11)


def test_nonrealizable_reports_failure():
    """A moment vector outside the realizable set (|u_1| too large for u_0) has no minimiser; the
    oracle must report a failure status rather than return an answer."""
    T = O.Tables(1, 10)
    u = np.array([[1.0, 5.0, 0.0]])
    a = O.isotropic_alpha(T, u)
    st, _ = O.closure(T, u, a)
    assert st[0] != 0


@pytest.mark.parametrize("N,order", [(2, 10), (3, 20)])
def test_closure_commutes_with_the_rules_azimuthal_symmetries(N, order):
    """Rotating a state about the pole by a multiple of the product rule's azimuthal step
    2 pi / N_phi (Sec. 3.2: equally spaced azimuths) maps the rule's points onto each other, and so
    does the reflection phi -> -phi. On the basis such a map is an orthogonal matrix R (fitted here
    from the basis at the moved points; the degree-N space is invariant), the moments of the moved
    state are R u, and the minimiser of the dual (Sec. 3.1) must move with it:
    alpha(R u) = R alpha(u). A misplaced weight, point or sign in the closure breaks this."""
    T = O.Tables(N, order)
    mu, phi, w, ox, oy = O.quadrature(order)
    nphi = 2 * order
    u = vmf_moments(T, 24, seed=11)
    a = O.isotropic_alpha(T, u)
    st, _ = O.closure(T, u, a)
    for moved in (phi + 2 * math.pi * 3 / nphi, phi + 2 * math.pi * 7 / nphi, -phi):
        Mm = np.array([O.basis(N, m_, p_) for m_, p_ in zip(mu, moved)])
        R = np.linalg.lstsq(T.M, Mm, rcond=None)[0].T
        assert np.abs(T.M @ R.T - Mm).max() < 1e-12
        assert np.abs(R @ R.T - np.eye(T.n)).max() < 1e-12
        assert np.abs(R - np.eye(T.n)).max() > 0.1  # the map moves the state
        ur = u @ R.T
        ar = O.isotropic_alpha(T, ur)
        st_r, _ = O.closure(T, ur, ar)
        ok = (st == 0) & (st_r == 0)
        assert ok.mean() > 0.9
        err = np.linalg.norm(ar[ok] - a[ok] @ R.T, axis=1) / np.linalg.norm(a[ok], axis=1)
        print("symmetry: max rel diff of alpha", err.max())
        assert err.max() <= 1e-10
