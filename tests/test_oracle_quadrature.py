"""Pins for the oracle's quadrature and basis (Sec. 3.1 real spherical harmonics, Sec. 3.2 product
quadrature). Each check is against something other than the oracle itself: textbook closed forms,
scipy's complex spherical harmonics, or exactness properties of Gauss rules."""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gauss_legendre_closed_forms.txt")


def _closed_forms():
    rows = {}
    env = {"sqrt": math.sqrt}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            # columns are separated by two or more spaces; expressions use single spaces
            parts = line.split("  ")
            parts = [p.strip() for p in parts if p.strip()]
            n, node, wt = int(parts[0]), parts[1], parts[2]
            rows.setdefault(n, []).append((eval(node, env), eval(wt, env)))
    return rows


def test_gauss_legendre_closed_forms():
    for n, pairs in _closed_forms().items():
        x, w = O.gauss_legendre(n)
        exp_x, exp_w = [], []
        for node, wt in pairs:
            if node == 0:
                exp_x.append(0.0)
                exp_w.append(wt)
            else:
                exp_x += [-node, node]
                exp_w += [wt, wt]
        order = np.argsort(exp_x)
        np.testing.assert_allclose(x, np.array(exp_x)[order], atol=1e-15)
        np.testing.assert_allclose(w, np.array(exp_w)[order], rtol=1e-14)


@pytest.mark.parametrize("n", [6, 10, 20, 30])
def test_gauss_legendre_exactness(n):
    # integrates x^k exactly for k <= 2n-1: int_{-1}^{1} x^k = 2/(k+1) for even k, 0 for odd
    x, w = O.gauss_legendre(n)
    for k in range(2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** k) - exact) < 1e-13


@pytest.mark.parametrize("order", [4, 10, 20, 30])
def test_product_quadrature_weights_and_points(order):
    mu, phi, w, ox, oy = O.quadrature(order)
    assert mu.shape[0] == 2 * order * order
    assert abs(w.sum() - 4 * math.pi) < 1e-12
    # 2D projection of unit vectors: |Omega_2D|^2 = 1 - mu^2
    np.testing.assert_allclose(ox ** 2 + oy ** 2, 1 - mu ** 2, atol=1e-15)
    # symmetric rule: first moments vanish, second moments are 4pi/3 each
    assert abs(np.dot(w, ox)) < 1e-13 and abs(np.dot(w, oy)) < 1e-13
    np.testing.assert_allclose([np.dot(w, ox ** 2), np.dot(w, oy ** 2), np.dot(w, mu ** 2)],
                               4 * math.pi / 3, rtol=1e-13)


def _real_sh_scipy(N, mu, phi):
    """Real SH from scipy's complex Y_l^m (which carries the Condon-Shortley phase (-1)^m):
    m_l^k = sqrt2 (-1)^k Re Y_l^k (k>0), sqrt2 (-1)^|k| Im Y_l^|k| (k<0), Y_l^0 (k=0);
    only l+|k| even is kept (functions even in mu)."""
    from scipy.special import sph_harm_y
    theta = math.acos(mu)
    out = []
    for l in range(N + 1):
        for k in range(-l, l + 1):
            if (l + abs(k)) % 2:
                continue
            y = complex(sph_harm_y(l, abs(k), theta, phi))
            if k == 0:
                out.append(y.real)
            elif k > 0:
                out.append(math.sqrt(2) * (-1) ** k * y.real)
            else:
                out.append(math.sqrt(2) * (-1) ** abs(k) * y.imag)
    return np.array(out)


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_basis_matches_scipy_spherical_harmonics(N):
    rng = np.random.default_rng(0)
    for _ in range(20):
        mu = rng.uniform(-1, 1)
        phi = rng.uniform(0, 2 * math.pi)
        np.testing.assert_allclose(O.basis(N, mu, phi), _real_sh_scipy(N, mu, phi), atol=1e-13)
    assert O.basis(N, 0.3, 1.0).shape[0] == (N + 1) * (N + 2) // 2


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_basis_even_in_mu(N):
    for mu, phi in [(0.2, 0.7), (0.9, 4.0), (-0.5, 2.5)]:
        np.testing.assert_allclose(O.basis(N, mu, phi), O.basis(N, -mu, phi), atol=1e-15)


@pytest.mark.parametrize("N,order", [(1, 2), (2, 3), (2, 10), (3, 4), (3, 20), (5, 6), (5, 30)])
def test_basis_orthonormal_under_quadrature(N, order):
    T = O.Tables(N, order)
    G = T.M.T @ (T.w[:, None] * T.M)
    np.testing.assert_allclose(G, np.eye(T.n), atol=1e-13)
    # <m> = sqrt(4 pi) e_0 and m_0 = 1/sqrt(4 pi)
    mbar = T.M.T @ T.w
    e0 = np.zeros(T.n)
    e0[0] = math.sqrt(4 * math.pi)
    np.testing.assert_allclose(mbar, e0, atol=1e-13)
    np.testing.assert_allclose(T.M[:, 0], 1 / math.sqrt(4 * math.pi), rtol=1e-15)


def test_basis_first_order_is_projected_direction():
    # the l=1 functions kept in 2D are sqrt(3/(4pi)) Omega_x (k=-1) and sqrt(3/(4pi)) Omega_y (k=1)
    T = O.Tables(1, 5)
    c = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(T.M[:, 1], c * T.ox, atol=1e-15)
    np.testing.assert_allclose(T.M[:, 2], c * T.oy, atol=1e-15)
