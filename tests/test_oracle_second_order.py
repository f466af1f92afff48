"""Pins for the oracle's second-order scheme (Sec. 4.3): the Green-Gauss gradient, the
Barth-Jespersen limiter, the reconstructed face values and the Heun time step, each checked
against a closed form or an invariant rather than against itself:
- on a mesh whose interior faces are all shared by parallelogram pairs (squares split along one
  diagonal), the face average of the two centroid values is the value at the face midpoint, so
  the Green-Gauss gradient of a linear field is exact in every interior cell, the reconstruction
  reproduces the field at the face midpoints and the limiter stays at 1;
- every limited face value lies between the two cell values it separates, on random data;
- a strict local extremum is limited to first order (limiter 0);
- the unlimited reconstruction of a smooth field converges at second order at the faces;
- Heun on a uniform state (no flux) multiplies each moment by 1 - s dt + (s dt)^2 / 2 with s its
  decay rate, which also pins the reading dt R (not dt R / A_i) of the Heun stages;
- the second-order step conserves mass up to the boundary flux (zero for an isotropic floor);
- the steps commute with mirroring the mesh in x or y (3e-16; face offsets planted reversed on the
  mirrored triangles give 1.3e-2)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_08417_gb300 import synth


def _split_squares(k, lo=0.0, hi=1.0):
    """k x k squares, each split along its rising diagonal."""
    x = np.linspace(lo, hi, k + 1)
    xy = np.array([[x[i], x[j]] for j in range(k + 1) for i in range(k + 1)])
    tri = []
    for j in range(k):
        for i in range(k):
            v0, v1, v2, v3 = j * (k + 1) + i, j * (k + 1) + i + 1, (j + 1) * (k + 1) + i + 1, (j + 1) * (k + 1) + i
            tri += [[v0, v1, v2], [v0, v2, v3]]
    return xy, np.array(tri, dtype=np.int32)


def _interior(G):
    return (G.nbr >= 0).all(axis=1)


def test_green_gauss_exact_and_limiter_inactive_on_linear_fields():
    xy, tri = _split_squares(8)
    G = O.Geometry(xy, tri)
    rng = np.random.default_rng(0)
    a, b = rng.normal(size=(4,)), rng.normal(size=(4, 2))
    psi = a[None, :] + G.cen @ b.T            # 4 independent linear "ordinates"
    grad, lim, psif = O.reconstruct(G, psi)
    inner = _interior(G)
    assert inner.sum() > 50
    np.testing.assert_allclose(grad[inner], np.broadcast_to(b, grad[inner].shape), atol=1e-12)
    assert np.all(lim[inner] == 1.0)
    mid = G.cen[:, None, :] + G.r              # face midpoints [C, 3, 2]
    exact = a[None, None, :] + mid @ b.T       # [C, 3, 4]
    np.testing.assert_allclose(psif[inner], np.transpose(exact, (0, 1, 2))[inner], atol=1e-12)


def test_face_offsets_point_to_the_face_midpoints():
    xy, tri = _split_squares(3)
    G = O.Geometry(xy, tri)
    for c in range(G.C):
        for k in range(3):
            # the midpoint lies on the face: (mid - a) is parallel to the face, orthogonal to n
            mid = G.cen[c] + G.r[c, k]
            n = G.nrm[c, k]
            # distance from the midpoint to the face line through either endpoint is zero
            v = [xy[t] for t in tri[c]]
            on = min(abs(np.dot(mid - p, n)) for p in v)
            assert on < 1e-14


@pytest.mark.parametrize("bc", [0, 1])
def test_limited_face_values_stay_between_the_cell_values(bc):
    m = synth.jittered_mesh(10, 0.0, 1.0, seed=3)
    G = O.Geometry(m.xy, m.tri)
    rng = np.random.default_rng(1)
    psi = rng.uniform(0.0, 1.0, size=(G.C, 5))
    _, lim, psif = O.reconstruct(G, psi, bc=bc)
    assert (lim >= 0).all() and (lim <= 1).all()
    for k in range(3):
        j = G.nbr[:, k]
        other = np.where((j >= 0)[:, None], psi[np.maximum(j, 0)], psi if bc == 0 else 0.0)
        lo, hi = np.minimum(psi, other), np.maximum(psi, other)
        f = psif[:, k, :]
        assert (f >= lo - 1e-15).all() and (f <= hi + 1e-15).all()


def test_strict_extremum_is_limited_to_first_order():
    xy, tri = _split_squares(6)
    G = O.Geometry(xy, tri)
    psi = np.ones((G.C, 1))
    peak = int(np.flatnonzero(_interior(G))[7])
    psi[peak, 0] = 3.0
    # neighbours of the peak hold distinct values below it so that its gradient is non-zero
    for k, j in enumerate(G.nbr[peak]):
        psi[j, 0] = 1.0 + 0.3 * k
    _, lim, psif = O.reconstruct(G, psi)
    assert lim[peak, 0] == 0.0
    np.testing.assert_array_equal(psif[peak, :, 0], 3.0)


def test_reconstruction_of_a_smooth_field_converges_at_second_order():
    def face_error(k):
        xy, tri = _split_squares(k)
        G = O.Geometry(xy, tri)
        f = lambda p: np.exp(0.7 * p[..., 0] + 0.4 * p[..., 1])
        psi = f(G.cen)[:, None]
        _, lim, psif = O.reconstruct(G, psi)
        inner = _interior(G) & (lim[:, 0] == 1.0)
        exact = f(G.cen[:, None, :] + G.r)
        return np.abs(psif[inner, :, 0] - exact[inner]).max()

    e1, e2 = face_error(8), face_error(16)
    assert e1 / e2 > 3.5, (e1, e2)


@pytest.mark.parametrize("bc", [0])
def test_heun_on_a_uniform_state_is_the_second_order_taylor_factor(bc):
    N, order = 2, 6
    T = O.Tables(N, order)
    xy, tri = _split_squares(4)
    G = O.Geometry(xy, tri)
    C = G.C
    # a uniform anisotropic state: the same realizable moment vector in every cell
    mu, phi, w, ox, oy = O.quadrature(order)
    c, kap, wt = synth.vmf_mixtures(1, 5, kappa_hi=3.0)
    u1 = synth.vmf_density(np.stack([ox, oy, mu], axis=1), c, kap, wt) @ (T.w[:, None] * T.M)
    u = np.repeat(u1, C, axis=0)
    alpha = O.isotropic_alpha(T, u)
    sa, ss = np.full(C, 0.7), np.full(C, 0.4)
    dt = 0.05
    u_new = u.copy()
    nf, _ = O.mn_run2(T, G, u_new, alpha, sa, ss, np.zeros(C), dt, 1, bc=bc, tau=1e-13)
    assert nf == 0
    rate = np.full(T.n, sa[0] + ss[0])
    rate[0] = sa[0]                           # scattering keeps the zeroth moment
    factor = 1 - rate * dt + (rate * dt) ** 2 / 2
    np.testing.assert_allclose(u_new, u * factor[None, :], rtol=1e-12, atol=1e-15)


def test_second_order_line_source_conserves_mass_and_stays_positive():
    N, order = 2, 6
    T = O.Tables(N, order)
    m = synth.jittered_mesh(20, -1.5, 1.5, seed=1)
    G = O.Geometry(m.xy, m.tri)
    # a pulse narrow enough that the boundary cells hold the isotropic floor exactly (their
    # boundary flux is then zero)
    u = synth.isotropic_moments(synth.line_source_density(G.cen, width=0.1), T.n)
    alpha = O.isotropic_alpha(T, u)
    C = G.C
    dt = G.cfl_dt(0.4)
    mass0 = (G.area * u[:, 0]).sum()
    nf, _ = O.mn_run2(T, G, u, alpha, np.zeros(C), np.ones(C), np.zeros(C), dt, 5)
    assert nf == 0
    assert abs((G.area * u[:, 0]).sum() / mass0 - 1) < 1e-13
    psi = O.ansatz(T, alpha)
    assert (psi > 0).all()


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("axis", [0, 1])
def test_second_order_step_commutes_with_mirroring_the_mesh(bc, axis):
    """Second-order steps (Sec. 4.3: Green-Gauss gradient, Barth-Jespersen limiter, Heun) on the
    mesh mirrored in x or y, from the mirrored moments, equal the mirrored steps: pins the face
    offsets, the gradient's orientation and the limiter's per-face bounds for clockwise
    triangles."""
    from mirror_map import mirror_basis, mirror_points, mirror_xy
    N, order = 2, 10
    T = O.Tables(N, order)
    m = synth.jittered_mesh(10, -1.0, 1.0, seed=7)
    G, Gr = O.Geometry(m.xy, m.tri), O.Geometry(mirror_xy(m.xy, axis), m.tri)
    mu, phi, w, ox, oy = O.quadrature(order)
    D = mirror_basis(T.M, mirror_points(ox, oy, mu, axis))
    c, k, wt = synth.vmf_mixtures(G.C, 13)
    u = synth.vmf_density(np.stack([ox, oy, mu], axis=1), c, k, wt) @ (T.w[:, None] * T.M)
    rng = np.random.default_rng(13)
    sa, ss, q = rng.uniform(0, 1, G.C), rng.uniform(0, 2, G.C), rng.uniform(0, 0.5, G.C)
    dt = G.cfl_dt(0.4)
    u1 = u.copy()
    a1 = O.isotropic_alpha(T, u1)
    assert O.mn_run2(T, G, u1, a1, sa, ss, q, dt, 3, bc=bc)[0] == 0
    ur = u @ D.T
    ar = O.isotropic_alpha(T, ur)
    assert O.mn_run2(T, Gr, ur, ar, sa, ss, q, dt, 3, bc=bc)[0] == 0
    err = np.linalg.norm(ur - u1 @ D.T) / np.linalg.norm(u1)
    print("second-order mirror diff", err)
    assert err <= 1e-12
