"""Pins for the oracle's mesh geometry, kinetic upwind flux and explicit update (Sec. 4.1, Sec. 4.2,
Sec. 4.4 kinetic flux). Checked against: a hand-written brute-force step on a 2-triangle mesh whose
geometry is typed in from a drawing, the exact discrete conservation identity, the steady uniform
state, and closed-form geometry of a structured mesh."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_08417_gb300 import synth


def test_geometry_unit_square_two_triangles():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2], [0, 3, 2]], dtype=np.int32)   # second one given clockwise
    G = O.Geometry(xy, tri)
    np.testing.assert_allclose(G.area, [0.5, 0.5])
    np.testing.assert_allclose(G.perim, [2 + math.sqrt(2)] * 2)
    np.testing.assert_allclose(G.cen, [[2 / 3, 1 / 3], [1 / 3, 2 / 3]])
    # cell 0 faces: (0,0)->(1,0) bottom, (1,0)->(1,1) right, (1,1)->(0,0) diagonal
    np.testing.assert_array_equal(G.nrm[0], [[0, -1], [1, 0], [-1, 1]])
    np.testing.assert_array_equal(G.nbr[0], [-1, -1, 1])
    # cell 1 (re-oriented to 0,2,3): diagonal (0,0)->(1,1), top (1,1)->(0,1), left (0,1)->(0,0)
    np.testing.assert_array_equal(G.nrm[1], [[1, -1], [0, 1], [-1, 0]])
    np.testing.assert_array_equal(G.nbr[1], [0, -1, -1])


def test_geometry_closed_polygons_and_shared_faces():
    m = synth.jittered_mesh(12, -1.0, 1.0, seed=4)
    G = O.Geometry(m.xy, m.tri)
    # sum of scaled outward normals of a closed polygon vanishes
    assert np.abs(G.nrm.sum(axis=1)).max() < 1e-15
    assert abs(G.area.sum() - 4.0) < 1e-13
    # interior faces: the neighbour sees the exactly negated normal
    for c in range(G.C):
        for k in range(3):
            j = G.nbr[c, k]
            if j < 0:
                continue
            kk = list(G.nbr[j]).index(c)
            np.testing.assert_array_equal(G.nrm[j, kk], -G.nrm[c, k])
    # boundary faces lie on the square and sum to its perimeter
    b = G.nbr < 0
    assert abs(np.linalg.norm(G.nrm[b], axis=1).sum() - 8.0) < 1e-13


def _brute_force_two_triangles(T, alpha, u, sa, ss, qs, dt, bc):
    """One step on the unit square split along its diagonal, written out by hand:
    cell 0 = (0,0),(1,0),(1,1); cell 1 = (0,0),(1,1),(0,1); area 1/2 each."""
    faces = {0: [((0.0, -1.0), None), ((1.0, 0.0), None), ((-1.0, 1.0), 1)],
             1: [((1.0, -1.0), 0), ((0.0, 1.0), None), ((-1.0, 0.0), None)]}
    Q, n = T.M.shape
    psi = [[math.exp(sum(alpha[c][a] * T.M[q][a] for a in range(n))) for q in range(Q)]
           for c in range(2)]
    out = []
    for c in range(2):
        F = [0.0] * n
        for (nx, ny), j in faces[c]:
            for q in range(Q):
                d = T.ox[q] * nx + T.oy[q] * ny
                if d > 0:
                    up = psi[c][q]
                elif j is not None:
                    up = psi[j][q]
                else:
                    up = psi[c][q] if bc == 0 else 0.0
                for a in range(n):
                    F[a] += T.w[q] * T.M[q][a] * d * up
        mbar = [sum(T.w[q] * T.M[q][a] for q in range(Q)) for a in range(n)]
        new = []
        for a in range(n):
            R = -sa[c] * u[c][a] - ss[c] * (u[c][a] - (u[c][0] if a == 0 else 0.0)) + qs[c] * mbar[a]
            new.append(u[c][a] - dt / 0.5 * F[a] + dt * R)
        out.append(new)
    return np.array(out)


@pytest.mark.parametrize("bc", [0, 1])
def test_flux_update_brute_force_two_triangles(bc):
    T = O.Tables(2, 4)
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    G = O.Geometry(xy, tri)
    rng = np.random.default_rng(5)
    alpha = rng.normal(scale=0.5, size=(2, T.n))
    u = rng.normal(size=(2, T.n))
    sa, ss, qs = np.array([0.3, 1.2]), np.array([0.7, 0.1]), np.array([0.0, 2.0])
    dt = 0.01
    expect = _brute_force_two_triangles(T, alpha, u, sa, ss, qs, dt, bc)
    psi = O.ansatz(T, alpha)
    uu = u.copy()
    O.flux_update(T, G, psi, uu, sa, ss, qs, dt, bc=bc)
    np.testing.assert_allclose(uu, expect, rtol=1e-14, atol=1e-14)


def _random_state(T, G, seed):
    mu, phi, w, ox, oy = O.quadrature(T.order)
    dirs = np.stack([ox, oy, mu], axis=1)
    c, k, wt = synth.vmf_mixtures(G.C, seed, kappa_hi=5.0)
    psi = synth.vmf_density(dirs, c, k, wt)
    return psi @ (T.w[:, None] * T.M)


@pytest.mark.parametrize("bc", [0, 1])
def test_discrete_conservation_identity(bc):
    """With sigma_a = 0 and no source, interior faces cancel pairwise, so
    sum_i A_i u_i0^{n+1} = sum_i A_i u_i0^n - dt * (zeroth-moment flux through boundary faces)."""
    T = O.Tables(2, 6)
    m = synth.jittered_mesh(10, -1.0, 1.0, seed=8)
    G = O.Geometry(m.xy, m.tri)
    u = _random_state(T, G, seed=9)
    alpha = O.isotropic_alpha(T, u)
    st, _ = O.closure(T, u, alpha)
    assert (st == 0).all()
    psi = O.ansatz(T, alpha)
    dt = G.cfl_dt(0.4)
    before = float((G.area * u[:, 0]).sum())
    bflux = 0.0
    for c in range(G.C):
        for k in range(3):
            if G.nbr[c, k] >= 0:
                continue
            d = T.ox * G.nrm[c, k, 0] + T.oy * G.nrm[c, k, 1]
            ghost = psi[c] if bc == 0 else np.zeros(T.Q)
            up = np.where(d > 0, psi[c], ghost)
            bflux += float(np.sum(T.w * T.M[:, 0] * d * up))
    uu = u.copy()
    O.flux_update(T, G, psi, uu, np.zeros(G.C), np.ones(G.C), np.zeros(G.C), dt, bc=bc)
    after = float((G.area * uu[:, 0]).sum())
    assert abs(bflux) > 1e-6 * abs(before)      # the identity is not trivially 0 = 0
    assert abs(after - (before - dt * bflux)) <= 1e-12 * abs(before)


def test_uniform_state_is_steady_with_neumann():
    T = O.Tables(2, 10)
    m = synth.jittered_mesh(12, -1.5, 1.5, seed=1)
    G = O.Geometry(m.xy, m.tri)
    u = np.zeros((G.C, T.n))
    u[:, 0] = 0.37
    alpha = O.isotropic_alpha(T, u)
    u0 = u.copy()
    nf, st = O.mn_run(T, G, u, alpha, np.zeros(G.C), np.ones(G.C), np.zeros(G.C), G.cfl_dt(0.4), 5)
    assert nf == 0
    assert np.abs(u - u0).max() <= 1e-14 * 0.37 * 10


def test_line_source_mass_and_positivity():
    """Line-source start (Sec. 7.1 initial condition with a floor), Neumann walls, sigma_a = 0:
    total mass stays constant to round-off and every closure succeeds (psi > 0 by construction)."""
    T = O.Tables(2, 10)
    m = synth.jittered_mesh(20, -1.5, 1.5, seed=1)
    G = O.Geometry(m.xy, m.tri)
    u = synth.isotropic_moments(synth.line_source_density(G.cen, width=0.15), T.n)
    alpha = O.isotropic_alpha(T, u)
    mass0 = float((G.area * u[:, 0]).sum())
    nf, st = O.mn_run(T, G, u, alpha, np.zeros(G.C), np.ones(G.C), np.zeros(G.C), G.cfl_dt(0.4), 10)
    assert nf == 0
    assert abs(float((G.area * u[:, 0]).sum()) / mass0 - 1) < 1e-12
    assert (O.ansatz(T, alpha) > 0).all()
