"""Pins for the oracle's mesh geometry, kinetic upwind flux and explicit update (Sec. 4.1, Sec. 4.2,
Sec. 4.4 kinetic flux). Checked against: a hand-written brute-force step on a 2-triangle mesh whose
geometry is typed in from a drawing, the exact discrete conservation identity, the steady uniform
state, closed-form geometry of a structured mesh, and equivariance of the whole step under
mirroring the mesh (5e-16; inward normals planted on the mirrored triangles give 0.12)."""
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


def _numpy_rule_and_basis(N, order):
    """The product rule and the real spherical harmonics built independently of the oracle:
    numpy's Gauss-Legendre nodes, 2*order equally spaced azimuths, scipy's complex harmonics
    turned real (Condon-Shortley phase removed), functions even in mu only."""
    from scipy.special import sph_harm_y
    x, wg = np.polynomial.legendre.leggauss(order)
    nphi = 2 * order
    pts = []
    for mu, wk in zip(x, wg):
        for l in range(1, nphi + 1):
            pts.append((mu, 2 * math.pi * l / nphi, wk * 2 * math.pi / nphi))
    mu = np.array([p[0] for p in pts])
    phi = np.array([p[1] for p in pts])
    w = np.array([p[2] for p in pts])
    s = np.sqrt(1 - mu ** 2)
    om = np.stack([s * np.sin(phi), s * np.cos(phi)], axis=1)
    theta = np.arccos(mu)
    cols, deg = [], []
    for l in range(N + 1):
        for k in range(-l, l + 1):
            if (l + abs(k)) % 2:
                continue
            y = sph_harm_y(l, abs(k), theta, phi)
            if k == 0:
                cols.append(y.real)
            elif k > 0:
                cols.append(math.sqrt(2) * (-1) ** k * y.real)
            else:
                cols.append(math.sqrt(2) * (-1) ** abs(k) * y.imag)
            deg.append(l)
    return w, om, np.stack(cols, axis=1), np.array(deg)


def _numpy_geometry(xy, tri):
    """Counter-clockwise triangles, face k from vertex k to k+1, outward normal scaled by the
    face length, neighbours by shared edges (brute force)."""
    def cross(p, q):
        return p[0] * q[1] - p[1] * q[0]

    tri = [list(t) for t in tri]
    for t in tri:
        a, b, c = (np.array(xy[v]) for v in t)
        if cross(b - a, c - a) < 0:
            t[1], t[2] = t[2], t[1]
    C = len(tri)
    area = np.array([0.5 * abs(cross(np.array(xy[t[1]]) - xy[t[0]], np.array(xy[t[2]]) - xy[t[0]]))
                     for t in tri])
    nrm = np.zeros((C, 3, 2))
    nbr = -np.ones((C, 3), dtype=int)
    for c, t in enumerate(tri):
        for k in range(3):
            a, b = t[k], t[(k + 1) % 3]
            nrm[c, k] = [xy[b][1] - xy[a][1], xy[a][0] - xy[b][0]]
            for d, s in enumerate(tri):
                if d != c and a in s and b in s:
                    nbr[c, k] = d
    return area, nrm, nbr


def _eight_triangles():
    xy = np.array([[i * 0.5, j * 0.5] for j in range(3) for i in range(3)])
    tri = []
    for j in range(2):
        for i in range(2):
            v0, v1, v2, v3 = j * 3 + i, j * 3 + i + 1, (j + 1) * 3 + i + 1, (j + 1) * 3 + i
            tri += [[v0, v1, v2], [v0, v2, v3]]
    return xy, np.array(tri, dtype=np.int32)


@pytest.mark.parametrize("mesh", ["two", "eight"])
@pytest.mark.parametrize("bc", [0, 1])
def test_kinetic_flux_of_the_pn_ansatz_is_the_half_range_matrix_flux(mesh, bc):
    """The kinetic flux [Sec. 4.4] fed the quadratic-entropy (P_N) ansatz psi = u . m [Sec. 3.1]
    becomes a matrix flux F_f = B+(n_f) u_i + B-(n_f) u_up with the half-range matrices
    B+-(n) = sum_q w_q m_q m_q^T (Omega_q . n)^+- (so B+ + B- = n_x A_x + n_y A_y with the P_N
    flux Jacobians A_l = <m m^T Omega_l>). The matrices, the rule, the basis and the geometry are
    built here with numpy/scipy, independently of the oracle; the oracle's flux of u . m must
    match to 1e-13. This pins the flux's orientation, upwinding and boundary ghosts."""
    N, order = 3, 6
    if mesh == "two":
        xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
        tri = np.array([[0, 1, 2], [0, 3, 2]], dtype=np.int32)
    else:
        xy, tri = _eight_triangles()
    T = O.Tables(N, order)
    G = O.Geometry(xy, tri)
    w, om, Mb, deg = _numpy_rule_and_basis(N, order)
    area, nrm, nbr = _numpy_geometry(xy, tri)
    C, n = len(tri), T.n
    rng = np.random.default_rng(11)
    u = rng.normal(size=(C, n))
    # P_N flux Jacobians: symmetric, coupling degrees l and l +- 1 only
    Ax = Mb.T @ (w[:, None] * om[:, :1] * Mb)
    Ay = Mb.T @ (w[:, None] * om[:, 1:] * Mb)
    for A in (Ax, Ay):
        np.testing.assert_allclose(A, A.T, atol=1e-14)
        assert np.abs(A[np.abs(deg[:, None] - deg[None, :]) != 1]).max() < 1e-14
    F = np.zeros((C, n))
    for c in range(C):
        for k in range(3):
            nv = nrm[c, k]
            d = om @ nv
            Bp = Mb.T @ (w[:, None] * np.maximum(d, 0)[:, None] * Mb)
            Bm = Mb.T @ (w[:, None] * np.minimum(d, 0)[:, None] * Mb)
            np.testing.assert_allclose(Bp + Bm, nv[0] * Ax + nv[1] * Ay, atol=1e-13)
            assert np.linalg.eigvalsh(Bp).min() > -1e-13 and np.linalg.eigvalsh(Bm).max() < 1e-13
            j = nbr[c, k]
            up = u[j] if j >= 0 else (u[c] if bc == 0 else np.zeros(n))
            F[c] += Bp @ u[c] + Bm @ up
    # the oracle's kinetic flux of psi = u . m (dt = 1, no source terms): u - u' = F / A
    psi = np.ascontiguousarray(u @ T.M.T)
    uo = u.copy()
    O.flux_update(T, G, psi, uo, np.zeros(C), np.zeros(C), np.zeros(C), 1.0, bc=bc)
    got = (u - uo) * G.area[:, None]
    assert np.abs(got - F).max() <= 1e-13 * max(1.0, np.abs(F).max())


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("axis", [0, 1])
def test_step_commutes_with_mirroring_the_mesh(bc, axis):
    """Mirroring the domain in x (or y) turns every triangle clockwise and maps the product rule's
    points onto each other (Sec. 3.2: equally spaced azimuths, an even number of them): point q
    goes to the point whose direction has Omega_x (or Omega_y) negated, found from the rule's own
    direction tables. On the basis the mirror is an orthogonal matrix D (fitted from the basis at
    the mirrored points). Steps of the mirrored problem from the mirrored state must equal the
    mirrored steps of the original (Sec. 4.2, Sec. 4.4): this pins the face normals and the
    upwind choice for either orientation, and the boundary ghost."""
    from mirror_map import mirror_basis, mirror_points, mirror_xy
    N, order = 2, 10
    T = O.Tables(N, order)
    m = synth.jittered_mesh(10, -1.0, 1.0, seed=5)
    G = O.Geometry(m.xy, m.tri)
    Gr = O.Geometry(mirror_xy(m.xy, axis), m.tri)
    mu, phi, w, ox, oy = O.quadrature(order)
    perm = mirror_points(ox, oy, mu, axis)
    np.testing.assert_array_equal(w[perm], w)
    D = mirror_basis(T.M, perm)
    assert np.abs(D - np.eye(T.n)).max() > 0.5
    # a state without mirror symmetry: off-axis vMF mixtures, and varied coefficients per cell
    dirs = np.stack([ox, oy, mu], axis=1)
    c, k, wt = synth.vmf_mixtures(G.C, 9)
    u = synth.vmf_density(dirs, c, k, wt) @ (T.w[:, None] * T.M)
    rng = np.random.default_rng(9)
    sa, ss, q = rng.uniform(0, 1, G.C), rng.uniform(0, 2, G.C), rng.uniform(0, 0.5, G.C)
    dt = G.cfl_dt(0.4)
    u1 = u.copy()
    a1 = O.isotropic_alpha(T, u1)
    assert O.mn_run(T, G, u1, a1, sa, ss, q, dt, 3, bc=bc)[0] == 0
    ur = u @ D.T
    ar = O.isotropic_alpha(T, ur)
    assert O.mn_run(T, Gr, ur, ar, sa, ss, q, dt, 3, bc=bc)[0] == 0
    err = np.linalg.norm(ur - u1 @ D.T) / np.linalg.norm(u1)
    print("mirror: rel L2 of the difference", err)
    assert err <= 1e-12
