"""Pins for the oracle's step of the transformed CSD equation (Sec. 2, Eq. BoltzmannCSDTrafo:
Omega . grad(psi / rho), cross sections depending on the pseudo-time only) and its dose (Sec. 2,
dose definition). Checked against: the plain step (rho = 1), the pseudo-time rescaling that a
constant density must be, a hand-written two-triangle step with two densities, the steady state
psi proportional to rho, the exact discrete conservation identity, and the density independence of
the dose of a uniform fluence in water-equivalent tissue."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_08417_gb300 import synth


def _state(T, G, seed):
    mu, phi, w, ox, oy = O.quadrature(T.order)
    dirs = np.stack([ox, oy, mu], axis=1)
    c, k, wt = synth.vmf_mixtures(G.C, seed, kappa_hi=5.0)
    return synth.vmf_density(dirs, c, k, wt)      # psi [C, Q] > 0


def _mesh(seed=8, k=10):
    m = synth.jittered_mesh(k, -1.0, 1.0, seed=seed)
    return O.Geometry(m.xy, m.tri)


@pytest.mark.parametrize("bc", [0, 1])
def test_unit_density_is_the_plain_step(bc):
    T = O.Tables(2, 6)
    G = _mesh()
    psi = _state(T, G, 3)
    u = psi @ (T.w[:, None] * T.M)
    rng = np.random.default_rng(1)
    sa, ss, q = rng.uniform(0, 1, G.C), rng.uniform(0, 1, G.C), rng.uniform(0, 1, G.C)
    a, b = u.copy(), u.copy()
    O.flux_update(T, G, psi, a, sa, ss, q, 0.01, bc=bc)
    O.flux_update_rho(T, G, np.ones(G.C), psi, b, sa, ss, q, 0.01, bc=bc)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("bc", [0, 1])
def test_constant_density_rescales_pseudo_time(bc):
    """rho = c makes particles move at speed 1/c: one step of length dt equals one plain step of
    length dt/c with cross sections and source multiplied by c."""
    T = O.Tables(2, 6)
    G = _mesh()
    psi = _state(T, G, 4)
    u = psi @ (T.w[:, None] * T.M)
    rng = np.random.default_rng(2)
    sa, ss, q = rng.uniform(0, 1, G.C), rng.uniform(0, 1, G.C), rng.uniform(0, 1, G.C)
    c, dt = 3.7, 0.02
    a, b = u.copy(), u.copy()
    O.flux_update_rho(T, G, np.full(G.C, c), psi, a, sa, ss, q, dt, bc=bc)
    O.flux_update(T, G, psi, b, c * sa, c * ss, c * q, dt / c, bc=bc)
    assert np.abs(a - u).max() > 1e-4 * np.abs(u).max()      # the step does something
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14 * np.abs(u).max())


def _brute_force_two_triangles_rho(T, psi, rho, u, sa, ss, qs, dt, bc):
    """One step on the unit square split along its diagonal, typed in from a drawing:
    cell 0 = (0,0),(1,0),(1,1); cell 1 = (0,0),(1,1),(0,1); area 1/2 each. The transported value
    across a face is psi / rho of the upwind cell."""
    faces = {0: [((0.0, -1.0), None), ((1.0, 0.0), None), ((-1.0, 1.0), 1)],
             1: [((1.0, -1.0), 0), ((0.0, 1.0), None), ((-1.0, 0.0), None)]}
    Q, n = T.M.shape
    out = []
    for c in range(2):
        F = [0.0] * n
        for (nx, ny), j in faces[c]:
            for q in range(Q):
                d = T.ox[q] * nx + T.oy[q] * ny
                if d > 0:
                    up = psi[c][q] / rho[c]
                elif j is not None:
                    up = psi[j][q] / rho[j]
                else:
                    up = psi[c][q] / rho[c] if bc == 0 else 0.0
                for a in range(n):
                    F[a] += T.w[q] * T.M[q][a] * d * up
        mbar = [sum(T.w[q] * T.M[q][a] for q in range(Q)) for a in range(n)]
        out.append([u[c][a] - dt / 0.5 * F[a] + dt * (-sa[c] * u[c][a] - ss[c] * (
            u[c][a] - (u[c][0] if a == 0 else 0.0)) + qs[c] * mbar[a]) for a in range(n)])
    return np.array(out)


@pytest.mark.parametrize("bc", [0, 1])
def test_brute_force_two_triangles_two_densities(bc):
    T = O.Tables(2, 4)
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    G = O.Geometry(xy, tri)
    rng = np.random.default_rng(6)
    psi = np.exp(rng.normal(scale=0.5, size=(2, T.Q)))
    u = rng.normal(size=(2, T.n))
    rho = np.array([1.0, 5.0])
    sa, ss, qs = np.array([0.3, 1.2]), np.array([0.7, 0.1]), np.array([0.0, 2.0])
    expect = _brute_force_two_triangles_rho(T, psi, rho, u, sa, ss, qs, 0.01, bc)
    uu = u.copy()
    O.flux_update_rho(T, G, rho, psi, uu, sa, ss, qs, 0.01, bc=bc)
    np.testing.assert_allclose(uu, expect, rtol=1e-14, atol=1e-14)


def _density(G):
    """Two tissues: density 1 on the left half, 5 on the right (the line-source density jump of
    the paper's Sec. 7.1 case), plus a denser disc."""
    rho = np.where(G.cen[:, 0] > 0.0, 5.0, 1.0)
    rho[np.hypot(G.cen[:, 0] + 0.4, G.cen[:, 1] - 0.3) < 0.25] = 2.5
    return rho


def test_psi_proportional_to_density_is_steady():
    """psi / rho uniform and isotropic, Neumann walls, no absorption or source: the transported
    value has no gradient, so the state is a fixed point of the step (with the closure); the plain
    step (no density) moves it."""
    T = O.Tables(2, 8)
    G = _mesh(seed=3, k=14)
    rho = _density(G)
    kappa = 0.21
    u = np.zeros((G.C, T.n))
    u[:, 0] = kappa * rho * 4 * math.pi * T.m0        # psi = kappa rho, u_0 = <m_0 psi>
    alpha = O.isotropic_alpha(T, u)
    dt = 0.4 * G.cfl_dt(1.0) * rho.min()
    sa, ss, q = np.zeros(G.C), np.ones(G.C), np.zeros(G.C)
    a = u.copy()
    nf, _ = O.mn_run_rho(T, G, rho, a, alpha.copy(), sa, ss, q, dt, 3)
    assert nf == 0
    assert np.abs(a - u).max() <= 1e-13 * np.abs(u).max()
    b = u.copy()
    nf, _ = O.mn_run(T, G, b, alpha.copy(), sa, ss, q, dt, 3)
    assert nf == 0
    assert np.abs(b - u).max() > 1e-3 * np.abs(u).max()


@pytest.mark.parametrize("bc", [0, 1])
def test_discrete_conservation_identity_with_density(bc):
    """Interior faces still cancel pairwise (both cells use psi_up / rho_up), so with sigma_a = 0
    and no source sum_i A_i u_i0 changes only by the boundary flux of psi / rho."""
    T = O.Tables(2, 6)
    G = _mesh(seed=8, k=10)
    rho = _density(G)
    psi = _state(T, G, 9)
    u = psi @ (T.w[:, None] * T.M)
    dt = 0.4 * G.cfl_dt(1.0) * rho.min()
    before = float((G.area * u[:, 0]).sum())
    bflux = 0.0
    for c in range(G.C):
        for k in range(3):
            if G.nbr[c, k] >= 0:
                continue
            d = T.ox * G.nrm[c, k, 0] + T.oy * G.nrm[c, k, 1]
            ghost = psi[c] / rho[c] if bc == 0 else np.zeros(T.Q)
            up = np.where(d > 0, psi[c] / rho[c], ghost)
            bflux += float(np.sum(T.w * T.M[:, 0] * d * up))
    uu = u.copy()
    O.flux_update_rho(T, G, rho, psi, uu, np.zeros(G.C), np.ones(G.C), np.zeros(G.C), dt, bc=bc)
    after = float((G.area * uu[:, 0]).sum())
    assert abs(bflux) > 1e-6 * abs(before)
    assert abs(after - (before - dt * bflux)) <= 1e-12 * abs(before)


def test_dose_of_uniform_fluence_does_not_depend_on_density():
    """Water-equivalent tissue (S = S_w rho): a uniform physical fluence psi deposits the same dose
    in every density. In the transformed variables psi~ = S_w rho psi, so the state u_0 = <m_0
    psi~> scales with rho while the dose increment dt S_w(t) Phi~ / rho does not. A pseudo-time
    step dt spans dE = S_w dt of energy, so over steps with stopping powers S_n the dose is
    dt sum_n S_n^2 4 pi psi."""
    T = O.Tables(2, 6)
    C = 7
    rho = np.array([0.2, 0.5, 1.0, 1.0, 2.0, 5.0, 11.0])
    psi = 0.13
    S = [2.0, 1.5, 0.7]
    dt = 0.05
    dose = np.zeros(C)
    for Sn in S:
        u = np.zeros((C, T.n))
        u[:, 0] = Sn * rho * psi * 4 * math.pi * T.m0     # u_0 of psi~ = S_w rho psi, isotropic
        O.dose_accumulate(T, u, rho, Sn, dt, dose)
    # straight from the dose definition: D = 1/rho int S_w rho psi 4 pi dE, and a pseudo-time
    # step dt spans dE = S_w dt of energy
    expect = dt * sum(Sn * Sn for Sn in S) * psi * 4 * math.pi
    np.testing.assert_allclose(dose, expect, rtol=1e-14)


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("axis", [0, 1])
def test_density_step_commutes_with_mirroring_the_mesh(bc, axis):
    """The transformed CSD step (psi~ / rho transported, Sec. 2) on the mesh mirrored in x or y,
    with each cell keeping its density and moments carried to the mirrored directions, equals the
    mirrored step (3 steps, two tissues)."""
    from mirror_map import mirror_basis, mirror_points, mirror_xy
    N, order = 2, 10
    T = O.Tables(N, order)
    m = synth.jittered_mesh(10, -1.5, 1.5, seed=3)
    G, Gr = O.Geometry(m.xy, m.tri), O.Geometry(mirror_xy(m.xy, axis), m.tri)
    mu, phi, w, ox, oy = O.quadrature(order)
    D = mirror_basis(T.M, mirror_points(ox, oy, mu, axis))
    rho = synth.two_tissue_density(G.cen)
    c, k, wt = synth.vmf_mixtures(G.C, 21)
    u = (synth.vmf_density(np.stack([ox, oy, mu], axis=1), c, k, wt) @ (T.w[:, None] * T.M)) * rho[:, None]
    rng = np.random.default_rng(21)
    sa, ss, q = rng.uniform(0, 1, G.C), rng.uniform(0, 2, G.C), rng.uniform(0, 0.5, G.C)
    dt = 0.4 * G.cfl_dt(1.0) * rho.min()
    u1 = u.copy()
    a1 = O.isotropic_alpha(T, u1)
    assert O.mn_run_rho(T, G, rho, u1, a1, sa, ss, q, dt, 3, bc=bc)[0] == 0
    ur = u @ D.T
    ar = O.isotropic_alpha(T, ur)
    assert O.mn_run_rho(T, Gr, rho, ur, ar, sa, ss, q, dt, 3, bc=bc)[0] == 0
    err = np.linalg.norm(ur - u1 @ D.T) / np.linalg.norm(u1)
    print("density mirror diff", err)
    assert err <= 1e-12
