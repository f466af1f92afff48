"""Pins for the oracle's S_N step (Sec. 2, Eq. SNEqns2: nodal transport with the P_N form
O Sigma M of the scattering operator; Sec. 4.2/4.4: explicit upwind step per ordinate). Checked
against: the oracle's M_N flux update (itself pinned by a hand-written step), which the moments of
an S_N step must reproduce; the addition theorem of spherical harmonics, which turns O Sigma M into
a direct sum over the scattering kernel's Legendre series; closed-form uniform states; and
equivariance under mirroring the mesh (3e-16)."""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre

import oracle as O
from paper_2205_08417_gb300 import synth


def _setup(k=7, N=3, order=6, seed=2):
    T = O.Tables(N, order)
    m = synth.jittered_mesh(k, -1.0, 1.0, seed=seed)
    G = O.Geometry(m.xy, m.tri)
    return T, G


def _ordinates(T, G, seed):
    """Positive ordinates that depend on the direction only through (Omega_x, Omega_y), so that
    they are even in mu like every state of the 2D slab problem."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.5, 2.0, size=G.C)
    b = rng.normal(size=(G.C, 2))
    c = rng.normal(size=(G.C, 3))
    ox, oy = T.ox[None, :], T.oy[None, :]
    return a[:, None] * np.exp(0.6 * (b[:, :1] * ox + b[:, 1:] * oy)
                               + 0.3 * (c[:, :1] * ox * ox + c[:, 1:2] * ox * oy + c[:, 2:] * oy * oy))


@pytest.mark.parametrize("bc", [0, 1])
def test_moments_of_sn_step_equal_mn_update_of_the_same_psi(bc):
    """With isotropic scattering, M psi' of one S_N step equals the M_N update of u = M psi driven
    by the same ordinates (the moment equations are the projection of the nodal ones)."""
    T, G = _setup()
    psi = _ordinates(T, G, 3)
    rng = np.random.default_rng(4)
    sa, ss, q = rng.uniform(0, 2, G.C), rng.uniform(0, 1, G.C), rng.uniform(0, 1, G.C)
    dt = G.cfl_dt(0.4)
    out = O.sn_step(T, G, psi, sa, ss, q, dt, bc=bc)
    u = psi @ (T.w[:, None] * T.M)
    O.flux_update(T, G, psi, u, sa, ss, q, dt, bc=bc)
    mom = out @ (T.w[:, None] * T.M)
    assert np.abs(mom - u).max() <= 1e-13 * np.abs(u).max()


def test_scattering_matches_addition_theorem_kernel_sum():
    """No transport (one isolated cell is not possible, so dt/A-scaled transport is removed by
    differencing two steps that differ only in sigma_s): the change of psi' per unit sigma_s is
    dt [(O G M psi)_q - psi_q], and by the addition theorem
    (O G M psi)_q = sum_p w_p psi_p sum_l g_l (2l+1)/(4 pi) P_l(Omega_q . Omega_p)
    for ordinates even in mu."""
    T, G = _setup(k=5, N=3, order=8)
    psi = _ordinates(T, G, 7)
    g = np.array([1.0, 0.7, 0.45, 0.2])
    z = np.zeros(G.C)
    dt = G.cfl_dt(0.4)
    s1 = np.full(G.C, 0.8)
    d = (O.sn_step(T, G, psi, z, s1, z, dt, g=g) - O.sn_step(T, G, psi, z, z, z, dt, g=g)) / (0.8 * dt)
    mu, phi, w, ox, oy = O.quadrature(T.order)
    dirs = np.stack([ox, oy, mu], axis=1)
    cosang = np.clip(dirs @ dirs.T, -1.0, 1.0)
    kern = sum(g[l] * (2 * l + 1) / (4 * math.pi) * eval_legendre(l, cosang) for l in range(len(g)))
    expect = psi @ (w[:, None] * kern.T) - psi
    assert np.abs(d - expect).max() <= 1e-11 * np.abs(psi).max()


def test_anisotropic_scattering_moments_scale_by_degree():
    """M (O Sigma M psi) = Sigma M psi on the quadrature: moment a of psi' changes by
    dt sigma_s (g_l(a) - delta_{l(a),0}) u_a relative to isotropic scattering."""
    T, G = _setup(N=3, order=6)
    psi = _ordinates(T, G, 11)
    g = np.array([1.0, 0.5, 0.25, 0.125])
    z = np.zeros(G.C)
    ss = np.linspace(0.1, 1.0, G.C)
    dt = G.cfl_dt(0.4)
    diff = O.sn_step(T, G, psi, z, ss, z, dt, g=g) - O.sn_step(T, G, psi, z, ss, z, dt)
    u = psi @ (T.w[:, None] * T.M)
    deg = np.concatenate([[l] * sum(1 for k in range(-l, l + 1) if (l + abs(k)) % 2 == 0)
                          for l in range(T.N + 1)])
    gl = g[deg] - (deg == 0)
    expect = dt * ss[:, None] * gl[None, :] * u
    got = diff @ (T.w[:, None] * T.M)
    assert np.abs(got - expect).max() <= 1e-13 * np.abs(u).max()


def test_uniform_isotropic_state_is_steady_and_absorbs_in_closed_form():
    T, G = _setup(k=9, N=2, order=5)
    psi = np.full((G.C, T.Q), 0.37)
    z = np.zeros(G.C)
    dt = G.cfl_dt(0.4)
    # Neumann walls, scattering only: a fixed point
    out = O.sn_step(T, G, psi, z, np.full(G.C, 0.9), z, dt, bc=0)
    assert np.abs(out - psi).max() <= 1e-14 * 0.37 * 10
    # absorption only: psi' = (1 - dt sigma_a) psi
    sa = np.linspace(0.0, 3.0, G.C)
    out = O.sn_step(T, G, psi, sa, z, z, dt, bc=0)
    np.testing.assert_allclose(out, (1 - dt * sa)[:, None] * psi, rtol=1e-13, atol=0)


def test_sn_run_conserves_mass_up_to_boundary_outflow():
    """Exact discrete identity with sigma_a = 0, no source, vacuum walls:
    sum_i A_i phi_i' = sum_i A_i phi_i - dt (outflow through boundary faces), phi = sum_q w psi."""
    T, G = _setup(k=8, N=2, order=5)
    psi = _ordinates(T, G, 5)
    z = np.zeros(G.C)
    dt = G.cfl_dt(0.4)
    out = O.sn_step(T, G, psi, z, np.full(G.C, 0.5), z, dt, bc=1)
    outflow = 0.0
    for c in range(G.C):
        for k in range(3):
            if G.nbr[c, k] >= 0:
                continue
            d = T.ox * G.nrm[c, k, 0] + T.oy * G.nrm[c, k, 1]
            outflow += float(np.sum(T.w * np.where(d > 0, d * psi[c], 0.0)))
    before = float(G.area @ (psi @ T.w))
    after = float(G.area @ (out @ T.w))
    assert outflow > 1e-3 * before
    assert abs(after - (before - dt * outflow)) <= 1e-13 * before
    # sn_run agrees with repeated steps
    p2 = psi.copy()
    O.sn_run(T, G, p2, z, np.full(G.C, 0.5), z, dt, 2, bc=1)
    ref = O.sn_step(T, G, out, z, np.full(G.C, 0.5), z, dt, bc=1)
    np.testing.assert_array_equal(p2, ref)


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("axis", [0, 1])
def test_sn_step_commutes_with_mirroring_the_mesh(bc, axis):
    """The S_N step (Eq. SNEqns2, Sec. 4.4 upwind flux per ordinate) on the mesh mirrored in x or y,
    from the ordinates carried to the mirrored directions, equals the mirrored step, with
    anisotropic scattering; pins the per-ordinate upwind choice for clockwise triangles."""
    from mirror_map import mirror_points, mirror_xy
    N, order = 3, 8
    T = O.Tables(N, order)
    m = synth.jittered_mesh(9, -1.0, 1.0, seed=2)
    G, Gr = O.Geometry(m.xy, m.tri), O.Geometry(mirror_xy(m.xy, axis), m.tri)
    mu, phi, w, ox, oy = O.quadrature(order)
    perm = mirror_points(ox, oy, mu, axis)
    rng = np.random.default_rng(4)
    psi = rng.uniform(0.1, 2.0, size=(G.C, T.Q))
    sa, ss, q = rng.uniform(0, 1, G.C), rng.uniform(0, 2, G.C), rng.uniform(0, 0.5, G.C)
    g = [1.0, 0.6, 0.3, 0.1]
    dt = G.cfl_dt(0.4)
    a = O.sn_run(T, G, psi.copy(), sa, ss, q, dt, 3, g=g, bc=bc)
    b = O.sn_run(T, Gr, psi[:, perm].copy(), sa, ss, q, dt, 3, g=g, bc=bc)
    print("S_N mirror diff", np.abs(b - a[:, perm]).max() / np.abs(a).max())
    assert np.abs(b - a[:, perm]).max() <= 1e-14 * np.abs(a).max()
