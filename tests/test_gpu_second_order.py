"""GPU parity of the second-order M_N step (Sec. 4.3: Green-Gauss gradient and Barth-Jespersen
limiter of the ansatz at every quadrature point, upwind flux of the reconstructed face values,
Heun time stepping) against the oracle's orc_mn_run2, through the C ABI.

Bars: FP64 1e-11 relative L2 on u (the FP64 bar of the first-order step); mixed modes 1e-5
relative L2 on u_0. Sizes span several tiles with a ragged tail; the two-triangle mesh is the
degenerate case (every face of one cell is a boundary face but one)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_08417_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_08417_gb300 import build, kitrt
    build.build()
    return kitrt


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _line_source(K, k, N, order, width=0.03):
    m = synth.jittered_mesh(k, -1.5, 1.5, seed=1)
    mesh = K.Mesh(m.xy, m.tri)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(N, order)
    u0 = synth.isotropic_moments(synth.line_source_density(G.cen, width=width), T.n)
    return m, mesh, G, T, u0


def test_second_order_line_source_m2_matches_oracle(K):
    """M_2 FP64 line source on the 3,872-triangle mesh, order-10 quadrature, CFL 0.4, 20 Heun
    steps (40 closures) against the oracle: 1e-11 relative L2 on u."""
    m, mesh, G, T, u0 = _line_source(K, 45, 2, 10)
    C = G.C
    dt = G.cfl_dt(0.4)
    sa, ss, q = np.zeros(C), np.ones(C), np.zeros(C)
    u_or = u0.copy()
    a_or = O.isotropic_alpha(T, u_or)
    nf, _ = O.mn_run2(T, G, u_or, a_or, sa, ss, q, dt, 20)
    assert nf == 0
    s = K.MNSolver(mesh, 2, 10, order=2)
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    rc, st = s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=20, stats=True)
    u_gpu = ud.cpu().numpy()
    err = rel_l2(u_gpu, u_or)
    print("second-order M_2 line source, 20 steps: rel L2", err, st)
    assert err <= 1e-11
    # two closures per step
    assert st["closures"] == 2 * 20 * C
    # mass conserved while the boundary holds the isotropic floor
    assert abs((G.area * u_gpu[:, 0]).sum() / (G.area * u0[:, 0]).sum() - 1) < 1e-12


@pytest.mark.parametrize("bc", ["neumann", "vacuum"])
def test_second_order_blocks_m3_matches_oracle(K, bc):
    """M_3, per-block sigma_a in [0,10], sigma_s in [0,1], unit source in the centre block,
    8 Heun steps, both boundary conditions: 1e-11 relative L2 on u."""
    N, order = 3, 10
    m = synth.jittered_mesh(24, 0.0, 7.0, seed=3)
    mesh = K.Mesh(m.xy, m.tri)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(N, order)
    blk, sab, ssb = synth.block_coefficients(G.cen, 0.0, 7.0, 7, seed=3)
    sa, ss = sab[blk], ssb[blk]
    q = np.where(blk == 24, 1.0, 0.0)
    u0 = np.zeros((G.C, T.n))
    u0[:, 0] = 1e-4 / math.sqrt(4 * math.pi)
    dt = G.cfl_dt(0.3)
    u_or = u0.copy()
    a_or = O.isotropic_alpha(T, u_or)
    nf, _ = O.mn_run2(T, G, u_or, a_or, sa, ss, q, dt, 8, bc=1 if bc == "vacuum" else 0)
    assert nf == 0
    s = K.MNSolver(mesh, N, order, bc=bc, order=2)
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=8)
    assert rel_l2(ud.cpu().numpy(), u_or) <= 1e-11


@pytest.mark.parametrize("mode", ["mixed_tf32", "mixed_bf16"])
def test_second_order_mixed_line_source_matches_oracle(K, mode):
    """The mixed modes (tensor-core Hessian, FP32 ansatz, reconstruction and flux) against the
    FP64 oracle: 1e-5 relative L2 on u_0 after 20 Heun steps."""
    m, mesh, G, T, u0 = _line_source(K, 45, 2, 10)
    C = G.C
    dt = G.cfl_dt(0.4)
    sa, ss, q = np.zeros(C), np.ones(C), np.zeros(C)
    u_or = u0.copy()
    a_or = O.isotropic_alpha(T, u_or)
    assert O.mn_run2(T, G, u_or, a_or, sa, ss, q, dt, 20)[0] == 0
    s = K.MNSolver(mesh, 2, 10, mode=mode, tau=1e-8, order=2)
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=20)
    u_gpu = ud.cpu().numpy()
    err0 = rel_l2(u_gpu[:, 0], u_or[:, 0])
    print(mode, "second-order u0 rel L2", err0)
    assert err0 <= 1e-5


def test_second_order_uniform_state_decays_by_the_heun_factor(K):
    """A uniform anisotropic state with Neumann walls has zero flux (zero gradients, exactly zero
    fluctuations), so each Heun step multiplies moment a by 1 - s dt + (s dt)^2/2, s = sigma_a
    (a = 0) or sigma_a + sigma_s."""
    m = synth.jittered_mesh(12, 0.0, 1.0, seed=2)
    mesh = K.Mesh(m.xy, m.tri)
    C = mesh.ncells
    T = O.Tables(2, 6)
    mu, phi, w, ox, oy = O.quadrature(6)
    c, kap, wt = synth.vmf_mixtures(1, 5, kappa_hi=3.0)
    u1 = synth.vmf_density(np.stack([ox, oy, mu], axis=1), c, kap, wt) @ (T.w[:, None] * T.M)
    u = np.repeat(u1, C, axis=0)
    s = K.MNSolver(mesh, 2, 6, order=2, tau=1e-13)
    ud = dev(u)
    ad = s.isotropic_alpha(ud)
    dt = 0.5 * mesh.geometry()["min_inradius"]
    sa, ss = 0.7, 0.4
    s.step(ud, ad, dev(np.full(C, sa)), dev(np.full(C, ss)), dev(np.zeros(C)), dt=dt, nsteps=3)
    rate = np.full(T.n, sa + ss)
    rate[0] = sa
    factor = (1 - rate * dt + (rate * dt) ** 2 / 2) ** 3
    np.testing.assert_allclose(ud.cpu().numpy(), u * factor[None, :], rtol=1e-12, atol=1e-16)


def test_second_order_two_triangle_mesh(K):
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    mesh = K.Mesh(xy, tri)
    G = O.Geometry(xy, tri)
    T = O.Tables(2, 4)
    u0 = np.zeros((2, T.n))
    u0[:, 0] = [1.0, 0.25]
    dt = G.cfl_dt(0.4)
    for bc, name in [(0, "neumann"), (1, "vacuum")]:
        u_or = u0.copy()
        a_or = O.isotropic_alpha(T, u_or)
        assert O.mn_run2(T, G, u_or, a_or, np.zeros(2), np.ones(2), np.zeros(2), dt, 3, bc=bc)[0] == 0
        s = K.MNSolver(mesh, 2, 4, bc=name, order=2)
        ud = dev(u0)
        ad = s.isotropic_alpha(ud)
        s.step(ud, ad, dev(np.zeros(2)), dev(np.ones(2)), dev(np.zeros(2)), dt=dt, nsteps=3)
        assert rel_l2(ud.cpu().numpy(), u_or) <= 1e-11, name
