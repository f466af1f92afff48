"""GPU parity of the transformed CSD equation's step (Sec. 2, Eq. BoltzmannCSDTrafo: the flux
transports psi / rho) and dose (Sec. 2), and of the checkerboard (Sec. 7.2) in the paper's
configuration (second-order flux, Heun, CFL 0.45), against the oracle through the C ABI.

Bars: FP64 1e-11 relative L2 on u (the FP64 bar of the step); mixed modes 1e-5 relative L2 on
u_0; dose 1e-13 relative."""
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


def _csd_case(k=45, N=2, order=10):
    """Line-source start in a two-tissue medium: psi~ = rho psi with the paper's Gaussian, so the
    moments of the transformed state scale with the density."""
    m = synth.jittered_mesh(k, -1.5, 1.5, seed=1)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(N, order)
    rho = synth.two_tissue_density(G.cen)
    u0 = synth.isotropic_moments(synth.line_source_density(G.cen, width=0.1), T.n) * rho[:, None]
    dt = 0.4 * G.cfl_dt(1.0) * rho.min()
    return m, G, T, rho, u0, dt


@pytest.mark.parametrize("bc", ["neumann", "vacuum"])
def test_csd_step_fp64_matches_oracle(K, bc):
    m, G, T, rho, u0, dt = _csd_case()
    C = G.C
    sa, ss, q = np.full(C, 0.2), np.full(C, 0.8), np.zeros(C)
    u_or = u0.copy()
    a_or = O.isotropic_alpha(T, u_or)
    nf, _ = O.mn_run_rho(T, G, rho, u_or, a_or, sa, ss, q, dt, 20, bc=1 if bc == "vacuum" else 0)
    assert nf == 0
    s = K.MNSolver(K.Mesh(m.xy, m.tri), T.N, 10, bc=bc)
    s.set_density(dev(rho))
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=20)
    err = rel_l2(ud.cpu().numpy(), u_or)
    print("CSD step FP64", bc, "rel L2", err)
    assert err <= 1e-11
    # the density changed the answer: the plain step from the same start differs
    s2 = K.MNSolver(K.Mesh(m.xy, m.tri), T.N, 10, bc=bc)
    u2 = dev(u0)
    s2.step(u2, s2.isotropic_alpha(u2), dev(sa), dev(ss), dev(q), dt=dt, nsteps=20)
    assert rel_l2(u2.cpu().numpy(), u_or) > 1e-3


@pytest.mark.parametrize("mode", ["mixed_tf32", "mixed_bf16"])
def test_csd_step_mixed_matches_oracle(K, mode):
    m, G, T, rho, u0, dt = _csd_case()
    C = G.C
    sa, ss, q = np.zeros(C), np.ones(C), np.zeros(C)
    u_or = u0.copy()
    a_or = O.isotropic_alpha(T, u_or)
    assert O.mn_run_rho(T, G, rho, u_or, a_or, sa, ss, q, dt, 20)[0] == 0
    s = K.MNSolver(K.Mesh(m.xy, m.tri), T.N, 10, mode=mode, tau=1e-8)
    s.set_density(dev(rho))
    ud = dev(u0)
    s.step(ud, s.isotropic_alpha(ud), dev(sa), dev(ss), dev(q), dt=dt, nsteps=20)
    err0 = rel_l2(ud.cpu().numpy()[:, 0], u_or[:, 0])
    print("CSD step", mode, "u0 rel L2", err0)
    assert err0 <= 1e-5


def test_csd_psi_proportional_to_density_is_steady_on_gpu(K):
    """psi~ / rho uniform (isotropic), Neumann, no absorption or source: a fixed point."""
    m, G, T, rho, _, dt = _csd_case(k=30)
    u = np.zeros((G.C, T.n))
    u[:, 0] = 0.3 * rho * 4 * math.pi * T.m0
    for mode in ("fp64", "mixed_tf32"):
        s = K.MNSolver(K.Mesh(m.xy, m.tri), T.N, 10, mode=mode, tau=1e-8 if mode != "fp64" else 1e-10)
        s.set_density(dev(rho))
        ud = dev(u)
        s.step(ud, s.isotropic_alpha(ud), dev(np.zeros(G.C)), dev(np.ones(G.C)),
               dev(np.zeros(G.C)), dt=dt, nsteps=5)
        err = np.abs(ud.cpu().numpy() - u).max() / np.abs(u).max()
        print("steady psi ~ rho,", mode, err)
        assert err <= (1e-13 if mode == "fp64" else 1e-6)


def test_dose_matches_oracle(K):
    m, G, T, rho, u0, dt = _csd_case(k=20)
    s = K.MNSolver(K.Mesh(m.xy, m.tri), T.N, 10)
    s.set_density(dev(rho))
    dose_or = np.zeros(G.C)
    dose = dev(np.zeros(G.C))
    for S in (2.0, 1.3, 0.6):
        O.dose_accumulate(T, u0, rho, S, dt, dose_or)
        s.dose_accumulate(dev(u0), S, dt, dose)
    assert rel_l2(dose.cpu().numpy(), dose_or) <= 1e-13


def test_density_validation(K):
    m, G, T, rho, u0, dt = _csd_case(k=16)
    C = G.C
    mesh = K.Mesh(m.xy, m.tri)
    s = K.MNSolver(mesh, T.N, 10)
    bad = rho.copy()
    bad[3] = 0.0
    with pytest.raises(RuntimeError):
        s.set_density(dev(bad))
    bad[3] = float("nan")
    with pytest.raises(RuntimeError):
        s.set_density(dev(bad))
    # a thin medium (rho = 0.1) speeds transport up 10x: the same dt breaks the step condition
    s.set_density(dev(np.full(C, 0.1)))
    ud = dev(u0)
    rc = s.step(ud, s.isotropic_alpha(ud), dev(np.zeros(C)), dev(np.ones(C)), dev(np.zeros(C)),
                dt=dt, check=False)
    assert rc != 0
    np.testing.assert_array_equal(ud.cpu().numpy(), u0)      # u untouched
    # removing the density gives back the plain step bit for bit
    s.set_density(None)
    plain = K.MNSolver(mesh, T.N, 10)
    a, b = dev(u0), dev(u0)
    s.step(a, s.isotropic_alpha(a), dev(np.zeros(C)), dev(np.ones(C)), dev(np.zeros(C)), dt=dt, nsteps=3)
    plain.step(b, plain.isotropic_alpha(b), dev(np.zeros(C)), dev(np.ones(C)), dev(np.zeros(C)),
               dt=dt, nsteps=3)
    assert torch.equal(a, b)
    # order 2, the adjoint and the S_N step do not take a density
    s2 = K.MNSolver(mesh, T.N, 10, order=2)
    s2.set_density(dev(rho))
    ud = dev(u0)
    assert s2.step(ud, s2.isotropic_alpha(ud), dev(np.zeros(C)), dev(np.ones(C)), dev(np.zeros(C)),
                   dt=dt, check=False) != 0


def _checkerboard(K, k, N, order):
    m = synth.jittered_mesh(k, 0.0, 7.0, seed=6)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(N, order)
    sa, ss, q = synth.checkerboard_medium(G.cen)
    u0 = np.zeros((G.C, T.n))
    u0[:, 0] = 1e-4 / math.sqrt(4 * math.pi)   # psi = 1e-4 / (4 pi) floor: the closure needs u_0 > 0
    return m, G, T, sa, ss, q, u0


def test_checkerboard_layout():
    """The reading of the lost layout figure: 11 absorbers in a checkerboard around the centre
    source, the block above the source open."""
    A = set(synth.CHECKERBOARD_ABSORBERS)
    assert len(A) == 11 and (3, 3) not in A and (3, 5) not in A
    assert {(3, 1), (1, 3), (5, 3), (2, 2), (4, 4)} <= A
    cen = np.array([[3.5, 3.5], [3.5, 1.5], [3.5, 5.5], [0.5, 0.5], [2.5, 2.5]])
    sa, ss, q = synth.checkerboard_medium(cen)
    np.testing.assert_array_equal(sa, [0, 10, 0, 0, 10])
    np.testing.assert_array_equal(ss, [1, 0, 1, 1, 0])
    np.testing.assert_array_equal(q, [1, 0, 0, 0, 0])


def test_checkerboard_second_order_fp64_matches_oracle(K):
    """The checkerboard as the paper runs it (second-order flux, Heun, CFL 0.45, vacuum), M_3,
    order 10, on a 2,450-triangle mesh, 12 steps: 1e-11 relative L2 on u."""
    m, G, T, sa, ss, q, u0 = _checkerboard(K, 36, 3, 10)
    dt = G.cfl_dt(0.45)
    u_or = u0.copy()
    a_or = O.isotropic_alpha(T, u_or)
    assert O.mn_run2(T, G, u_or, a_or, sa, ss, q, dt, 12, bc=1)[0] == 0
    s = K.MNSolver(K.Mesh(m.xy, m.tri), 3, 10, bc="vacuum", order=2)
    ud = dev(u0)
    s.step(ud, s.isotropic_alpha(ud), dev(sa), dev(ss), dev(q), dt=dt, nsteps=12)
    err = rel_l2(ud.cpu().numpy(), u_or)
    print("checkerboard M_3 second order FP64, 12 steps: rel L2", err)
    assert err <= 1e-11


def test_checkerboard_second_order_mixed_matches_oracle(K):
    m, G, T, sa, ss, q, u0 = _checkerboard(K, 36, 3, 10)
    dt = G.cfl_dt(0.45)
    u_or = u0.copy()
    a_or = O.isotropic_alpha(T, u_or)
    assert O.mn_run2(T, G, u_or, a_or, sa, ss, q, dt, 12, bc=1)[0] == 0
    s = K.MNSolver(K.Mesh(m.xy, m.tri), 3, 10, bc="vacuum", order=2, mode="mixed_tf32", tau=1e-8)
    ud = dev(u0)
    s.step(ud, s.isotropic_alpha(ud), dev(sa), dev(ss), dev(q), dt=dt, nsteps=12)
    err0 = rel_l2(ud.cpu().numpy()[:, 0], u_or[:, 0])
    print("checkerboard M_3 second order mixed TF32: u0 rel L2", err0)
    assert err0 <= 1e-5
