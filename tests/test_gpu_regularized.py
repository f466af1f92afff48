"""GPU parity of the (partially) regularized closure (Sec. 3.1, Eq. entropyOCP_reg and
Eq. entropyOCP_part_reg; dual + gamma/2 |alpha^r|^2) against the oracle, through the C ABI:
closures of von Mises-Fisher moments (alpha within the conditioning bound of the closure
parity tests), a regularized M_3 step on the block medium (1e-11 relative L2 on u, FP64), the
mixed modes (1e-5 on u_0), and moments outside the realizable set, which the regularized
closure solves and the entropy closure cannot."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_08417_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GAMMA = 1e-3  # the paper's regularized M_3 run


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


def _vmf_u(T, count, seed, kappa_hi=20.0):
    mu, phi, w, ox, oy = O.quadrature(T.order)
    c, k, wt = synth.vmf_mixtures(count, seed, kappa_hi=kappa_hi)
    psi = synth.vmf_density(np.stack([ox, oy, mu], axis=1), c, k, wt)
    scale = np.exp(np.random.default_rng(seed).uniform(-3, 2, size=count))
    return (psi * scale[:, None]) @ (T.w[:, None] * T.M)


@pytest.mark.parametrize("keep_mass", [1, 0])
@pytest.mark.parametrize("N,order", [(2, 10), (3, 20)])
def test_regularized_closure_matches_oracle(K, N, order, keep_mass):
    T = O.Tables(N, order)
    m = synth.jittered_mesh(16, 0.0, 1.0, seed=4)
    mesh = K.Mesh(m.xy, m.tri)
    C = mesh.ncells
    u = _vmf_u(T, C, seed=60 + N)
    reg0 = 1 if keep_mass else 0
    a_or = O.isotropic_alpha(T, u)
    st_or, _ = O.closure_reg(T, u, a_or, GAMMA, reg0)
    assert (st_or == 0).all()
    s = K.MNSolver(mesh, N, order, reg_gamma=GAMMA, reg_keep_mass=keep_mass)
    ud = dev(u)
    ad = s.isotropic_alpha(ud)
    st = torch.zeros(C, dtype=torch.int32, device="cuda")
    s.closure(ud, ad, st)
    assert (st.cpu().numpy() == 0).all()
    a_gpu = ad.cpu().numpy()
    for i in range(C):
        e = T.w * np.exp(T.M @ a_or[i])
        H = T.M.T @ (e[:, None] * T.M)
        H[np.arange(reg0, T.n), np.arange(reg0, T.n)] += GAMMA
        lmin = np.linalg.eigvalsh(H)[0]
        bound = 1e-9 * np.linalg.norm(u[i]) / lmin + 1e-12 * np.linalg.norm(a_or[i])
        assert np.linalg.norm(a_gpu[i] - a_or[i]) <= bound, i
        # the regularized ansatz: u_0 exact when kept, the other moments short by gamma alpha
        mom = T.M.T @ (T.w * np.exp(T.M @ a_gpu[i]))
        shift = GAMMA * a_gpu[i]
        if keep_mass:
            shift[0] = 0.0
        assert np.linalg.norm(mom - (u[i] - shift)) <= 2e-10 * np.linalg.norm(u[i])


def _blocks(N, order, k=24):
    m = synth.jittered_mesh(k, 0.0, 7.0, seed=3)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(N, order)
    blk, sab, ssb = synth.block_coefficients(G.cen, 0.0, 7.0, 7, seed=3)
    sa, ss = sab[blk], ssb[blk]
    q = np.where(blk == 24, 1.0, 0.0)
    u0 = np.zeros((G.C, T.n))
    u0[:, 0] = 1e-4 / math.sqrt(4 * math.pi)
    return m, G, T, sa, ss, q, u0


@pytest.mark.parametrize("bc", ["vacuum", "neumann"])
def test_regularized_step_matches_oracle(K, bc):
    """Regularized M_3 (gamma = 1e-3, u_0 kept) on the block medium with a unit source, 10 FP64
    steps: 1e-11 relative L2 on u."""
    N, order = 3, 10
    m, G, T, sa, ss, q, u0 = _blocks(N, order)
    dt = G.cfl_dt(0.4)
    bci = 1 if bc == "vacuum" else 0
    u_or = u0.copy()
    a_or = O.isotropic_alpha(T, u_or)
    nf, _ = O.mn_run_reg(T, G, u_or, a_or, sa, ss, q, dt, 10, GAMMA, 1, bc=bci)
    assert nf == 0
    mesh = K.Mesh(m.xy, m.tri)
    s = K.MNSolver(mesh, N, order, bc=bc, reg_gamma=GAMMA)
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=10)
    err = rel_l2(ud.cpu().numpy(), u_or)
    print("regularized M_3 blocks", bc, "rel L2", err)
    assert err <= 1e-11


@pytest.mark.parametrize("mode", ["mixed_tf32", "mixed_bf16"])
def test_regularized_mixed_step_matches_oracle(K, mode):
    N, order = 3, 10
    m, G, T, sa, ss, q, u0 = _blocks(N, order)
    dt = G.cfl_dt(0.4)
    u_or = u0.copy()
    a_or = O.isotropic_alpha(T, u_or)
    assert O.mn_run_reg(T, G, u_or, a_or, sa, ss, q, dt, 20, GAMMA, 1, bc=1)[0] == 0
    mesh = K.Mesh(m.xy, m.tri)
    s = K.MNSolver(mesh, N, order, bc="vacuum", mode=mode, tau=1e-8, reg_gamma=GAMMA)
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=20)
    err0 = rel_l2(ud.cpu().numpy()[:, 0], u_or[:, 0])
    print(mode, "regularized u0 rel L2", err0)
    assert err0 <= 1e-5


def test_regularized_closure_solves_non_realizable_moments(K):
    """|u_1| too large for u_0: the entropy closure reports a failure, the partially regularized
    one converges and keeps u_0."""
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    mesh = K.Mesh(xy, tri)
    T = O.Tables(1, 10)
    u = np.array([[1.0, 5.0, 0.0], [1.0, 0.0, -4.0]])
    plain = K.MNSolver(mesh, 1, 10)
    ud = dev(u)
    a = plain.isotropic_alpha(ud)
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    rc = plain.closure(ud, a, st, check=False)
    assert rc != 0 and (st.cpu().numpy() != 0).all()
    reg = K.MNSolver(mesh, 1, 10, reg_gamma=GAMMA, tau=1e-12)
    a = reg.isotropic_alpha(ud)
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    reg.closure(ud, a, st)
    assert (st.cpu().numpy() == 0).all()
    a_or = O.isotropic_alpha(T, u)
    assert (O.closure_reg(T, u, a_or, GAMMA, 1, tau=1e-12)[0] == 0).all()
    np.testing.assert_allclose(a.cpu().numpy(), a_or, rtol=1e-9, atol=1e-9)
    mom = np.exp(a.cpu().numpy() @ T.M.T) @ (T.w[:, None] * T.M)
    np.testing.assert_allclose(mom[:, 0], u[:, 0], rtol=1e-11)
