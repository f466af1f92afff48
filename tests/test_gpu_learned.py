"""Learned closure on the GPU: the MLP kernels against the oracle's FP64 MLP (forward, loss,
gradient, Adam), the von Mises-Fisher moment generator against the oracle's quadrature, the
learned M_N step against the FP64 oracle (1e-5 relative L2 on u_0), and what the trained network
gains over the same closure without it (quadrature passes of cold closures)."""
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


def _mlp_case(seed, din, H, dout, B):
    rng = np.random.default_rng(seed)
    P = O.mlp_param_count(din, H, dout)
    p = rng.normal(scale=0.3, size=P)
    X = rng.normal(size=(B, din))
    T = rng.normal(size=(B, dout))
    return p, X, T


def test_mlp_forward_and_gradient_match_oracle(K):
    din, H, dout, B = 9, 64, 9, 300   # ragged batch (not a multiple of the 64-row tile)
    p, X, T = _mlp_case(0, din, H, dout, B)
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    # compare against the oracle on the FP32-rounded inputs
    p32, X32, T32 = [a.astype(np.float32).astype(np.float64) for a in (p, X, T)]
    Y = K.mlp_forward(f32(p), f32(X), din, H, dout).cpu().numpy()
    Yo = O.mlp_forward(p32, X32, din, H, dout)
    assert np.linalg.norm(Y - Yo) / np.linalg.norm(Yo) < 1e-5
    loss, g = K.mlp_loss_grad(f32(p), f32(X), f32(T), din, H, dout)
    lo, go = O.mlp_loss_grad(p32, X32, T32, din, H, dout)
    assert abs(float(loss.cpu()[0]) - lo) / lo < 1e-5
    g = g.cpu().numpy()
    assert np.linalg.norm(g - go) / np.linalg.norm(go) < 1e-5


def test_mlp_adam_matches_oracle(K):
    rng = np.random.default_rng(1)
    P = 1000
    p, m, v = rng.normal(size=P), np.zeros(P), np.zeros(P)
    pd = torch.from_numpy(p.astype(np.float32)).cuda()
    md, vd = torch.zeros_like(pd), torch.zeros_like(pd)
    po = p.astype(np.float32).astype(np.float64)
    for t in range(1, 6):
        g = rng.normal(size=P)
        K.mlp_adam(pd, torch.from_numpy(g.astype(np.float32)).cuda(), md, vd, t, lr=1e-2)
        O.adam(po, g.astype(np.float32).astype(np.float64), m, v, t, lr=1e-2)
    assert np.abs(pd.cpu().numpy() - po).max() < 1e-5


def test_vmf_moments_match_oracle_quadrature(K):
    N, order = 3, 20
    m = synth.jittered_mesh(6, 0.0, 1.0, seed=0)
    mesh = K.Mesh(m.xy, m.tri)
    s = K.MNSolver(mesh, N, order)
    count = 77
    c, kap, wt = synth.vmf_mixtures(count, seed=5)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    u = s.vmf_moments(dev(c), dev(kap), dev(wt)).cpu().numpy()
    T = O.Tables(N, order)
    mu, phi, w, ox, oy = O.quadrature(order)
    psi = synth.vmf_density(np.stack([ox, oy, mu], axis=1), c, kap, wt)
    u_or = psi @ (T.w[:, None] * T.M)
    assert np.abs(u - u_or).max() <= 1e-12 * np.abs(u_or).max()
    # a normalised density has zeroth moment m_0 = 1/sqrt(4 pi) up to quadrature error
    assert np.abs(u[:, 0] * math.sqrt(4 * math.pi) - 1).max() < 1e-3


@pytest.fixture(scope="module")
def trained_m2(K):
    from paper_2205_08417_gb300 import learned
    m = synth.jittered_mesh(100, 0.0, 1.0, seed=9)
    mesh = K.Mesh(m.xy, m.tri)
    s = K.MNSolver(mesh, 2, 10, mode="fp64", tau=1e-12)
    u, a = learned.training_data(s, 200_000, seed=4)
    net = learned.train(u, a, epochs=30, batch=1024, lr=3e-3)
    assert net.losses[-1] < 0.2 * net.losses[0]
    return net


def test_learned_line_source_matches_oracle(K, trained_m2):
    """M_2 line source (3872 triangles, order 10), 50 learned steps: network + exact mass + FP64
    residual test (fallback to Newton above 1e-6) against the FP64 Newton oracle on u_0."""
    m = synth.jittered_mesh(45, -1.5, 1.5, seed=1)
    mesh = K.Mesh(m.xy, m.tri)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(2, 10)
    u0 = synth.isotropic_moments(synth.line_source_density(G.cen), T.n)
    C = G.C
    dt = G.cfl_dt(0.4)
    sa, ss, q = np.zeros(C), np.ones(C), np.zeros(C)
    u_or = u0.copy()
    a_or = O.isotropic_alpha(T, u_or)
    assert O.mn_run(T, G, u_or, a_or, sa, ss, q, dt, 50)[0] == 0
    s = K.MNSolver(mesh, 2, 10, mode="learned", tau=1e-8, fallback_tol=1e-6)
    s.set_mlp(trained_m2.params, trained_m2.norm)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    rc, st = s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=50, stats=True)
    u_gpu = ud.cpu().numpy()
    err0 = float(np.linalg.norm(u_gpu[:, 0] - u_or[:, 0]) / np.linalg.norm(u_or[:, 0]))
    print("learned u0 rel L2", err0, "stats", st)
    assert err0 <= 1e-5
    # rejected proposals whose previous point was better stepped from the stored factor
    assert st["restarts"] > 0
    # the FP32 flux conserves total mass to FP32 rounding of the exchanged fluxes
    assert abs((G.area * u_gpu[:, 0]).sum() / (G.area * u0[:, 0]).sum() - 1) < 1e-7


def test_network_reduces_quadrature_passes_of_cold_closures(K, trained_m2):
    """What the trained network gains: closures of fresh moments (no warm start). Baseline: the
    same solver arithmetic started from the isotropic closed form. Counted: quadrature passes per
    cell (the learned mode counts its network residual pass too)."""
    m = synth.jittered_mesh(60, 0.0, 1.0, seed=10)
    mesh = K.Mesh(m.xy, m.tri)
    C = mesh.ncells
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    base = K.MNSolver(mesh, 2, 10, mode="mixed_tf32", tau=1e-8)
    lrn = K.MNSolver(mesh, 2, 10, mode="learned", tau=1e-8, fallback_tol=1e-6)
    lrn.set_mlp(trained_m2.params, trained_m2.norm)
    c, kap, wt = synth.vmf_mixtures(C, seed=77)
    u = base.vmf_moments(dev(c), dev(kap), dev(wt))
    a1 = base.isotropic_alpha(u)
    s1 = torch.zeros(C, dtype=torch.int32, device="cuda")
    _, st1 = base.closure(u, a1, s1, stats=True, check=False)
    a2 = lrn.isotropic_alpha(u)
    s2 = torch.zeros(C, dtype=torch.int32, device="cuda")
    _, st2 = lrn.closure(u, a2, s2, stats=True, check=False)
    ok = ((s1 == 0) & (s2 == 0)).cpu().numpy()
    assert ok.mean() > 0.95
    print("cold closures: passes/cell without network", st1["evaluations"] / C,
          "with network", st2["evaluations"] / C, "fallbacks", st2["fallbacks"] / C)
    assert st2["evaluations"] < 0.95 * st1["evaluations"]
    # both answers solve the same closure
    A1, A2 = a1.cpu().numpy()[ok], a2.cpu().numpy()[ok]
    T = O.Tables(2, 10)
    for A in (A1, A2):
        rec = np.exp(A @ T.M.T) @ (T.w[:, None] * T.M)
        uu = u.cpu().numpy()[ok]
        assert (np.linalg.norm(rec - uu, axis=1) / np.linalg.norm(uu, axis=1)).max() < 2e-6
