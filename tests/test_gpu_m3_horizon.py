"""M_3 evidence on the line source (Sec. 7.1) at the benchmark's sizes and horizon:
- the learned closure at M_3 (the network trained as the benchmark trains it: 2M vMF samples
  closed by FP64 Newton, 20 epochs) stepping the line source against the FP64 oracle, bar 1e-5
  relative L2 on u_0, with its acceptance rate reported;
- the 99,458-triangle M_3 line source (order 20) run to t_final = 1.0 (about 1,790 steps) in every
  mode: FP64 (tau 1e-10 + polish), mixed TF32 and BF16 (tau 1e-8) and learned, each mode's u_0
  against the FP64 GPU run at t = 1 (bar 1e-5), and the FP64 GPU run held to the oracle at t = 1
  by recomputing one more step for sampled cells on the CPU (bar 1e-11)."""
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


@pytest.fixture(scope="module")
def trained_m3(K):
    from paper_2205_08417_gb300 import learned
    m = synth.jittered_mesh(100, 0.0, 1.0, seed=9)
    s = K.MNSolver(K.Mesh(m.xy, m.tri), 3, 20, mode="fp64", tau=1e-12)
    u, a = learned.training_data(s, 2_000_000, seed=4)
    net = learned.train(u, a, batch=4096, epochs=20)
    print("M_3 network: samples", net.samples, "loss", net.losses[0], "->", net.losses[-1])
    return net


def test_learned_m3_line_source_matches_oracle(K, trained_m3):
    """M_3, order 20, 3,872 triangles, 50 learned steps (network + exact mass + FP64 residual
    test, Newton fallback above 1e-6) against the FP64 Newton oracle: 1e-5 on u_0."""
    m = synth.jittered_mesh(45, -1.5, 1.5, seed=1)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(3, 20)
    u0 = synth.isotropic_moments(synth.line_source_density(G.cen), T.n)
    C = G.C
    dt = G.cfl_dt(0.4)
    sa, ss, q = np.zeros(C), np.ones(C), np.zeros(C)
    u_or = u0.copy()
    a_or = O.isotropic_alpha(T, u_or)
    assert O.mn_run(T, G, u_or, a_or, sa, ss, q, dt, 50)[0] == 0
    s = K.MNSolver(K.Mesh(m.xy, m.tri), 3, 20, mode="learned", tau=1e-8, fallback_tol=1e-6)
    s.set_mlp(trained_m3.params, trained_m3.norm)
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    rc, st = s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=50, stats=True)
    err0 = rel_l2(ud.cpu().numpy()[:, 0], u_or[:, 0])
    # every closure the network was asked for either passed the 1e-6 residual test or fell back
    print("learned M_3 u0 rel L2", err0, "stats", st)
    assert err0 <= 1e-5


def test_d2_to_t_final_every_mode(K, trained_m3):
    k, N, order = 224, 3, 20
    m = synth.jittered_mesh(k, -1.5, 1.5, seed=1)
    mesh = K.Mesh(m.xy, m.tri)
    g = mesh.geometry()
    C = mesh.ncells
    u0 = synth.isotropic_moments(synth.line_source_density(g["centroid"]), (N + 1) * (N + 2) // 2)
    dt = 0.4 * g["min_inradius"]
    nsteps = int(math.ceil(1.0 / dt))
    sa, ss, q = dev(np.zeros(C)), dev(np.ones(C)), dev(np.zeros(C))
    out = {}
    for mode, tau in [("fp64", 1e-10), ("mixed_tf32", 1e-8), ("mixed_bf16", 1e-8), ("learned", 1e-8)]:
        s = K.MNSolver(mesh, N, order, mode=mode, tau=tau)
        if mode == "learned":
            s.set_mlp(trained_m3.params, trained_m3.norm)
        ud = dev(u0)
        ad = s.isotropic_alpha(ud)
        if mode == "fp64":
            # stop one step short: the last step is recomputed below for sampled cells
            s.step(ud, ad, sa, ss, q, dt=dt, nsteps=nsteps - 1)
            u_prev, a_prev = ud.cpu().numpy().copy(), ad.cpu().numpy().copy()
            s.step(ud, ad, sa, ss, q, dt=dt, nsteps=1)
        else:
            s.step(ud, ad, sa, ss, q, dt=dt, nsteps=nsteps)
        out[mode] = ud.cpu().numpy()
    ref = out["fp64"][:, 0]
    for mode in ("mixed_tf32", "mixed_bf16", "learned"):
        err = rel_l2(out[mode][:, 0], ref)
        print(f"t = {nsteps * dt:.4f} ({nsteps} steps): {mode} u0 rel L2 vs FP64 {err:.3e}")
        assert err <= 1e-5, mode
    # the FP64 run's last step against the oracle for sampled cells (their update depends only on
    # themselves and their face neighbours)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(N, order)
    rng = np.random.default_rng(1)
    r = np.sqrt((G.cen ** 2).sum(axis=1))
    front = np.flatnonzero(np.abs(r - 1.0) < 0.1)     # where the wave front is at t = 1
    sample = np.unique(np.concatenate([rng.choice(C, 150, replace=False),
                                       rng.choice(front, min(150, front.size), replace=False)]))
    cells = np.unique(np.concatenate([sample, G.nbr[sample][G.nbr[sample] >= 0]]))
    Gs = O.Geometry(m.xy, m.tri[cells])
    us, als = u_prev[cells].copy(), a_prev[cells].copy()
    z = np.zeros(cells.size)
    assert O.mn_run(T, Gs, us, als, z, np.ones(cells.size), z, dt, 1)[0] == 0
    pos = np.searchsorted(cells, sample)
    err = rel_l2(out["fp64"][sample], us[pos])
    print("FP64 GPU last step vs oracle on", sample.size, "sampled cells:", err)
    assert err <= 1e-11
    # positivity and mass (Neumann walls, no absorption): the floor reaches the boundary only
    # as the isotropic state, whose boundary flux is zero
    mass = lambda u: float((g["area"] * u[:, 0]).sum())
    assert abs(mass(out["fp64"]) / mass(u0) - 1) < 1e-9


def test_learned_m3_residual_histogram(K, trained_m3):
    """What the M_3 network delivers: the relative moment residual |<m e> - u| / |u| of its
    proposals (alpha_1.. from the network in FP32, alpha_0 from the exact mass constraint) on
    held-out von Mises-Fisher samples and on the states of the line source, counted per decade
    against the 1e-6 acceptance threshold. Printed for the record; the assertions only check that
    the proposals are finite and better than the isotropic start."""
    N, order = 3, 20
    m = synth.jittered_mesh(45, -1.5, 1.5, seed=1)
    mesh = K.Mesh(m.xy, m.tri)
    s = K.MNSolver(mesh, N, order, mode="mixed_tf32", tau=1e-8)
    w, om, M = s.quadrature()
    n = s.n
    net = trained_m3
    # held-out samples
    c, kap, wt = synth.vmf_mixtures(20000, seed=99)
    u_v = s.vmf_moments(dev(c), dev(kap), dev(wt)).cpu().numpy()
    # line-source states after 40 steps
    g = mesh.geometry()
    u0 = synth.isotropic_moments(synth.line_source_density(g["centroid"]), n)
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    C = mesh.ncells
    s.step(ud, ad, dev(np.zeros(C)), dev(np.ones(C)), dev(np.zeros(C)),
           dt=0.4 * g["min_inradius"], nsteps=40)
    u_l = ud.cpu().numpy()
    # only the anisotropic ones are a question for the network
    u_l = u_l[np.linalg.norm(u_l[:, 1:], axis=1) > 1e-3 * np.abs(u_l[:, 0])]
    norm = net.norm.cpu().numpy().reshape(4, n - 1)
    edges = [0, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1, np.inf]
    for name, u in (("held-out vMF", u_v), ("line source t=40 dt", u_l)):
        x = (u[:, 1:] / u[:, :1] - norm[0]) / norm[1]
        y = K.mlp_forward(net.params, torch.from_numpy(x.astype(np.float32)).cuda(), n - 1, 64, n - 1)
        a1 = y.cpu().numpy().astype(np.float64) * norm[3] + norm[2]
        z = a1 @ M[:, 1:].T                                   # [samples, Q']
        e = np.exp(z)
        U = e @ (w[:, None] * M)                              # moments with alpha_0 = 0
        scale = u[:, 0] / U[:, 0]                             # exact mass: exp(alpha_0 m_0)
        res = np.linalg.norm(U * scale[:, None] - u, axis=1) / np.linalg.norm(u, axis=1)
        iso = np.linalg.norm(u[:, 1:], axis=1) / np.linalg.norm(u, axis=1)
        hist = np.histogram(res, bins=edges)[0] / res.size
        print(f"M_3 network residuals, {name} ({res.size} samples): median {np.median(res):.2e}, "
              f"accepted at 1e-6: {np.mean(res <= 1e-6):.4f}; per decade "
              + ", ".join(f"[{lo:g},{hi:g}): {h:.3f}" for lo, hi, h in zip(edges, edges[1:], hist)))
        assert np.isfinite(res).all()
        assert np.median(res) < np.median(iso)
