"""GPU parity of the FP64 path against the CPU oracle, through the C ABI.

Tolerances: the FP64 step must match the oracle to 1e-11 relative L2 on u; the closure alpha to
round-off scaled by the conditioning of the dual Hessian; geometry bit-exact for integers."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_08417_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTHREADS = 0  # oracle: OpenMP default (all host cores)


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


def vmf_u(order, M_full, w_full, count, seed, kappa_hi=50.0):
    mu, phi, w, ox, oy = O.quadrature(order)
    dirs = np.stack([ox, oy, mu], axis=1)
    c, k, wt = synth.vmf_mixtures(count, seed, kappa_hi=kappa_hi)
    psi = synth.vmf_density(dirs, c, k, wt)
    scale = np.exp(np.random.default_rng(seed).uniform(-4, 3, size=count))
    return (psi * scale[:, None]) @ (w_full[:, None] * M_full)


def test_mesh_geometry_matches_oracle(K):
    m = synth.jittered_mesh(45, -1.5, 1.5, seed=1)
    mesh = K.Mesh(m.xy, m.tri)
    g = mesh.geometry()
    G = O.Geometry(m.xy, m.tri)
    np.testing.assert_array_equal(g["nbr"], G.nbr)
    np.testing.assert_array_equal(g["nrm"], G.nrm)
    np.testing.assert_allclose(g["area"], G.area, rtol=1e-15)
    np.testing.assert_allclose(g["perim"], G.perim, rtol=1e-15)
    np.testing.assert_allclose(g["centroid"], G.cen, rtol=1e-15, atol=1e-16)
    assert abs(g["min_inradius"] - np.min(2 * G.area / G.perim)) < 1e-16


@pytest.mark.parametrize("N,order", [(1, 3), (2, 10), (3, 20), (5, 30), (3, 7)])
def test_folded_quadrature_matches_oracle_tables(K, N, order):
    m = synth.jittered_mesh(4, 0.0, 1.0, seed=0)
    mesh = K.Mesh(m.xy, m.tri)
    s = K.MNSolver(mesh, N, order)
    w, om, M = s.quadrature()
    assert s.Q == 2 * order * order and s.Qf == (order + 1) // 2 * 2 * order
    T = O.Tables(N, order)
    # same integrals: Gram matrix and first moments over the folded and the full rule
    np.testing.assert_allclose(M.T @ (w[:, None] * M), T.M.T @ (T.w[:, None] * T.M), atol=1e-13)
    assert abs(w.sum() - 4 * math.pi) < 1e-12
    # every folded point carries the oracle's basis values at its (|mu|, phi)
    s2 = (om ** 2).sum(axis=1)
    mu = np.sqrt(np.maximum(0.0, 1.0 - s2))
    phi = np.mod(np.arctan2(om[:, 0], om[:, 1]), 2 * math.pi)
    for q in range(0, s.Qf, max(1, s.Qf // 40)):
        np.testing.assert_allclose(M[q], O.basis(N, mu[q], phi[q]), atol=2e-13)


@pytest.mark.parametrize("N,order", [(2, 10), (3, 20), (5, 30)])
def test_isotropic_closed_form_on_gpu(K, N, order):
    m = synth.jittered_mesh(8, 0.0, 1.0, seed=0)
    mesh = K.Mesh(m.xy, m.tri)
    s = K.MNSolver(mesh, N, order)
    T = O.Tables(N, order)
    rng = np.random.default_rng(1)
    u = np.zeros((mesh.ncells, s.n))
    u[:, 0] = np.exp(rng.uniform(-8, 4, size=mesh.ncells))
    a = s.isotropic_alpha(dev(u))
    np.testing.assert_allclose(a.cpu().numpy(), O.isotropic_alpha(T, u), rtol=1e-15, atol=1e-15)
    # the closure from a perturbed start returns it
    a2 = a + 0.2 * torch.randn_like(a)
    st = torch.zeros(mesh.ncells, dtype=torch.int32, device="cuda")
    s.closure(dev(u), a2, st)
    assert int(st.abs().max()) == 0
    np.testing.assert_allclose(a2.cpu().numpy(), a.cpu().numpy(), atol=1e-12 * float(a.abs().max()))


@pytest.mark.parametrize("N,order,count", [(2, 10, 333), (3, 20, 517), (5, 30, 130)])
def test_closure_matches_oracle(K, N, order, count):
    """Random realizable moments (vMF mixtures up to kappa 50, scales e^-4..e^3); several tiles
    and a ragged tail. Both sides converge to the unique minimiser; alpha agrees to a bound set by
    the smallest Hessian eigenvalue."""
    T = O.Tables(N, order)
    # a mesh with exactly `count` cells is not needed: the closure is per cell, so use a mesh with
    # at least `count` cells and compare the first `count`
    k = int(math.ceil(math.sqrt(count / 2))) + 2
    m = synth.jittered_mesh(k, 0.0, 1.0, seed=2)
    mesh = K.Mesh(m.xy, m.tri)
    C = mesh.ncells
    s = K.MNSolver(mesh, N, order)
    u = vmf_u(order, T.M, T.w, C, seed=10 + N)
    a_or = O.isotropic_alpha(T, u)
    st_or, it_or = O.closure(T, u, a_or, nthreads=NTHREADS)
    ud = dev(u)
    ad = s.isotropic_alpha(ud)
    st = torch.zeros(C, dtype=torch.int32, device="cuda")
    rc, stats = s.closure(ud, ad, st, stats=True, check=False)
    st = st.cpu().numpy()
    a_gpu = ad.cpu().numpy()
    ok = (st == 0) & (st_or == 0)
    assert ok.mean() > 0.9, (np.bincount(st), np.bincount(st_or))
    # failures agree in kind: a cell the oracle solves the GPU solves too (and vice versa)
    assert ((st == 0) == (st_or == 0)).mean() > 0.98
    for i in np.flatnonzero(ok):
        e = T.w * np.exp(T.M @ a_or[i])
        H = T.M.T @ (e[:, None] * T.M)
        lmin = np.linalg.eigvalsh(H)[0]
        bound = 1e-9 * np.linalg.norm(u[i]) / lmin + 1e-12 * np.linalg.norm(a_or[i])
        assert np.linalg.norm(a_gpu[i] - a_or[i]) <= bound, (i, np.linalg.norm(a_gpu[i] - a_or[i]), bound)
    # moment reproduction of the GPU answer, computed by the oracle's tables
    rec = np.exp(a_gpu[ok] @ T.M.T) @ (T.w[:, None] * T.M)
    rel = np.linalg.norm(rec - u[ok], axis=1) / np.linalg.norm(u[ok], axis=1)
    assert rel.max() <= 1e-10
    assert stats["closures"] == C and stats["max_evals"] >= 1


def _line_source(K, k, N, order, width=0.03):
    m = synth.jittered_mesh(k, -1.5, 1.5, seed=1)
    mesh = K.Mesh(m.xy, m.tri)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(N, order)
    u0 = synth.isotropic_moments(synth.line_source_density(G.cen, width=width), T.n)
    return m, mesh, G, T, u0


def test_line_source_m2_50_steps_matches_oracle(K):
    """M_2 FP64 line source: 45^2 jittered points (3872 triangles), order-10 quadrature, Gaussian
    width 0.03 + 1e-4 floor, sigma_s = 1, sigma_a = 0, CFL 0.4, Neumann, tau 1e-10, 50 steps.
    Parity bar: 1e-11 relative L2 on u."""
    m, mesh, G, T, u0 = _line_source(K, 45, 2, 10)
    C = G.C
    dt = G.cfl_dt(0.4)
    sa, ss, q = np.zeros(C), np.ones(C), np.zeros(C)
    u_or = u0.copy()
    a_or = O.isotropic_alpha(T, u_or)
    nf, _ = O.mn_run(T, G, u_or, a_or, sa, ss, q, dt, 50, nthreads=NTHREADS)
    assert nf == 0
    s = K.MNSolver(mesh, 2, 10)
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    rc, stats = s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=50, stats=True)
    u_gpu = ud.cpu().numpy()
    err = rel_l2(u_gpu, u_or)
    print("M2 line source 50 steps rel L2", err, stats)
    assert err <= 1e-11
    assert rel_l2(ad.cpu().numpy(), a_or) <= 1e-9
    # mass: sum A u_0 conserved (Neumann walls, no absorption)
    assert abs((G.area * u_gpu[:, 0]).sum() / (G.area * u0[:, 0]).sum() - 1) < 1e-12


@pytest.mark.parametrize("bc", ["neumann", "vacuum"])
def test_blocks_m3_matches_oracle(K, bc):
    """M_3 with per-block sigma_a in [0,10], sigma_s in [0,1] and a unit source in the centre
    block (checkerboard-like medium, Sec. 7.2), 10 steps."""
    N, order = 3, 10
    m = synth.jittered_mesh(30, 0.0, 7.0, seed=3)
    mesh = K.Mesh(m.xy, m.tri)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(N, order)
    blk, sab, ssb = synth.block_coefficients(G.cen, 0.0, 7.0, 7, seed=3)
    sa, ss = sab[blk], ssb[blk]
    q = np.where(blk == 24, 1.0, 0.0)
    u0 = np.zeros((G.C, T.n))
    u0[:, 0] = 1e-4 / math.sqrt(4 * math.pi)
    dt = G.cfl_dt(0.4)
    assert dt * (sa + ss).max() <= 0.6
    u_or = u0.copy()
    a_or = O.isotropic_alpha(T, u_or)
    nf, _ = O.mn_run(T, G, u_or, a_or, sa, ss, q, dt, 10, bc=1 if bc == "vacuum" else 0,
                     nthreads=NTHREADS)
    assert nf == 0
    s = K.MNSolver(mesh, N, order, bc=bc)
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=10)
    assert rel_l2(ud.cpu().numpy(), u_or) <= 1e-11


def test_two_triangle_mesh_and_tiny_inputs(K):
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    mesh = K.Mesh(xy, tri)
    G = O.Geometry(xy, tri)
    T = O.Tables(2, 4)
    s = K.MNSolver(mesh, 2, 4)
    u = vmf_u(4, T.M, T.w, 2, seed=5, kappa_hi=3.0)
    sa, ss, q = np.array([0.3, 1.2]), np.array([0.7, 0.1]), np.array([0.0, 2.0])
    u_or = u.copy()
    a_or = O.isotropic_alpha(T, u_or)
    O.mn_run(T, G, u_or, a_or, sa, ss, q, 0.01, 3)
    ud = dev(u)
    ad = s.isotropic_alpha(ud)
    s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=0.01, nsteps=3)
    assert rel_l2(ud.cpu().numpy(), u_or) <= 1e-12


def test_nonrealizable_and_nan_inputs_return_status(K):
    """Moments outside the realizable set and NaN inputs come back as per-cell status codes and a
    non-zero return value; the kernels do not trap and the context stays usable."""
    m = synth.jittered_mesh(5, 0.0, 1.0, seed=0)
    mesh = K.Mesh(m.xy, m.tri)
    C = mesh.ncells
    s = K.MNSolver(mesh, 1, 6, max_iter=30)
    T = O.Tables(1, 6)
    u = np.zeros((C, s.n))
    u[:, 0] = 1.0
    u[0, 1] = 5.0             # |u_1| far beyond u_0: not realizable
    u[1, :] = np.nan
    ud = dev(u)
    ad = s.isotropic_alpha(dev(np.where(np.isnan(u), 1.0, u)))
    st = torch.zeros(C, dtype=torch.int32, device="cuda")
    rc = s.closure(ud, ad, st, check=False)
    st = st.cpu().numpy()
    assert rc != 0
    assert st[0] != 0 and st[1] != 0
    assert (st[2:] == 0).all()
    # the context still works
    u2 = np.zeros((C, s.n))
    u2[:, 0] = 2.0
    a2 = s.isotropic_alpha(dev(u2))
    assert s.closure(dev(u2), a2) == 0


def test_d2_size_one_step_sampled_against_oracle(K):
    """Full-size M_3 line source (224^2 points, ~100k triangles, order 20) in the benchmark's
    launch configuration: one FP64 step on the GPU; the oracle recomputes the step for a sample of
    cells on a submesh holding each sampled cell and its neighbours (their updates depend on
    nothing else)."""
    m, mesh, G, T, u0 = _line_source(K, 224, 3, 20)
    C = G.C
    dt = G.cfl_dt(0.4)
    sa, ss, q = np.zeros(C), np.ones(C), np.zeros(C)
    s = K.MNSolver(mesh, 3, 20)
    # a non-trivial state: advance 3 steps on the GPU first, then compare the 4th
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=3)
    u_start = ud.cpu().numpy().copy()
    a_start = ad.cpu().numpy().copy()
    s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=1)
    u_gpu = ud.cpu().numpy()
    rng = np.random.default_rng(0)
    r2 = (G.cen ** 2).sum(axis=1)
    front = np.flatnonzero(r2 < 0.05)                       # cells the pulse has reached
    sample = np.unique(np.concatenate([rng.choice(C, 150, replace=False),
                                       rng.choice(front, min(150, front.size), replace=False)]))
    cells = np.unique(np.concatenate([sample, G.nbr[sample][G.nbr[sample] >= 0]]))
    sub_tri = m.tri[cells]
    Gs = O.Geometry(m.xy, sub_tri)
    us = u_start[cells].copy()
    als = a_start[cells].copy()
    O.mn_run(T, Gs, us, als, sa[cells], ss[cells], q[cells], dt, 1)
    pos = np.searchsorted(cells, sample)
    err = np.linalg.norm(us[pos] - u_gpu[sample]) / np.linalg.norm(u_gpu[sample])
    assert err <= 1e-11, err


def test_table_exp_against_reference_exp(K):
    """The quadrature kernels' FP64 exp (Tang's table-driven method) against the C library's exp:
    with alpha = (a, 0, ...) the exponent is the single rounded product a * m_0, so the ansatz
    returned by kitrt_ansatz is exp of a known double; 1 + 2^-52 relative (about two ulps) over
    the whole finite range, 0 below -707."""
    m = synth.jittered_mesh(40, 0.0, 1.0, seed=0)
    mesh = K.Mesh(m.xy, m.tri)
    C = mesh.ncells
    s = K.MNSolver(mesh, 1, 2)
    w, om, M = s.quadrature()
    m0 = M[0, 0]
    rng = np.random.default_rng(7)
    a0 = np.concatenate([rng.uniform(-700, 700, C - 6) / m0,
                         np.array([0.0, 1e-300, -1e-12, 709.7, -706.9, -720.0]) / m0])
    alpha = np.zeros((C, s.n))
    alpha[:, 0] = a0
    psi = s.ansatz(dev(alpha)).cpu().numpy()
    z = a0 * m0
    ref = np.exp(z)
    live = z > -707
    rel = np.abs(psi[live, 0] - ref[live]) / ref[live]
    assert rel.max() <= 2.0 ** -51, rel.max()
    assert (psi[~live, 0] == 0).all()
    assert np.all(psi == psi[:, :1])  # m_0 is constant: every point sees the same exponent


def test_step_calls_continue_from_the_solver_state(K):
    """Stepping one kitrt_step call at a time with the same alpha buffer continues from the
    solver's closure state: the result is bitwise that of one call of all the steps, the continued
    calls evaluate fewer cells than a cold first step, and kitrt_mn_reset (or another alpha
    buffer) starts cold again with the same result to the closure tolerance."""
    m = synth.jittered_mesh(45, -1.5, 1.5, seed=1)
    mesh = K.Mesh(m.xy, m.tri)
    C = mesh.ncells
    s = K.MNSolver(mesh, 2, 10, tau=1e-10)
    u0 = synth.isotropic_moments(synth.line_source_density(m.centroids()), s.n)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sa, ss, q = dev(np.zeros(C)), dev(np.ones(C)), dev(np.zeros(C))
    dt, nsteps = 0.4 * mesh.geometry()["min_inradius"], 8
    ua = dev(u0)
    aa = s.isotropic_alpha(ua)
    s.step(ua, aa, sa, ss, q, dt=dt, nsteps=nsteps)
    s.reset()
    ub = dev(u0)
    ab = s.isotropic_alpha(ub)
    evals = []
    for _ in range(nsteps):
        _, st = s.step(ub, ab, sa, ss, q, dt=dt, nsteps=1, stats=True)
        evals.append(st["evaluations"])
    assert torch.equal(ua, ub) and torch.equal(aa, ab)
    assert evals[0] >= C and max(evals[1:]) < evals[0]
    # a continued step and a cold step from the same state reach the same closure to tolerance
    ad = ab.clone()
    uc, ud = ub.clone(), ub.clone()
    s.step(uc, ab, sa, ss, q, dt=dt, nsteps=1)  # continues (same alpha buffer)
    s.reset()
    s.step(ud, ad, sa, ss, q, dt=dt, nsteps=1)  # cold, from the same alpha
    assert (torch.linalg.norm(uc - ud) / torch.linalg.norm(uc)).item() <= 1e-12


def test_a_new_warm_start_in_a_reused_buffer_starts_cold(K):
    """Continuation is decided per cell by the alpha's contents, not by the buffer it sits in: a
    warm start written into the buffer of the last call, or into a freshly allocated buffer that
    may reuse a freed one's address, gives bitwise the result of a solver that never stepped
    (a cold start); the solver's own output passed back in a different buffer continues."""
    m = synth.jittered_mesh(45, -1.5, 1.5, seed=1)
    mesh = K.Mesh(m.xy, m.tri)
    C = mesh.ncells
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sa, ss, q = dev(np.zeros(C)), dev(np.ones(C)), dev(np.zeros(C))
    dt = 0.4 * mesh.geometry()["min_inradius"]
    s = K.MNSolver(mesh, 2, 10, tau=1e-10)
    u0 = synth.isotropic_moments(synth.line_source_density(m.centroids()), s.n)
    ua = dev(u0)
    aa = s.isotropic_alpha(ua)
    s.step(ua, aa, sa, ss, q, dt=dt, nsteps=5)
    u_mid = ua.clone()
    # (1) a new warm start written into the same buffer (every row differs from the solver's
    # output: its alpha_0 is scaled)
    aa.copy_(aa * 0.999)
    a_start = aa.clone()
    _, st = s.step(ua, aa, sa, ss, q, dt=dt, nsteps=3, stats=True)
    fresh = K.MNSolver(mesh, 2, 10, tau=1e-10)
    ub = u_mid.clone()
    ab = a_start
    _, st_fresh = fresh.step(ub, ab, sa, ss, q, dt=dt, nsteps=3, stats=True)
    assert torch.equal(ua, ub) and torch.equal(aa, ab)
    assert st["evaluations"] == st_fresh["evaluations"]
    # (2) the old buffer freed, a new one allocated (the caching allocator may hand back the same
    # address) and filled with a different warm start
    ptr = aa.data_ptr()
    u_mid2 = ua.clone()
    del aa
    torch.cuda.synchronize()
    ac = torch.empty((C, s.n), dtype=torch.float64, device="cuda")
    ac.copy_(s.isotropic_alpha(ua) * 1.001)
    print("reallocated at the same address:", ac.data_ptr() == ptr)
    s.step(ua, ac, sa, ss, q, dt=dt, nsteps=2)
    fresh2 = K.MNSolver(mesh, 2, 10, tau=1e-10)
    ud = u_mid2.clone()
    ad = fresh2.isotropic_alpha(ud) * 1.001
    fresh2.step(ud, ad, sa, ss, q, dt=dt, nsteps=2)
    assert torch.equal(ua, ud) and torch.equal(ac, ad)
    # (3) the solver's own output, copied to another buffer, continues: fewer passes than cold
    ae = ac.clone()
    _, st_cont = s.step(ua, ae, sa, ss, q, dt=dt, nsteps=1, stats=True)
    assert st_cont["evaluations"] < C


def test_step_rejects_an_unstable_time_step_before_touching_u(K):
    """dt (P_i/(2 A_i) + sigma_a,i + sigma_s,i) <= 1 in every cell keeps the kinetic update of every
    ordinate positive; a step beyond it, or a negative coefficient, returns EINVAL and leaves u
    and alpha as they were."""
    m = synth.jittered_mesh(20, 0.0, 1.0, seed=3)
    mesh = K.Mesh(m.xy, m.tri)
    C = mesh.ncells
    g = mesh.geometry()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    s = K.MNSolver(mesh, 2, 10, tau=1e-10)
    u = dev(synth.isotropic_moments(np.full(C, 1.0), s.n))
    a = s.isotropic_alpha(u)
    sa, ss, q = np.zeros(C), np.ones(C), np.zeros(C)
    hpa = g["perim"] / (2 * g["area"])
    dt_max = 1.0 / (hpa + sa + ss).max()
    u_keep, a_keep = u.clone(), a.clone()
    rc = s.step(u, a, dev(sa), dev(ss), dev(q), dt=1.01 * dt_max, nsteps=2, check=False)
    assert rc == 1 and torch.equal(u, u_keep) and torch.equal(a, a_keep)
    bad = ss.copy()
    bad[C // 2] = -0.5
    rc = s.step(u, a, dev(sa), dev(bad), dev(q), dt=0.5 * dt_max, nsteps=1, check=False)
    assert rc == 1 and torch.equal(u, u_keep)
    # at the bound itself the step runs
    rc = s.step(u, a, dev(sa), dev(ss), dev(q), dt=dt_max, nsteps=1, check=False)
    assert rc == 0
