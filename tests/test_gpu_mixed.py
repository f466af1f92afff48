"""GPU parity of the mixed-precision paths (tensor-core Hessian moments in TF32 or BF16, FP64
gradient / Cholesky / line search, FP32 ansatz and flux) against the CPU oracle, through the C ABI.

Bars: the Hessian within FP32 accumulation error (the tensor-core operands are split into high
and low parts, so TF32 keeps about 21 and BF16 about 16 significant bits of each product, summed
over several hundred points in FP32); the closure to the same tolerance as FP64 (its
gradient and test are FP64); the step within 1e-5 relative L2 on the zeroth moment."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_08417_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED = ["mixed_tf32", "mixed_bf16"]


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


def vmf_u(T, count, seed, kappa_hi=20.0):
    mu, phi, w, ox, oy = O.quadrature(T.order)
    dirs = np.stack([ox, oy, mu], axis=1)
    c, k, wt = synth.vmf_mixtures(count, seed, kappa_hi=kappa_hi)
    psi = synth.vmf_density(dirs, c, k, wt)
    scale = np.exp(np.random.default_rng(seed).uniform(-3, 2, size=count))
    return (psi * scale[:, None]) @ (T.w[:, None] * T.M)


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-13), ("mixed_tf32", 1e-5), ("mixed_bf16", 1e-4)])
@pytest.mark.parametrize("N,order", [(1, 4), (2, 10), (3, 20), (5, 30)])
def test_hessian_matches_definition(K, mode, tol, N, order):
    """H = <m m^T exp(alpha.m)> on the oracle's full rule vs the library (FP64, or tensor-core
    moments); ragged cell count (not a multiple of the 128-row tile)."""
    m = synth.jittered_mesh(18, 0.0, 1.0, seed=3)
    mesh = K.Mesh(m.xy, m.tri)
    C = mesh.ncells
    assert C % 128 != 0
    s = K.MNSolver(mesh, N, order, mode=mode)
    T = O.Tables(N, order)
    u = vmf_u(T, C, seed=30 + N)
    a = O.isotropic_alpha(T, u)
    O.closure(T, u, a)
    Hg = s.hessian(dev(a)).cpu().numpy()
    worst = 0.0
    for i in range(C):
        e = T.w * np.exp(T.M @ a[i])
        H = T.M.T @ (e[:, None] * T.M)
        worst = max(worst, np.abs(Hg[i] - H).max() / np.abs(H).max())
    assert worst <= tol, worst


@pytest.mark.parametrize("mode", MIXED)
@pytest.mark.parametrize("N,order", [(1, 4), (3, 20), (5, 30)])
def test_mixed_gradient_moments_are_fp64(K, mode, N, order):
    """The mixed sweep's FP64 part: column 0 of H is m_0 <m exp(alpha.m)>, the ansatz moments
    (m_0 is constant), which the mixed modes form in FP64 with the scaled exponential and never
    from the tensor cores. Against the oracle's full rule for peaked vMF states: 1e-14 + 16 eps
    max_q sum_c |alpha_c m_c(q)| relative (the exponent is a sum of terms of that size, formed
    with a few roundings after scaling, and its absolute error is the exponential's relative one;
    1e-14 covers the exponential's own error; a TF32 or BF16 path would be off by 1e-7 or more);
    and, for exponents that are one constant z per cell, exp(z) within 1e-14 + 4|z| 2^-52
    relative over z in [-720, 80], which reaches the range test's slow path below -512 and gives
    exactly 0 below -707."""
    m = synth.jittered_mesh(18, 0.0, 1.0, seed=3)
    mesh = K.Mesh(m.xy, m.tri)
    C = mesh.ncells
    s = K.MNSolver(mesh, N, order, mode=mode)
    T = O.Tables(N, order)
    u = vmf_u(T, C, seed=60 + N, kappa_hi=50.0)
    a = O.isotropic_alpha(T, u)
    O.closure(T, u, a)
    Hg = s.hessian(dev(a)).cpu().numpy()
    col = np.empty((C, T.n))
    cond = np.empty(C)
    for i in range(C):
        col[i] = T.M.T @ (T.w * np.exp(T.M @ a[i]) * T.M[:, 0])
        cond[i] = np.abs(T.M * a[i]).sum(axis=1).max()
    rel = np.abs(Hg[:, :, 0] - col).max(axis=1) / np.abs(col).max(axis=1)
    bound = 1e-14 + 16.0 * 2.0 ** -52 * cond
    print("column 0 rel err: max", rel.max(), "median", np.median(rel), "max err/bound", (rel / bound).max())
    assert (rel <= bound).all(), (rel / bound).max()
    # constant exponent per cell: alpha = (z / m_0, 0, ...)
    m0 = T.M[0, 0]
    z = np.concatenate([np.random.default_rng(8).uniform(-720.0, 80.0, C - 5),
                        [0.0, -706.9, -707.5, -513.0, 79.0]])
    al = np.zeros((C, T.n))
    al[:, 0] = z / m0
    H00 = s.hessian(dev(al)).cpu().numpy()[:, 0, 0]
    norm = float((T.w * T.M[:, 0] ** 2).sum())
    ref = np.exp(z) * norm
    live = z > -707.0
    rel = np.abs(H00[live] - ref[live]) / ref[live]
    bound = 1e-14 + 4.0 * np.abs(z[live]) * 2.0 ** -52
    print("constant exponent: max rel err", rel.max(), "max err/bound", (rel / bound).max())
    assert (rel <= bound).all(), (rel / bound).max()
    assert (H00[z < -707.1] == 0).all()


@pytest.mark.parametrize("mode", MIXED)
@pytest.mark.parametrize("N,order", [(2, 10), (3, 20), (5, 30)])
def test_mixed_closure_matches_oracle(K, mode, N, order):
    T = O.Tables(N, order)
    m = synth.jittered_mesh(20, 0.0, 1.0, seed=4)
    mesh = K.Mesh(m.xy, m.tri)
    C = mesh.ncells
    s = K.MNSolver(mesh, N, order, mode=mode)
    u = vmf_u(T, C, seed=40 + N, kappa_hi=50.0)
    a_or = O.isotropic_alpha(T, u)
    st_or, _ = O.closure(T, u, a_or)
    ud = dev(u)
    ad = s.isotropic_alpha(ud)
    st = torch.zeros(C, dtype=torch.int32, device="cuda")
    rc, stats = s.closure(ud, ad, st, stats=True, check=False)
    st = st.cpu().numpy()
    ok = (st == 0) & (st_or == 0)
    assert ((st == 0) == (st_or == 0)).mean() > 0.98
    assert ok.mean() > 0.9
    a_gpu = ad.cpu().numpy()
    rec = np.exp(a_gpu[ok] @ T.M.T) @ (T.w[:, None] * T.M)
    rel = np.linalg.norm(rec - u[ok], axis=1) / np.linalg.norm(u[ok], axis=1)
    assert rel.max() <= 1e-10
    for i in np.flatnonzero(ok):
        e = T.w * np.exp(T.M @ a_or[i])
        lmin = np.linalg.eigvalsh(T.M.T @ (e[:, None] * T.M))[0]
        bound = 1e-9 * np.linalg.norm(u[i]) / lmin + 1e-12 * np.linalg.norm(a_or[i])
        assert np.linalg.norm(a_gpu[i] - a_or[i]) <= bound


@pytest.mark.parametrize("tau", [1e-10, 1e-8])
@pytest.mark.parametrize("mode", MIXED)
def test_mixed_line_source_m2_matches_oracle(K, mode, tau):
    """M_2 line source (3872 triangles, order 10), 50 steps: mixed vs the FP64 oracle on u_0, at
    the FP64 Newton tolerance and at the tolerance the benchmark uses for the mixed modes."""
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
    s = K.MNSolver(mesh, 2, 10, mode=mode, tau=tau)
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=50)
    u_gpu = ud.cpu().numpy()
    err0 = rel_l2(u_gpu[:, 0], u_or[:, 0])
    print(mode, "u0 rel L2", err0, "u rel L2", rel_l2(u_gpu, u_or))
    assert err0 <= 1e-5


@pytest.mark.parametrize("mode", MIXED)
def test_mixed_blocks_vacuum_m3_matches_oracle(K, mode):
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
    u_or = u0.copy()
    a_or = O.isotropic_alpha(T, u_or)
    assert O.mn_run(T, G, u_or, a_or, sa, ss, q, dt, 10, bc=1)[0] == 0
    s = K.MNSolver(mesh, N, order, mode=mode, bc="vacuum")
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=10)
    assert rel_l2(ud.cpu().numpy()[:, 0], u_or[:, 0]) <= 1e-5


@pytest.mark.parametrize("mode", MIXED)
def test_mixed_d2_size_sampled_against_oracle(K, mode):
    """Full-size M_3 line source (~100k triangles, order 20) in the benchmark's launch
    configuration: 3 mixed steps, then one more checked on sampled cells against the oracle (each
    sampled cell recomputed on a submesh of it and its neighbours)."""
    m = synth.jittered_mesh(224, -1.5, 1.5, seed=2)
    mesh = K.Mesh(m.xy, m.tri)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(3, 20)
    u0 = synth.isotropic_moments(synth.line_source_density(G.cen), T.n)
    C = G.C
    dt = G.cfl_dt(0.4)
    sa, ss, q = np.zeros(C), np.ones(C), np.zeros(C)
    s = K.MNSolver(mesh, 3, 20, mode=mode, tau=1e-8)
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=3)
    u_start, a_start = ud.cpu().numpy().copy(), ad.cpu().numpy().copy()
    s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=1)
    u_gpu = ud.cpu().numpy()
    rng = np.random.default_rng(1)
    front = np.flatnonzero((G.cen ** 2).sum(axis=1) < 0.05)
    sample = np.unique(np.concatenate([rng.choice(C, 150, replace=False),
                                       rng.choice(front, min(150, front.size), replace=False)]))
    cells = np.unique(np.concatenate([sample, G.nbr[sample][G.nbr[sample] >= 0]]))
    Gs = O.Geometry(m.xy, m.tri[cells])
    us, als = u_start[cells].copy(), a_start[cells].copy()
    O.mn_run(T, Gs, us, als, sa[cells], ss[cells], q[cells], dt, 1)
    pos = np.searchsorted(cells, sample)
    assert rel_l2(u_gpu[sample, 0], us[pos, 0]) <= 1e-5


@pytest.mark.parametrize("mode", ["fp64", "mixed_tf32"])
def test_m5_million_triangles_sampled_against_oracle(K, mode):
    """The large configuration: ~1M triangles (707^2 points), M_5 (21 moments), order-30
    quadrature (1800 points, 900 folded), line-source start in a seeded 7x7 block medium
    (sigma_a in [0,10], sigma_s in [0,1]). Two steps on the GPU, then a third checked on sampled
    cells against the oracle (each recomputed on a submesh of it and its neighbours)."""
    import bench
    W = bench.make_workload("m5_line_source_1m")
    m = W["mesh"]
    mesh = K.Mesh(m.xy, m.tri)
    C = W["C"]
    assert C > 990_000
    dt = 0.4 * mesh.geometry()["min_inradius"]
    s = K.MNSolver(mesh, 5, 30, mode=mode, tau=1e-10 if mode == "fp64" else 1e-8)
    ud = dev(W["u0"])
    ad = s.isotropic_alpha(ud)
    sa, ss, q = dev(W["sa"]), dev(W["ss"]), dev(W["q"])
    s.step(ud, ad, sa, ss, q, dt=dt, nsteps=2)
    u_start, a_start = ud.cpu().numpy().copy(), ad.cpu().numpy().copy()
    s.step(ud, ad, sa, ss, q, dt=dt, nsteps=1)
    u_gpu = ud.cpu().numpy()
    G_nbr = mesh.geometry()["nbr"]
    rng = np.random.default_rng(5)
    r2 = (W["cen"] ** 2).sum(axis=1)
    front = np.flatnonzero(r2 < 0.01)
    sample = np.unique(np.concatenate([rng.choice(C, 60, replace=False),
                                       rng.choice(front, min(60, front.size), replace=False)]))
    cells = np.unique(np.concatenate([sample, G_nbr[sample][G_nbr[sample] >= 0]]))
    T = O.Tables(5, 30)
    Gs = O.Geometry(m.xy, m.tri[cells])
    us, als = u_start[cells].copy(), a_start[cells].copy()
    nf, _ = O.mn_run(T, Gs, us, als, W["sa"][cells], W["ss"][cells], W["q"][cells], dt, 1)
    assert nf == 0
    pos = np.searchsorted(cells, sample)
    if mode == "fp64":
        assert rel_l2(u_gpu[sample], us[pos]) <= 1e-11
    else:
        assert rel_l2(u_gpu[sample, 0], us[pos, 0]) <= 1e-5


@pytest.mark.parametrize("mode", MIXED)
def test_peaked_closures_go_over_to_the_fp64_hessian(K, mode):
    """Cold closures of strongly peaked densities (vMF lobes up to kappa = 400, near the
    realizability boundary, where the Hessian is ill-conditioned): part of the cells leave the
    tensor-core Hessian for the FP64 one (FP32 factor not positive definite, or a stalled
    residual), are evaluated by the FP64 sweep, and have their FP64 quadrature parts summed in
    FP64. Every closure that the oracle solves is solved, to the same moments and alpha."""
    N, order = 3, 20
    T = O.Tables(N, order)
    m = synth.jittered_mesh(20, 0.0, 1.0, seed=4)
    mesh = K.Mesh(m.xy, m.tri)
    C = mesh.ncells
    s = K.MNSolver(mesh, N, order, mode=mode, tau=1e-10)
    u = vmf_u(T, C, seed=77, kappa_hi=400.0)
    a_or = O.isotropic_alpha(T, u)
    st_or, _ = O.closure(T, u, a_or)
    ud = dev(u)
    ad = s.isotropic_alpha(ud)
    st = torch.zeros(C, dtype=torch.int32, device="cuda")
    rc, stats = s.closure(ud, ad, st, stats=True, check=False)
    print(mode, "hand-overs", stats["handovers"], "of", C, "cells; evaluations", stats["evaluations"])
    assert stats["handovers"] > 0
    st = st.cpu().numpy()
    ok = (st == 0) & (st_or == 0)
    assert ((st == 0) == (st_or == 0)).mean() > 0.98
    assert ok.mean() > 0.9
    a_gpu = ad.cpu().numpy()
    rec = np.exp(a_gpu[ok] @ T.M.T) @ (T.w[:, None] * T.M)
    rel = np.linalg.norm(rec - u[ok], axis=1) / np.linalg.norm(u[ok], axis=1)
    assert rel.max() <= 1e-9
