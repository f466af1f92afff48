"""The GPU S_N step (kitrt_sn_step; Sec. 2, Eq. SNEqns2, with the upwind flux of Sec. 4.4 per
ordinate) against the oracle's S_N step: element by element on the ordinates, FP64 to 1e-12 and
FP32 to FP32 rounding, with isotropic and anisotropic (Henyey-Greenstein) scattering, both
boundary conditions, odd and even step counts, a ragged quadrature (Q' not a multiple of 32), the
full line-source mesh, and the argument checks."""
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


def _field(ox, oy, C, seed):
    """Positive ordinates depending on the direction only through (Omega_x, Omega_y), i.e. even in
    mu like every state of the 2D problem; evaluated at any set of directions."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.5, 2.0, size=C)
    b = rng.normal(size=(C, 2))
    c = rng.normal(size=(C, 3))
    ox, oy = ox[None, :], oy[None, :]
    return a[:, None] * np.exp(0.6 * (b[:, :1] * ox + b[:, 1:] * oy)
                               + 0.3 * (c[:, :1] * ox * ox + c[:, 1:2] * ox * oy + c[:, 2:] * oy * oy))


def _fold_map(T, om):
    """Index of one full-rule point with the direction of each folded point, and a check that
    every full point has a folded partner."""
    key = lambda x, y: (round(float(x), 11), round(float(y), 11))
    full = {}
    for q in range(T.Q):
        full.setdefault(key(T.ox[q], T.oy[q]), []).append(q)
    idx = np.array([full[key(x, y)][0] for x, y in om])
    assert sum(len(v) for v in full.values()) == T.Q and len(full) == om.shape[0]
    return idx


def _run_pair(K, k, N, order, bc, g, nsteps, fp32, seed=1, lo=-1.0, hi=1.0):
    m = synth.jittered_mesh(k, lo, hi, seed=seed)
    mesh = K.Mesh(m.xy, m.tri)
    s = K.MNSolver(mesh, N, order, bc=bc)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(N, order)
    w, om, _ = s.quadrature()
    idx = _fold_map(T, om)
    C = G.C
    rng = np.random.default_rng(seed + 10)
    sa, ss, q = rng.uniform(0, 2, C), rng.uniform(0, 1, C), rng.uniform(0, 0.5, C)
    dt = G.cfl_dt(0.4)
    psi_full = _field(T.ox, T.oy, C, seed)
    psi_fold = _field(om[:, 0], om[:, 1], C, seed)
    dtype = torch.float32 if fp32 else torch.float64
    dev = lambda a, dt_=torch.float64: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt_)
    p = dev(psi_fold, dtype)
    work = torch.empty_like(p)
    s.sn_step(p, work, dev(sa), dev(ss), dev(q), dt=dt, nsteps=nsteps, g=g)
    got = p.double().cpu().numpy()
    O.sn_run(T, G, psi_full, sa, ss, q, dt, nsteps, g=g, bc=0 if bc == "neumann" else 1)
    return got, psi_full[:, idx], psi_full


@pytest.mark.parametrize("bc", ["neumann", "vacuum"])
@pytest.mark.parametrize("g", [None, [1.0, 0.6, 0.36, 0.216]])
@pytest.mark.parametrize("nsteps", [7, 12])
def test_sn_fp64_matches_oracle(K, bc, g, nsteps):
    # order 6: Q' = 36 folded points (one full warp pass plus a ragged tail of 4)
    got, ref, full = _run_pair(K, 15, 3, 6, bc, g, nsteps, fp32=False)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("g", [None, [1.0, 0.6, 0.36, 0.216]])
def test_sn_fp32_matches_oracle(K, g):
    got, ref, full = _run_pair(K, 15, 3, 6, "vacuum", g, 12, fp32=True)
    # FP32 rounding of the start (6e-8) and of about ten operations per ordinate and step
    assert np.abs(got - ref).max() <= 5e-6 * np.abs(ref).max()


def test_sn_odd_order_keeps_the_equator_once(K):
    # order 5: mu = 0 is a node of its own (weight w, not 2w) after folding
    got, ref, full = _run_pair(K, 9, 2, 5, "neumann", None, 5, fp32=False)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("fp32", [False, True])
def test_sn_line_source_full_mesh(K, fp32):
    """The line-source mesh and quadrature of the benchmark (224^2 points, 99,458 triangles, order
    20: Q' = 400), isotropic Gaussian start, sigma_s = 1, Neumann walls; 2 steps, every ordinate
    of every cell compared with the oracle."""
    N, order, nsteps = 3, 20, 2
    m = synth.jittered_mesh(224, -1.5, 1.5, seed=2)
    mesh = K.Mesh(m.xy, m.tri)
    s = K.MNSolver(mesh, N, order)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(N, order)
    w, om, _ = s.quadrature()
    idx = _fold_map(T, om)
    C = G.C
    phi = synth.line_source_density(G.cen)
    psi_full = np.repeat((phi / (4 * math.pi))[:, None], T.Q, axis=1)
    psi_fold = np.ascontiguousarray(psi_full[:, idx])
    sa, ss, q = np.zeros(C), np.ones(C), np.zeros(C)
    dt = G.cfl_dt(0.4)
    dtype = torch.float32 if fp32 else torch.float64
    dev = lambda a, dt_=torch.float64: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt_)
    p = dev(psi_fold, dtype)
    work = torch.empty_like(p)
    s.sn_step(p, work, dev(sa), dev(ss), dev(q), dt=dt, nsteps=nsteps)
    got = p.double().cpu().numpy()
    O.sn_run(T, G, psi_full, sa, ss, q, dt, nsteps)
    ref = psi_full[:, idx]
    tol = 2e-6 if fp32 else 1e-12
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    # total particle number changes only by the (tiny) boundary outflow of the floor
    mass = lambda ps: float(G.area @ (ps @ w))
    m0 = mass(psi_fold)
    assert abs(mass(got) / m0 - 1) < (1e-6 if fp32 else 1e-12)


def test_sn_argument_checks_and_zero_steps(K):
    m = synth.jittered_mesh(4, 0.0, 1.0, seed=0)
    mesh = K.Mesh(m.xy, m.tri)
    s = K.MNSolver(mesh, 2, 4)
    C = mesh.ncells
    p = torch.rand((C, s.Qf), dtype=torch.float64, device="cuda")
    p0 = p.clone()
    work = torch.empty_like(p)
    z = torch.zeros(C, dtype=torch.float64, device="cuda")
    assert s.sn_step(p, work, z, z, z, nsteps=0) == 0
    assert torch.equal(p, p0)
    # g[0] must be 1; g must be finite
    assert s.sn_step(p, work, z, z, z, g=[0.5, 0.0, 0.0], check=False) == 1
    assert s.sn_step(p, work, z, z, z, g=[1.0, float("nan"), 0.0], check=False) == 1
    # the scratch must not overlap the ordinates
    lib = K._lib()
    rc = lib.kitrt_sn_step(s.handle, K._dev(p), K._dev(p), 0, K._dev(z), K._dev(z), K._dev(z),
                           None, 0.0, 1, K._stream())
    assert rc == 1
    assert torch.equal(p, p0)
    # a pure absorber with uniform ordinates decays in closed form (1 - dt sigma_a) per step
    u = torch.full((C, s.Qf), 0.25, dtype=torch.float64, device="cuda")
    sa = torch.full((C,), 2.0, dtype=torch.float64, device="cuda")
    dt = 0.01
    s.sn_step(u, work, sa, z, z, dt=dt, nsteps=3)
    assert torch.allclose(u, torch.full_like(u, 0.25 * (1 - dt * 2.0) ** 3), rtol=1e-14, atol=0)


def test_sn_two_triangle_mesh(K):
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    mesh = K.Mesh(xy, tri)
    s = K.MNSolver(mesh, 1, 3, bc="vacuum")
    G = O.Geometry(xy, tri)
    T = O.Tables(1, 3)
    w, om, _ = s.quadrature()
    idx = _fold_map(T, om)
    sa, ss, q = np.array([0.3, 1.2]), np.array([0.7, 0.1]), np.array([0.0, 2.0])
    psi_full = _field(T.ox, T.oy, 2, 3)
    psi_fold = _field(om[:, 0], om[:, 1], 2, 3)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    p = dev(psi_fold)
    s.sn_step(p, torch.empty_like(p), dev(sa), dev(ss), dev(q), dt=0.05, nsteps=1, g=[1.0, 0.4])
    ref = O.sn_step(T, G, psi_full, sa, ss, q, 0.05, g=[1.0, 0.4], bc=1)[:, idx]
    assert np.abs(p.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
