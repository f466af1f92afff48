"""The GPU discrete adjoint (kitrt_adjoint) against the oracle's adjoint, against central finite
differences of the GPU forward (step 1e-6, agreement to 1e-6 relative to the gradient's scale),
and through the torch.autograd binding. Checkerboard-like block media (Sec. 7.2): per-block
sigma_a in [0,10], sigma_s in [0,1], unit isotropic source in the centre block, vacuum walls,
absorbed energy in the centre 3x3 blocks."""
import math
import os

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


def blocks_problem(K, k, N, order, seed=3, nb=7):
    m = synth.jittered_mesh(k, 0.0, 7.0, seed=seed)
    mesh = K.Mesh(m.xy, m.tri)
    cen = m.centroids()
    blk, sa, ss = synth.block_coefficients(cen, 0.0, 7.0, nb, seed)
    q = np.where(blk == (nb // 2) * nb + nb // 2, 1.0, 0.0)
    bx, by = blk // nb, blk % nb
    tgt = ((bx >= 2) & (bx <= 4) & (by >= 2) & (by <= 4)).astype(np.uint8)
    n = (N + 1) * (N + 2) // 2
    u0 = np.zeros((m.ncells, n))
    u0[:, 0] = 1e-4 / math.sqrt(4 * math.pi)
    return m, mesh, blk, sa, ss, q, tgt, u0


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_J_grad(K, s, blk, sa, ss, q, tgt, u0, dt, nsteps, ckpt):
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    J, gsa, gss = s.adjoint(ud, ad, dev(sa[blk]), dev(ss[blk]), dev(q), dev(blk.astype(np.int32)),
                            len(sa), dev(tgt), dt, nsteps, ckpt)
    return J, gsa, gss


@pytest.mark.parametrize("ckpt", [5, 16])
def test_adjoint_matches_oracle_adjoint(K, ckpt):
    N, order, nsteps = 2, 4, 12
    m, mesh, blk, sa, ss, q, tgt, u0 = blocks_problem(K, 13, N, order)
    s = K.MNSolver(mesh, N, order, bc="vacuum", tau=1e-13)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(N, order)
    dt = G.cfl_dt(0.4)
    J, gsa, gss = gpu_J_grad(K, s, blk, sa, ss, q, tgt, u0, dt, nsteps, ckpt)
    Jo, gsao, gsso = O.mn_adjoint(T, G, blk.astype(np.int32), sa, ss, q, tgt, dt, nsteps, u0,
                                  O.isotropic_alpha(T, u0), bc=1, tau=1e-13)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    g, go = np.concatenate([gsa, gss]), np.concatenate([gsao, gsso])
    assert np.linalg.norm(g - go) / np.linalg.norm(go) <= 1e-9


def test_adjoint_m3_order10_matches_oracle_adjoint(K):
    """The adjoint configuration's arithmetic at a size the oracle handles: M_3, order 10, a
    31^2-point mesh of the 7x7 block medium, 32 steps with checkpoints every 16 (two segments, the
    recomputation path): J to 1e-12 and the 98 gradients to 1e-9 relative L2 of the oracle's
    exact transpose."""
    N, order, nsteps, ckpt = 3, 10, 32, 16
    m, mesh, blk, sa, ss, q, tgt, u0 = blocks_problem(K, 31, N, order)
    s = K.MNSolver(mesh, N, order, bc="vacuum", tau=1e-13)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(N, order)
    dt = G.cfl_dt(0.4)
    J, gsa, gss = gpu_J_grad(K, s, blk, sa, ss, q, tgt, u0, dt, nsteps, ckpt)
    Jo, gsao, gsso = O.mn_adjoint(T, G, blk.astype(np.int32), sa, ss, q, tgt, dt, nsteps, u0,
                                  O.isotropic_alpha(T, u0), bc=1, tau=1e-13)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    g, go = np.concatenate([gsa, gss]), np.concatenate([gsao, gsso])
    err = np.linalg.norm(g - go) / np.linalg.norm(go)
    print("M_3 order 10 adjoint vs oracle: rel L2", err)
    assert err <= 1e-9


def test_adjoint_matches_central_differences(K):
    """All 98 coefficients of a ~1,800-triangle M_3 blocks problem, 50 steps, checkpoints every
    16: |FD - adjoint| <= 1e-6 max |gradient|."""
    N, order, nsteps, h = 3, 10, 50, 1e-6
    m, mesh, blk, sa, ss, q, tgt, u0 = blocks_problem(K, 31, N, order)
    s = K.MNSolver(mesh, N, order, bc="vacuum", tau=1e-12)
    dt = 0.4 * mesh.geometry()["min_inradius"]
    assert dt * (sa.max() + ss.max()) <= 0.6
    J, gsa, gss = gpu_J_grad(K, s, blk, sa, ss, q, tgt, u0, dt, nsteps, 16)
    g = np.concatenate([gsa, gss])
    scale = np.abs(g).max()
    fd = np.zeros_like(g)
    for k in range(g.size):
        p = np.concatenate([sa, ss])
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        Jp = gpu_J_grad(K, s, blk, pp[:49], pp[49:], q, tgt, u0, dt, nsteps, nsteps)[0]
        Jm = gpu_J_grad(K, s, blk, pm[:49], pm[49:], q, tgt, u0, dt, nsteps, nsteps)[0]
        fd[k] = (Jp - Jm) / (2 * h)
    err = np.abs(fd - g).max() / scale
    print("adjoint vs FD: max |diff| / max |g| =", err, "J =", J)
    assert err <= 1e-6


def test_autograd_function(K):
    from paper_2205_08417_gb300.adjoint import absorbed_energy
    N, order, nsteps = 2, 6, 20
    m, mesh, blk, sa, ss, q, tgt, u0 = blocks_problem(K, 15, N, order)
    s = K.MNSolver(mesh, N, order, bc="vacuum", tau=1e-12)
    dt = 0.4 * mesh.geometry()["min_inradius"]
    sab = dev(sa).requires_grad_(True)
    ssb = dev(ss).requires_grad_(True)
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    J = absorbed_energy(sab, ssb, s, ud, ad, dev(q), dev(blk.astype(np.int32)), dev(tgt), dt, nsteps, 8)
    J.backward()
    J2, gsa, gss = gpu_J_grad(K, s, blk, sa, ss, q, tgt, u0, dt, nsteps, 8)
    assert abs(float(J) - J2) <= 1e-13 * abs(J2)
    assert torch.allclose(sab.grad.cpu(), torch.from_numpy(gsa), rtol=1e-12, atol=0)
    assert torch.allclose(ssb.grad.cpu(), torch.from_numpy(gss), rtol=1e-12, atol=0)


def test_adjoint_full_size_blocks_sampled_fd(K):
    """The adjoint configuration at full size: ~60k triangles on [0,7]^2 (173^2 points), M_3,
    order 10, 400 steps, checkpoints every 16; central differences on a sample of coefficients."""
    N, order, nsteps, h = 3, 10, 400, 1e-6
    m, mesh, blk, sa, ss, q, tgt, u0 = blocks_problem(K, 173, N, order)
    s = K.MNSolver(mesh, N, order, bc="vacuum", tau=1e-12)
    dt = 0.4 * mesh.geometry()["min_inradius"]
    J, gsa, gss = gpu_J_grad(K, s, blk, sa, ss, q, tgt, u0, dt, nsteps, 16)
    g = np.concatenate([gsa, gss])
    scale = np.abs(g).max()
    assert scale > 0
    p0 = np.concatenate([sa, ss])
    for k in [24, 24 + 49]:  # the source block's absorption and scattering
        pp, pm = p0.copy(), p0.copy()
        pp[k] += h
        pm[k] -= h
        Jp = gpu_J_grad(K, s, blk, pp[:49], pp[49:], q, tgt, u0, dt, nsteps, nsteps)[0]
        Jm = gpu_J_grad(K, s, blk, pm[:49], pm[49:], q, tgt, u0, dt, nsteps, nsteps)[0]
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * scale, (k, fd, g[k], scale)


@pytest.mark.skipif(os.environ.get("KITRT_EVIDENCE_FD") != "1",
                    reason="evidence run (about 3 minutes): set KITRT_EVIDENCE_FD=1")
def test_adjoint_full_size_all_98_coefficients_fd(K):
    """The adjoint configuration at full size (~60k triangles, M_3, order 10, 400 steps,
    checkpoints every 16) against central differences (h = 1e-6) of every one of the 98
    coefficients: |FD - adjoint| <= 1e-6 max |gradient| (196 forward runs)."""
    N, order, nsteps, h = 3, 10, 400, 1e-6
    m, mesh, blk, sa, ss, q, tgt, u0 = blocks_problem(K, 173, N, order)
    s = K.MNSolver(mesh, N, order, bc="vacuum", tau=1e-12)
    dt = 0.4 * mesh.geometry()["min_inradius"]
    J, gsa, gss = gpu_J_grad(K, s, blk, sa, ss, q, tgt, u0, dt, nsteps, 16)
    g = np.concatenate([gsa, gss])
    scale = np.abs(g).max()
    p0 = np.concatenate([sa, ss])
    fd = np.zeros_like(g)
    for k in range(g.size):
        pp, pm = p0.copy(), p0.copy()
        pp[k] += h
        pm[k] -= h
        Jp = gpu_J_grad(K, s, blk, pp[:49], pp[49:], q, tgt, u0, dt, nsteps, nsteps)[0]
        Jm = gpu_J_grad(K, s, blk, pm[:49], pm[49:], q, tgt, u0, dt, nsteps, nsteps)[0]
        fd[k] = (Jp - Jm) / (2 * h)
    err = np.abs(fd - g) / scale
    print("full-size adjoint vs FD over 98 coefficients: max", err.max(), "median", np.median(err),
          "J", J)
    assert err.max() <= 1e-6
