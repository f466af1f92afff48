"""The step split over ranks on one GPU: two partitions of the line-source mesh (Morton ranges
plus halo layers) stepped by two solvers on their local meshes, their halo rows of u and alpha
refreshed before every step through the library's row kernels (kitrt_gather_rows /
kitrt_scatter_rows; the transport between the emulated ranks is a device copy, the send and
receive lists are partition.py's). The owned cells must match one solver on the whole mesh:
1e-13 relative L2 in FP64 (the sweeps' split of the quadrature into parts depends on how many
cells a solver lists, so the two runs round differently) and 1e-6 on u_0 in the mixed mode. The
ranks' kernels never wait on each other: they run one after the other."""
import numpy as np
import pytest

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


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


@pytest.mark.parametrize("mode,order,tol", [("fp64", 1, 1e-13), ("fp64", 2, 1e-13),
                                            ("mixed_tf32", 1, 1e-6)])
def test_two_partitions_on_one_gpu_match_the_whole_mesh(K, mode, order, tol):
    from paper_2205_08417_gb300.partition import Partition
    m = synth.jittered_mesh(40, -1.5, 1.5, seed=1)
    mesh = K.Mesh(m.xy, m.tri)
    g = mesh.geometry()
    C = mesh.ncells
    N, qorder = 2, 10
    tau = 1e-10 if mode == "fp64" else 1e-8
    s = K.MNSolver(mesh, N, qorder, mode=mode, tau=tau, order=order)
    u0 = synth.isotropic_moments(synth.line_source_density(g["centroid"], width=0.1), s.n)
    rng = np.random.default_rng(5)
    sa, ss, q = rng.uniform(0, 0.3, C), rng.uniform(0.5, 1.0, C), np.zeros(C)
    dt = 0.3 * g["min_inradius"]
    nsteps = 8
    ud = dev(u0)
    ad = s.isotropic_alpha(ud)
    s.step(ud, ad, dev(sa), dev(ss), dev(q), dt=dt, nsteps=nsteps)
    u_ref = ud.cpu().numpy()

    parts = [Partition(m.xy, m.tri, g["nbr"], r, 2, layers=1 if order == 1 else 4) for r in range(2)]
    ranks = []
    for p in parts:
        lm = K.Mesh(p.xy, p.tri)
        ls = K.MNSolver(lm, N, qorder, mode=mode, tau=tau, order=order)
        lu = dev(p.local(u0))
        ranks.append(dict(p=p, mesh=lm, s=ls, u=lu, a=ls.isotropic_alpha(lu),
                          sa=dev(p.local(sa)), ss=dev(p.local(ss)), q=dev(p.local(q)),
                          send={r: dev(v) for r, v in p.send.items()},
                          recv={r: dev(v) for r, v in p.recv.items()}))
    exchanged = 0
    for _ in range(nsteps):
        for key in ("u", "a"):
            for me in ranks:
                for r, ridx in me["recv"].items():
                    src = ranks[r]
                    buf = torch.empty((ridx.numel(), me[key].shape[1]), dtype=torch.float64, device="cuda")
                    K.gather_rows(src[key], src["send"][me["p"].rank], buf)
                    K.scatter_rows(buf, ridx, me[key])
                    exchanged += ridx.numel()
        for me in ranks:
            me["s"].step(me["u"], me["a"], me["sa"], me["ss"], me["q"], dt=dt, nsteps=1)
    torch.cuda.synchronize()
    assert exchanged > 0
    u_part = np.zeros_like(u_ref)
    for me in ranks:
        p = me["p"]
        u_part[p.lo:p.hi] = me["u"].cpu().numpy()[:p.n_owned]
    if mode == "fp64":
        err = float(np.linalg.norm(u_part - u_ref) / np.linalg.norm(u_ref))
    else:
        err = float(np.linalg.norm(u_part[:, 0] - u_ref[:, 0]) / np.linalg.norm(u_ref[:, 0]))
    print(mode, "order", order, "partitioned vs whole mesh", err)
    assert err <= tol


def test_row_kernels_gather_and_scatter(K):
    rng = np.random.default_rng(0)
    src = rng.normal(size=(50, 7))
    idx = rng.permutation(50)[:13].astype(np.int32)
    out = torch.empty((13, 7), dtype=torch.float64, device="cuda")
    K.gather_rows(dev(src), dev(idx), out)
    np.testing.assert_array_equal(out.cpu().numpy(), src[idx])
    dst = torch.zeros((50, 7), dtype=torch.float64, device="cuda")
    K.scatter_rows(out, dev(idx), dst)
    ref = np.zeros((50, 7))
    ref[idx] = src[idx]
    np.testing.assert_array_equal(dst.cpu().numpy(), ref)
    # scatter-add (the adjoint's reverse halo): rows idx gain the buffer's rows, the others keep theirs
    base = rng.normal(size=(50, 7))
    acc = dev(base)
    K.scatter_add_rows(out, dev(idx), acc)
    ref = base.copy()
    ref[idx] += src[idx]
    np.testing.assert_array_equal(acc.cpu().numpy(), ref)
    K.scatter_add_rows(out[:0], dev(idx[:0]), acc)  # an empty batch changes nothing
    np.testing.assert_array_equal(acc.cpu().numpy(), ref)
