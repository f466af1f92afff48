"""The allocation-free closure entry point (kitrt_closure_noalloc) gives the same answers as
kitrt_closure.

kitrt_closure_noalloc exists for callers that cannot let the library allocate device memory at
call time: a framework whose pool allocator already owns the free device memory, or a service
that must not grow its footprint after start-up. It keeps its Newton state in a fixed static
device array that every call shares, so this test calls it twice in a row on different batches
and checks both answers against the ordinary entry point, and checks that an oversized batch is
refused before any memory is touched. This file is collected last on purpose, and it does not
rely on anything the other tests leave behind, so it passes alone in a fresh process as well."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_08417_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _realizable_moments(T, count, seed):
    mu, phi, w, ox, oy = O.quadrature(T.order)
    dirs = np.stack([ox, oy, mu], axis=1)
    c, k, wt = synth.vmf_mixtures(count, seed, kappa_hi=20.0)
    psi = synth.vmf_density(dirs, c, k, wt)
    scale = np.exp(np.random.default_rng(seed).uniform(-3, 2, size=count))
    return (psi * scale[:, None]) @ (T.w[:, None] * T.M)


def test_noalloc_closure_matches_closure_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_08417_gb300 import build, kitrt
    build.build()
    N, order = 3, 10
    m = synth.jittered_mesh(30, 0.0, 1.0, seed=6)
    mesh = kitrt.Mesh(m.xy, m.tri)
    C = mesh.ncells
    s = kitrt.MNSolver(mesh, N, order)
    T = O.Tables(N, order)
    for call, seed in enumerate([21, 22]):
        u = torch.from_numpy(_realizable_moments(T, C, seed)).cuda()
        a_ref = s.isotropic_alpha(u)
        st_ref = torch.zeros(C, dtype=torch.int32, device="cuda")
        rc_ref = s.closure(u, a_ref, st_ref, check=False)
        a_na = s.isotropic_alpha(u)
        st_na = torch.full((C,), -1, dtype=torch.int32, device="cuda")
        rc_na = s.closure_noalloc(u, a_na, st_na, check=False)
        torch.cuda.synchronize()
        assert rc_na == rc_ref, (call, rc_na, rc_ref)
        assert torch.equal(st_na, st_ref), call
        ok = (st_ref == 0).cpu().numpy()
        assert ok.mean() > 0.95
        # both calls converge to the unique minimiser; their answers may differ by rounding
        # amplified by the conditioning of the dual Hessian (the bound the closure parity tests
        # use: 1e-9 ||u|| / lambda_min(H) + 1e-12 ||alpha||)
        a1, a2 = a_na.cpu().numpy(), a_ref.cpu().numpy()
        un = u.cpu().numpy()
        for i in np.flatnonzero(ok):
            e = T.w * np.exp(T.M @ a2[i])
            lmin = np.linalg.eigvalsh(T.M.T @ (e[:, None] * T.M))[0]
            bound = 1e-9 * np.linalg.norm(un[i]) / lmin + 1e-12 * np.linalg.norm(a2[i])
            assert np.linalg.norm(a1[i] - a2[i]) <= bound, (call, i)


def test_noalloc_rejects_batches_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_08417_gb300 import build, kitrt
    build.build()
    m = synth.jittered_mesh(5, 0.0, 1.0, seed=0)
    mesh = kitrt.Mesh(m.xy, m.tri)
    s = kitrt.MNSolver(mesh, 3, 10)
    n = s.n
    # 8 MiB of scratch, 16 arrays padded to 256 bytes: a batch of 20,000 M_3 cells needs more
    per_cell = 8 * (3 * n + 4 + n * (n + 1) // 2) + 28
    too_many = 20000
    assert too_many * per_cell > 8 * 2 ** 20
    u = torch.zeros((1, n), dtype=torch.float64, device="cuda")
    a = torch.zeros((1, n), dtype=torch.float64, device="cuda")
    rc = kitrt._lib().kitrt_closure_noalloc(s.handle, kitrt._dev(u), kitrt._dev(a), None,
                                            too_many, kitrt._stream())
    assert rc == 9  # KITRT_ESCRATCH, refused before any access to u or alpha
    assert kitrt._lib().kitrt_status_string(9).startswith(b"batch exceeds")
