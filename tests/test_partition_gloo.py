"""The step split over ranks (Sec. 6: cells split over parallel workers): two gloo ranks on the
CPU, each owning a Morton range of the cells plus halo layers, exchange their halo rows of u and
alpha before every step and step their local meshes; their owned cells must equal the single-rank
result bit for bit (first order with one halo layer, the second-order Heun step with four). The
arithmetic on the CPU ranks is the oracle's; the partition, the local meshes, the send and
receive lists and the exchange are the library's (partition.py), which the GPU ranks drive with
the row kernels and NCCL."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    import oracle as O
    from paper_2205_08417_gb300 import synth
    m = synth.jittered_mesh(14, -1.5, 1.5, seed=7)
    G = O.Geometry(m.xy, m.tri)
    T = O.Tables(2, 6)
    u0 = synth.isotropic_moments(synth.line_source_density(G.cen, width=0.3), T.n)
    C = G.C
    rng = np.random.default_rng(3)
    sa, ss, q = rng.uniform(0, 0.5, C), rng.uniform(0.2, 1.0, C), np.zeros(C)
    return m, G, T, u0, sa, ss, q


def _run(O, T, G, u, a, sa, ss, q, dt, order):
    if order == 1:
        nf, _ = O.mn_run(T, G, u, a, sa, ss, q, dt, 1)
    else:
        nf, _ = O.mn_run2(T, G, u, a, sa, ss, q, dt, 1)
    assert nf == 0


def _rank(rank, world, port, order, nsteps, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import oracle as O
    from paper_2205_08417_gb300.partition import Partition
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m, G, T, u0, sa, ss, q = _problem()
        dt = G.cfl_dt(0.3)
        part = Partition(m.xy, m.tri, G.nbr, rank, world, layers=1 if order == 1 else 4)
        Gl = O.Geometry(part.xy, part.tri)
        u = part.local(u0)
        a = O.isotropic_alpha(T, u)
        sal, ssl, ql = part.local(sa), part.local(ss), part.local(q)
        n = T.n
        pack = lambda uu, idx: torch.from_numpy(np.ascontiguousarray(uu[idx]))
        def unpack(buf, idx, uu):
            uu[idx] = buf.numpy()
        empty = lambda k: torch.empty((k, n), dtype=torch.float64)
        for _ in range(nsteps):
            part.exchange(u, pack, unpack, empty, dist)
            part.exchange(a, pack, unpack, empty, dist)
            _run(O, T, Gl, u, a, sal, ssl, ql, dt, order)
        out.put((rank, part.lo, part.hi, u[:part.n_owned].copy(),
                 {r: v.size for r, v in part.send.items()}))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("order", [1, 2])
def test_two_ranks_equal_the_single_rank_step_bitwise(order):
    import oracle as O
    nsteps = 6
    m, G, T, u0, sa, ss, q = _problem()
    dt = G.cfl_dt(0.3)
    u_ref = u0.copy()
    a_ref = O.isotropic_alpha(T, u_ref)
    for _ in range(nsteps):
        _run(O, T, G, u_ref, a_ref, sa, ss, q, dt, order)
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, order, nsteps, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    covered = np.zeros(G.C, dtype=bool)
    for rank, lo, hi, uo, sends in res:
        assert np.array_equal(uo, u_ref[lo:hi]), (order, rank)
        assert sum(sends.values()) > 0  # ranks did exchange rows
        covered[lo:hi] = True
    assert covered.all()


def test_partition_bookkeeping():
    """Owned ranges tile the mesh; each rank's receive list from r is r's send list to it (same
    global cells in the same order); halo layers grow outwards from the owned range."""
    from paper_2205_08417_gb300.partition import Partition, halo_cells
    m, G, T, u0, sa, ss, q = _problem()
    parts = [Partition(m.xy, m.tri, G.nbr, r, 3, layers=2) for r in range(3)]
    assert parts[0].lo == 0 and parts[-1].hi == G.C
    for a, b in zip(parts, parts[1:]):
        assert a.hi == b.lo
    for p in parts:
        for r, idx in p.recv.items():
            assert np.array_equal(p.cells[idx], parts[r].cells[parts[r].send[p.rank]])
        # every face neighbour of an owned cell is local
        nb = G.nbr[p.lo:p.hi].ravel()
        assert np.isin(nb[nb >= 0], p.cells).all()
    h1 = halo_cells(G.nbr, 0, 50, 1)
    h2 = halo_cells(G.nbr, 0, 50, 2)
    assert np.array_equal(h2[:h1.size], h1) and h2.size > h1.size


def _vjp_state():
    """A line-source state after a few oracle steps, its closure, and a seeded adjoint row set."""
    import oracle as O
    m, G, T, u0, sa, ss, q = _problem()
    dt = G.cfl_dt(0.3)
    u = u0.copy()
    a = O.isotropic_alpha(T, u)
    for _ in range(3):
        _run(O, T, G, u, a, sa, ss, q, dt, 1)
    st, _ = O.closure(T, u, a)
    assert (st == 0).all()
    lam = np.random.default_rng(11).normal(size=u.shape)
    return m, G, T, u, a, sa, ss, dt, lam


def _rank_vjp(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import oracle as O
    from paper_2205_08417_gb300.partition import Partition
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m, G, T, u, a, sa, ss, dt, lam = _vjp_state()
        part = Partition(m.xy, m.tri, G.nbr, rank, world, layers=1)
        Gl = O.Geometry(part.xy, part.tri)
        # the linearisation point on the local cells; adjoint rows of the owned cells only
        ul, al = part.local(u), part.local(a)
        laml = part.local(lam)
        laml[part.n_owned:] = 0.0
        v = O.step_vjp(T, Gl, ul, al, part.local(sa), part.local(ss), dt, laml)
        n = T.n
        pack = lambda vv, idx: torch.from_numpy(np.ascontiguousarray(vv[idx]))
        def unpack_add(buf, idx, vv):
            vv[idx] += buf.numpy()
        empty = lambda k: torch.empty((k, n), dtype=torch.float64)
        before = v[:part.n_owned].copy()
        part.reverse_exchange(v, pack, unpack_add, empty, dist)
        out.put((rank, part.lo, part.hi, v[:part.n_owned].copy(), before))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_adjoint_step_with_the_reverse_halo():
    """The transposed step split over two ranks: each applies the oracle's one-step transpose on
    its local mesh to its owned adjoint rows (zero on the halo) and sends the halo rows' results
    back to their owners, which add them (the reverse halo of the adjoint). The owned rows equal
    the single-rank transposed step to round-off (the additions come in another order)."""
    import oracle as O
    m, G, T, u, a, sa, ss, dt, lam = _vjp_state()
    ref = O.step_vjp(T, G, u, a, sa, ss, dt, lam)
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_vjp, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = np.zeros_like(ref)
    local_only = np.zeros_like(ref)
    for rank, lo, hi, vo, before in res:
        got[lo:hi] = vo
        local_only[lo:hi] = before
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    # without the reverse halo the cells next to the cut miss their neighbours' terms
    assert np.abs(local_only - ref).max() > 1e-3 * np.abs(ref).max()
