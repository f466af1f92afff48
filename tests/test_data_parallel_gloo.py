"""Data-parallel training of the learned closure's network over ranks (two gloo ranks on the CPU):
each rank takes its share of every batch (learned.train's split, the same permutation on every
rank), computes the gradient of its share, and the ranks average the gradients with one
all-reduce (learned.allreduce_mean) before the Adam step. The arithmetic on the CPU ranks is the
oracle's MLP; the averaged gradient must equal the whole batch's gradient, and the ranks' Adam
steps must stay identical."""
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


def _data(din=9, dout=9, B=64, hidden=16, seed=5):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(B, din))
    Y = rng.normal(size=(B, dout))
    P = din * hidden + hidden + 2 * (hidden * hidden + hidden) + hidden * dout + dout
    params = rng.normal(scale=0.3, size=P)
    return X, Y, params, din, hidden, dout


def _rank(rank, world, port, steps, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import oracle as O
    from paper_2205_08417_gb300.learned import allreduce_mean
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, Y, p, din, H, dout = _data()
        m, v = np.zeros_like(p), np.zeros_like(p)
        grads = []
        for t in range(1, steps + 1):
            idx = np.arange(X.shape[0])[rank::world]  # this rank's share of the batch
            _, g = O.mlp_loss_grad(p, X[idx], Y[idx], din, H, dout)
            gt = torch.from_numpy(g)
            allreduce_mean(gt, dist)
            g = gt.numpy()
            grads.append(g.copy())
            O.adam(p, g, m, v, t, lr=1e-2)
        out.put((rank, grads, p.copy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_average_to_the_whole_batch_gradient():
    import oracle as O
    steps = 3
    X, Y, p, din, H, dout = _data()
    m, v = np.zeros_like(p), np.zeros_like(p)
    ref_grads = []
    for t in range(1, steps + 1):
        _, g = O.mlp_loss_grad(p, X, Y, din, H, dout)
        ref_grads.append(g.copy())
        O.adam(p, g, m, v, t, lr=1e-2)
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, steps, out)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted([out.get(timeout=300) for _ in procs], key=lambda x: x[0])
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    (_, g0, p0), (_, g1, p1) = res
    assert np.array_equal(p0, p1)  # identical steps on both ranks
    for a, b, r in zip(g0, g1, ref_grads):
        assert np.array_equal(a, b)
        assert np.abs(a - r).max() <= 1e-13 * np.abs(r).max()
    np.testing.assert_allclose(p0, p, rtol=0, atol=1e-12)
