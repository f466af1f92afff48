"""Training of the learned entropy closure with the library's own kernels.

Data: realizable moment vectors of random positive angular densities (mixtures of 1-4 von
Mises-Fisher lobes on S^2, integrated with the solver's quadrature on the GPU) and their alphas
from the library's Newton closure; samples whose closure fails are dropped. Features are the
normalised moments u_{1..n-1}/u_0, targets alpha_{1..n-1} (both standardised; the scales travel
with the network). Training: mean-squared loss, Adam, minibatches, all on the GPU through the
kitrt MLP kernels. The result is attached to a KITRT_LEARNED solver with MNSolver.set_mlp.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import kitrt, synth


@dataclass
class TrainedMLP:
    params: object   # torch float32 [P] on the GPU
    norm: object     # torch float32 [4 (n-1)]: feature mean, feature scale, output mean, scale
    hidden: int
    losses: list
    samples: int


def training_data(solver: "kitrt.MNSolver", count: int, seed: int, kappa_hi: float = 50.0):
    """(u [m, n], alpha [m, n]) device FP64 for the m <= count samples whose closure succeeded.
    Closures run in chunks of the solver's mesh size."""
    import torch
    c, k, wt = synth.vmf_mixtures(count, seed, kappa_hi=kappa_hi)
    rng = np.random.default_rng(seed + 1)
    scale = np.exp(rng.uniform(-4.0, 3.0, size=count))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    u = solver.vmf_moments(dev(c), dev(k), dev(wt * scale[:, None]))
    m0 = 1.0 / math.sqrt(4.0 * math.pi)
    alpha = torch.zeros_like(u)
    alpha[:, 0] = torch.log(u[:, 0] / (4.0 * math.pi * m0)) / m0
    status = torch.zeros(count, dtype=torch.int32, device=u.device)
    cap = solver.mesh.ncells
    for s0 in range(0, count, cap):
        s1 = min(count, s0 + cap)
        solver.closure_batch(u[s0:s1], alpha[s0:s1], status[s0:s1], check=False)
    ok = status == 0
    return u[ok].contiguous(), alpha[ok].contiguous()


def allreduce_mean(t, dist):
    """Data-parallel training over ranks: the mean over the ranks of a gradient (or loss) tensor,
    in place. Every rank computes the gradient of its equal share of a batch; the loss being a
    mean over samples, the mean of the shares' gradients is the whole batch's gradient, so the
    ranks take identical Adam steps from identical parameters."""
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    t /= dist.get_world_size()
    return t


def train(u, alpha, hidden: int = 64, epochs: int = 30, batch: int = 1024, lr: float = 3e-3,
          seed: int = 0, log_every: int = 0, dist=None) -> TrainedMLP:
    import torch
    n = u.shape[1]
    din = dout = n - 1
    x = (u[:, 1:] / u[:, :1]).float()
    y = alpha[:, 1:].float()
    xm, xs = x.mean(0), x.std(0).clamp_min(1e-6)
    ym, ys = y.mean(0), y.std(0).clamp_min(1e-6)
    X = ((x - xm) / xs).contiguous()
    Y = ((y - ym) / ys).contiguous()
    P = kitrt.mlp_param_count(din, hidden, dout)
    g = torch.Generator(device="cpu").manual_seed(seed)
    params = torch.empty(P)
    off = 0
    for fan_in, fan_out in [(din, hidden), (hidden, hidden), (hidden, hidden), (hidden, dout)]:
        bound = math.sqrt(6.0 / (fan_in + fan_out))
        params[off:off + fan_in * fan_out] = (torch.rand(fan_in * fan_out, generator=g) * 2 - 1) * bound
        off += fan_in * fan_out
        params[off:off + fan_out] = 0.0
        off += fan_out
    params = params.cuda()
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    work = torch.empty(kitrt._lib().kitrt_mlp_work_floats(batch, hidden, dout), dtype=torch.float32,
                       device=params.device)
    nb = X.shape[0] // batch
    perm_gen = torch.Generator(device="cpu").manual_seed(seed + 1)
    losses, t = [], 0
    for ep in range(epochs):
        perm = torch.randperm(X.shape[0], generator=perm_gen).cuda()
        lr_ep = lr * 0.5 * (1 + math.cos(math.pi * ep / epochs))
        ep_loss = torch.zeros((), device=params.device)
        for b in range(nb):
            idx = perm[b * batch:(b + 1) * batch]
            if dist is not None:  # this rank's share of the batch (same permutation on every rank)
                idx = idx[dist.get_rank()::dist.get_world_size()]
            xb, yb = X[idx].contiguous(), Y[idx].contiguous()
            loss, grad = kitrt.mlp_loss_grad(params, xb, yb, din, hidden, dout, work=work)
            if dist is not None:
                allreduce_mean(grad, dist)
                allreduce_mean(loss, dist)
            t += 1
            kitrt.mlp_adam(params, grad, m, v, t, lr=lr_ep)
            ep_loss += loss[0]
        losses.append(float(ep_loss) / max(1, nb))
        if log_every and (ep + 1) % log_every == 0:
            print(f"epoch {ep + 1}: loss {losses[-1]:.3e}")
    norm = torch.cat([xm, xs, ym, ys]).float().contiguous()
    return TrainedMLP(params=params, norm=norm, hidden=hidden, losses=losses, samples=int(X.shape[0]))
