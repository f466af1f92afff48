#!/usr/bin/env python
"""Benchmark of the M_N step on one GB300 (or N independent replicas under torchrun).

Workload: M_3 line source on the square [-1.5,1.5]^2, seeded jittered-point Delaunay mesh of
224^2 points (~100k triangles), 10 moments, order-20 product quadrature (800 points, 400 after
folding), Gaussian initial density of width 0.03 plus a 1e-4 floor, sigma_s = 1, sigma_a = 0,
CFL 0.4, Neumann walls, Newton tolerance 1e-10.

One step = one explicit M_N time step of the whole mesh: entropy closure of every cell (Newton),
kinetic upwind flux, source and Euler update. `value` times K steps with the state resident in
device memory; `e2e` times K steps through the same C ABI call with the state copied from pinned
host memory before and back after every step.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "M_N cell-updates/s & closures/s, mixed vs FP64 on one GB300 at stated error"
UNIT = "cell-updates/s"
WORKLOAD = "m3_line_source_100k"


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank timings over all ranks (the job takes as long as its
    slowest replica)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def replica_throughput(cells, steps, max_ms, world):
    """Whole-job cell-updates/s of `world` independent replicas, each advancing `cells` cells by
    `steps` steps, timed by the slowest replica."""
    return world * cells * steps / (max_ms / 1e3)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", default="mixed_tf32", help="headline closure mode")
    ap.add_argument("--compare", default="fp64,mixed_bf16,learned", help="comma list of extra modes to time")
    ap.add_argument("--train-samples", type=int, default=2_000_000,
                    help="training moment vectors of the learned closure")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="synth.WORKLOADS key (the default is the benchmarked configuration)")
    ap.add_argument("--t-start", type=float, default=0.25,
                    help="simulated time reached by untimed set-up steps before warm-up")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sn", action="store_true", help="skip the S_N step measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the measurements beside the headline (like-for-like FP64, second "
                         "order, regularized, adjoint, M_5)")
    ap.add_argument("--tau", type=float, default=1e-10, help="Newton tolerance of the FP64 mode")
    ap.add_argument("--tau-mixed", type=float, default=1e-8,
                    help="Newton tolerance of the mixed modes (matched to their FP32 ansatz)")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------------
# workload
# ------------------------------------------------------------------------------------------------
def make_workload(name=WORKLOAD):
    from paper_2205_08417_gb300 import synth
    spec = synth.WORKLOADS[name]
    m = synth.jittered_mesh(spec["k"], spec["lo"], spec["hi"], spec["seed"])
    cen = m.centroids()
    n = (spec["N"] + 1) * (spec["N"] + 2) // 2
    u0 = synth.isotropic_moments(synth.line_source_density(cen), n)
    C = m.ncells
    sa, ss = np.zeros(C), np.ones(C)
    if spec.get("blocks"):
        # large M_5 configuration: the line-source start in a 7x7 block medium with seeded
        # sigma_a in [0,10] and sigma_s in [0,1] (the block structure of the adjoint problem)
        blk, sab, ssb = synth.block_coefficients(cen, spec["lo"], spec["hi"], 7, spec["seed"])
        sa, ss = sab[blk], ssb[blk]
    return dict(mesh=m, cen=cen, u0=u0, N=spec["N"], order=spec["order"], n=n, C=C,
                sa=sa, ss=ss, q=np.zeros(C))


def oracle_sample_cells(W, size):
    """A Morton-contiguous block of `size` cells centred on the cell nearest the pulse (the whole
    mesh when size is None or not smaller than the mesh)."""
    C = W["C"]
    if size is None or size >= C:
        return np.arange(C)
    c0 = int(np.argmin((W["cen"] ** 2).sum(axis=1)))
    lo = max(0, min(C - size, c0 - size // 2))
    return np.arange(lo, lo + size)


# ------------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------------
# oracle legs (CPU)
# ------------------------------------------------------------------------------------------------
def oracle_timing(W, steps: int, warmup: int, sample_cells: int):
    """Time the CPU oracle on a bounded sample: `steps` oracle steps on a Morton-contiguous
    submesh of `sample_cells` cells around the pulse (or the whole mesh), after `warmup` untimed
    steps from the initial state. The oracle evaluates the dual at least once for every cell in
    every step, so its cost per cell barely depends on how far the pulse has spread."""
    import oracle as O
    cells = oracle_sample_cells(W, sample_cells)
    m = W["mesh"]
    G = O.Geometry(m.xy, m.tri[cells])
    T = O.Tables(W["N"], W["order"])
    u = np.ascontiguousarray(W["u0"][cells])
    a = O.isotropic_alpha(T, u)
    dt = 0.4 * float(np.min(2 * G.area / G.perim))
    sa, ss, q = W["sa"][cells], W["ss"][cells], W["q"][cells]
    if warmup:
        O.mn_run(T, G, u, a, sa, ss, q, dt, warmup)
    t0 = time.perf_counter()
    nf, _ = O.mn_run(T, G, u, a, sa, ss, q, dt, steps)
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return len(cells) * steps / el, cores, el, len(cells)


# ------------------------------------------------------------------------------------------------
# GPU leg
# ------------------------------------------------------------------------------------------------
def fp64_peak_tflops(torch):
    """Measured FP64 throughput of cuBLAS DGEMM (4096^3, best of 5) on this GPU."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e9
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return 2.0 * n ** 3 / best / 1e12


def train_network(K, torch, W, samples, seed=4):
    """Learned closure for this workload's basis: training data from vMF mixtures closed by the
    FP64 Newton solver, trained with the library's MLP kernels (untimed set-up)."""
    from paper_2205_08417_gb300 import learned
    mesh = K.Mesh(W["mesh"].xy, W["mesh"].tri)
    s = K.MNSolver(mesh, W["N"], W["order"], mode="fp64", tau=1e-12)
    t0 = time.perf_counter()
    u, a = learned.training_data(s, samples, seed=seed)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    net = learned.train(u, a, batch=4096 if samples > 500_000 else 1024, epochs=20 if samples > 500_000 else 30)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    net.info = {"samples": net.samples, "requested": samples, "data_s": t1 - t0, "train_s": t2 - t1,
                "final_loss": net.losses[-1], "first_loss": net.losses[0]}
    return net


def log(msg):
    """Progress to stderr (stdout carries the one JSON line)."""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def run_mode(K, torch, W, mode, steps, warmup, t_start, tau, e2e=True, net=None, density=None,
             cfl=0.4, **opts):
    mesh = K.Mesh(W["mesh"].xy, W["mesh"].tri)
    s = K.MNSolver(mesh, W["N"], W["order"], mode=mode, tau=tau, **opts)
    if net is not None:
        s.set_mlp(net.params, net.norm)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    u0 = W["u0"] if density is None else W["u0"] * density[:, None]
    u = d(u0)
    alpha = s.isotropic_alpha(u)
    sa, ss, q = d(W["sa"]), d(W["ss"]), d(W["q"])
    geo = mesh.geometry()
    dt = cfl * geo["min_inradius"]
    if density is not None:
        # the transformed CSD equation transports psi / rho: speed 1 / rho
        s.set_density(d(density))
        dt *= float(density.min())
    setup = int(round(t_start / dt))
    before = 0
    t0 = time.perf_counter()
    if setup:
        before += s.step(u, alpha, sa, ss, q, dt=dt, nsteps=setup, stats=True)[1]["launches"]
    before += s.step(u, alpha, sa, ss, q, dt=dt, nsteps=warmup, stats=True)[1]["launches"]
    torch.cuda.synchronize()
    log(f"mode {mode}: {setup} set-up + {warmup} warm-up steps in {time.perf_counter() - t0:.1f} s")
    s.profile(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    rc, st = s.step(u, alpha, sa, ss, q, dt=dt, nsteps=steps, stats=True)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    prof = s.profile_read()
    s.profile(False)
    out = dict(mode=mode, ms=ms, stats=st, prof=prof, dt=dt, setup=setup, launches_before=before,
               u=u.cpu().numpy(),
               alpha=alpha.cpu().numpy(), nbr=geo["nbr"], solver=s, mesh=mesh)
    if e2e:
        C, n = W["C"], W["n"]
        host = torch.from_numpy(out["u"].copy()).pin_memory()
        ud = torch.empty_like(u)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            ud.copy_(host, non_blocking=True)
            s.step(ud, alpha, sa, ss, q, dt=dt, nsteps=1)
            host.copy_(ud, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        out["e2e_ms"] = e0.elapsed_time(e1)
        out["e2e_bytes"] = C * n * 8
    return out


# DRAM bytes (read + write) per launch of the S_N step from one ncu capture of the bench's own
# launches (profiles/sn_tile_kernel_m3_line_source_100k.md); other workloads have no capture.
SN_TRAFFIC = {("m3_line_source_100k", True): 286.9e6}


def run_sn(K, torch, W, steps, warmup, fp32, hbm_peak, workload):
    """S_N steps (the nodal system with isotropic scattering) on the same mesh, quadrature and
    line-source start: ordinates psi = Phi / (4 pi) at the folded points, [C x Q'] resident on the
    device, double-buffered. Roofline: algorithmic bytes per cell = own row read + written
    (2 Q' b) + cell data (neighbours 16 B, normals 48 B, area 8 B, sigma_a, sigma_s, q 24 B); the
    three upwind rows are other cells' rows and count once."""
    mesh = K.Mesh(W["mesh"].xy, W["mesh"].tri)
    s = K.MNSolver(mesh, W["N"], W["order"])
    C, Qf = W["C"], s.Qf
    phi = W["u0"][:, 0] * math.sqrt(4 * math.pi)
    dtype = torch.float32 if fp32 else torch.float64
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    psi = d(np.repeat((phi / (4 * math.pi))[:, None], Qf, axis=1)).to(dtype)
    work = torch.empty_like(psi)
    sa, ss, q = d(W["sa"]), d(W["ss"]), d(W["q"])
    dt = 0.4 * mesh.geometry()["min_inradius"]
    s.sn_step(psi, work, sa, ss, q, dt=dt, nsteps=max(warmup, 3))
    torch.cuda.synchronize()
    s.profile(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.sn_step(psi, work, sa, ss, q, dt=dt, nsteps=steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    pe = s.profile_read()["sn_step"]
    s.profile(False)
    b = 4 if fp32 else 8
    per_cell = 2 * Qf * b + 96
    launch_ms = pe["total_ms"] / pe["launches"]
    gbs = C * per_cell / (launch_ms / 1e3) / 1e9
    out = {"cell_updates_per_s": C * steps / (ms / 1e3), "ms_per_step": ms / steps,
           "dtype": "f32" if fp32 else "f64", "scattering": "isotropic",
           "roofline": {"kernel": "sn_step", "bound": "hbm", "achieved": gbs, "peak": hbm_peak,
                        "unit": "GB/s", "frac": gbs / hbm_peak,
                        "traffic": SN_TRAFFIC.get((workload, fp32)),
                        "bytes_per_cell": per_cell, "avg_launch_ms": launch_ms,
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}}
    if not fp32:
        # per ordinate: 3 face dots (2 flops each), 3 fluctuation terms (3 each), moment (2) and
        # scattering (2) and update (4 FP64 flops)
        flops = C * Qf * (6 + 9 + 2 + 2 + 4)
        out["fp64_tflops"] = flops / (launch_ms / 1e3) / 1e12
    return out


def flux_roofline(W, work_n, Qf, prof, hbm_peak, fp32=True):
    """HBM roofline of the flux kernel: algorithmic bytes per cell = the cell's own ansatz row
    (Q' b; the three upwind rows are other cells' rows and count once), u read and written
    (16 n), neighbours (16), normals and inverse area (28 FP32 / 56 FP64), sigma_a, sigma_s, q
    (24)."""
    pf = prof.get("flux_update")
    if not pf:
        return None
    b = 4 if fp32 else 8
    per_cell = Qf * b + 16 * work_n + 16 + (28 if fp32 else 56) + 24
    launch_ms = pf["total_ms"] / pf["launches"]
    gbs = W["C"] * per_cell / (launch_ms / 1e3) / 1e9
    return {"kernel": "flux_update", "bound": "hbm", "achieved": gbs, "peak": hbm_peak,
            "unit": "GB/s", "frac": gbs / hbm_peak, "bytes_per_cell": per_cell,
            "avg_launch_ms": launch_ms, "traffic": None,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}


def mode_line(W, r, steps):
    line = {"ms_per_step": r["ms"] / steps, "cell_updates_per_s": W["C"] * steps / (r["ms"] / 1e3),
            "evaluations_per_cell_step": r["stats"]["evaluations"] / (W["C"] * steps),
            "kernels_ms_per_step": {k: v["total_ms"] / steps for k, v in r["prof"].items()}}
    st = r["stats"]
    line["fp64_handovers_per_cell_step"] = st.get("handovers", 0) / (W["C"] * steps)
    if st.get("proposals"):
        line["network_proposals_per_cell_step"] = st["proposals"] / (W["C"] * steps)
        line["network_accept_rate"] = 1.0 - st["fallbacks"] / st["proposals"]
        line["fallbacks_per_cell_step"] = st["fallbacks"] / (W["C"] * steps)
    return line


def sweep_roofline(r, work, peak):
    key = "closure_eval_fp64" if r["mode"] == "fp64" else "closure_eval_mixed"
    pe = r["prof"].get(key)
    if not pe or pe["total_ms"] <= 0:
        return None
    t = pe["total_ms"] / 1e3
    out = {"kernel": key, "fp64_ops_per_cell_eval": work["sweep_fp64_ops"],
           "fp64_pipe_frac": pe["units"] * work["sweep_fp64_ops"] / t / 1e12 / (peak / 2.0),
           "cell_evals": pe["units"]}
    if work["tensor_flops"]:
        out["tensor_tflops"] = pe["units"] * work["tensor_flops"] / t / 1e12
    return out


def run_extras(K, torch, args, peak, hbm_peak, head_results):
    """Untimed-region measurements beside the headline (each timed the same way: CUDA events
    around K steps after warm-up): the like-for-like FP64 line, the second-order and regularized
    steps on the same workload, the adjoint configuration's gradient, and the large M_5
    configuration in every mode."""
    ex = {}
    W = make_workload(args.workload)
    steps = min(args.steps, 10)
    ref_u0 = head_results["fp64"]["u"][:, 0] if "fp64" in head_results else None

    def err(r):
        if ref_u0 is None:
            return None
        return float(np.linalg.norm(r["u"][:, 0] - ref_u0) / np.linalg.norm(ref_u0))

    # same step count as the headline FP64 run, so that both states are at the same time
    r = run_mode(K, torch, W, "fp64", args.steps, args.warmup, args.t_start, args.tau_mixed,
                 e2e=False)
    ex["d2_fp64_tau_like_mixed"] = dict(mode_line(W, r, args.steps), tau=args.tau_mixed,
                                        u0_rel_l2_vs_fp64=err(r))
    log(f"extra fp64 tau {args.tau_mixed}: {r['ms'] / args.steps:.3f} ms/step")
    for mode in ("mixed_tf32", "fp64"):
        r = run_mode(K, torch, W, mode, steps, args.warmup, args.t_start,
                     args.tau if mode == "fp64" else args.tau_mixed, e2e=False, order=2)
        ex[f"d2_second_order_{mode}"] = mode_line(W, r, steps)
        ex[f"d2_second_order_{mode}"]["u"] = r["u"]
        log(f"extra second order {mode}: {r['ms'] / steps:.3f} ms/step")
    a, b = ex["d2_second_order_mixed_tf32"].pop("u"), ex["d2_second_order_fp64"].pop("u")
    ex["d2_second_order_mixed_tf32"]["u0_rel_l2_vs_fp64"] = float(
        np.linalg.norm(a[:, 0] - b[:, 0]) / np.linalg.norm(b[:, 0]))
    r = run_mode(K, torch, W, "mixed_tf32", steps, args.warmup, args.t_start, args.tau_mixed,
                 e2e=False, reg_gamma=1e-3)
    ex["d2_regularized_mixed_tf32"] = dict(mode_line(W, r, steps), reg_gamma=1e-3, reg_keep_mass=1)
    log(f"extra regularized: {r['ms'] / steps:.3f} ms/step")

    # the transformed CSD equation (psi / rho transported) on the same mesh with a two-tissue
    # density (1 | 5, and a disc of 2.5): the line-source start scaled by rho, pseudo-time steps
    from paper_2205_08417_gb300 import synth
    rho = synth.two_tissue_density(W["cen"])
    csd = {}
    for mode, tau in (("mixed_tf32", args.tau_mixed), ("fp64", args.tau)):
        r = run_mode(K, torch, W, mode, steps, args.warmup, args.t_start, tau, e2e=False,
                     density=rho)
        csd[mode] = r
        ex[f"d2_csd_density_{mode}"] = dict(mode_line(W, r, steps), density="two_tissue 1|5, disc 2.5")
        log(f"extra CSD density {mode}: {r['ms'] / steps:.3f} ms/step")
    ex["d2_csd_density_mixed_tf32"]["u0_rel_l2_vs_fp64"] = float(
        np.linalg.norm(csd["mixed_tf32"]["u"][:, 0] - csd["fp64"]["u"][:, 0]) /
        np.linalg.norm(csd["fp64"]["u"][:, 0]))

    # the checkerboard of Sec. 7.2 as the paper runs it: M_3, second-order flux with Heun, CFL
    # 0.45, vacuum walls, 25,088 triangles, from the 1e-4 floor to pseudo-time 1
    Wc = make_workload("m3_checkerboard_25k")
    Wc["sa"], Wc["ss"], Wc["q"] = synth.checkerboard_medium(Wc["cen"])
    Wc["u0"] = np.zeros((Wc["C"], Wc["n"]))
    Wc["u0"][:, 0] = 1e-4 / math.sqrt(4 * math.pi)
    cb = {}
    for mode, tau in (("mixed_tf32", args.tau_mixed), ("fp64", args.tau)):
        r = run_mode(K, torch, Wc, mode, steps, args.warmup, 1.0, tau, e2e=False, cfl=0.45,
                     order=2, bc="vacuum")
        cb[mode] = r
        ex[f"checkerboard_m3_second_order_{mode}"] = dict(mode_line(Wc, r, steps), cells=Wc["C"],
                                                          cfl=0.45, t_start=1.0)
        log(f"extra checkerboard {mode}: {r['ms'] / steps:.3f} ms/step")
    ex["checkerboard_m3_second_order_mixed_tf32"]["u0_rel_l2_vs_fp64"] = float(
        np.linalg.norm(cb["mixed_tf32"]["u"][:, 0] - cb["fp64"]["u"][:, 0]) /
        np.linalg.norm(cb["fp64"]["u"][:, 0]))

    # adjoint configuration: 7x7 block medium on [0,7]^2, M_3, order 10, 400 steps, checkpoints
    # every 16, absorbed energy of the centre 3x3 blocks and its 98 gradients
    spec = synth.WORKLOADS["m3_blocks_60k"]
    m = synth.jittered_mesh(spec["k"], spec["lo"], spec["hi"], spec["seed"])
    cen = m.centroids()
    blk, sab, ssb = synth.block_coefficients(cen, 0.0, 7.0, 7, spec["seed"])
    bx, by = blk // 7, blk % 7
    tgt = ((bx >= 2) & (bx <= 4) & (by >= 2) & (by <= 4)).astype(np.uint8)
    q = np.where(blk == 24, 1.0, 0.0)
    n3 = (spec["N"] + 1) * (spec["N"] + 2) // 2
    u0 = np.zeros((m.ncells, n3))
    u0[:, 0] = 1e-4 / math.sqrt(4 * math.pi)
    mesh = K.Mesh(m.xy, m.tri)
    s = K.MNSolver(mesh, spec["N"], spec["order"], bc="vacuum", tau=1e-12)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    ud = d(u0)
    ad = s.isotropic_alpha(ud)
    args3 = (ud, ad, d(sab[blk]), d(ssb[blk]), d(q), d(blk.astype(np.int32)), 49, d(tgt),
             0.4 * mesh.geometry()["min_inradius"], 400, 16)
    s.adjoint(*args3)  # warm-up (allocates the checkpoint workspace)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, gsa, gss = s.adjoint(*args3)
    el = time.perf_counter() - t0
    ex["d3_adjoint"] = {"cells": m.ncells, "steps": 400, "ckpt_every": 16, "coefficients": 98,
                        "seconds_per_gradient": el, "J": J,
                        "cell_steps_per_s_forward_and_reverse": m.ncells * 400 / el}
    log(f"extra adjoint: {el:.3f} s per gradient")

    # large M_5 configuration: ~1M triangles, block medium, a few steps after t = 0.01 in each mode
    W5 = make_workload("m5_line_source_1m")
    net5 = train_network(K, torch, W5, 500_000)
    d5 = {"cells": W5["C"], "nmom": W5["n"], "quad_points": 2 * W5["order"] ** 2, "modes": {}}
    res5 = {}
    for mode, tau in (("mixed_tf32", args.tau_mixed), ("fp64", args.tau), ("learned", args.tau_mixed)):
        r = run_mode(K, torch, W5, mode, 5, 2, 0.01, tau, e2e=False,
                     net=net5 if mode == "learned" else None)
        res5[mode] = r
        line = mode_line(W5, r, 5)
        line["sweep"] = sweep_roofline(r, r["solver"].work(), peak)
        line["flux"] = flux_roofline(W5, W5["n"], W5["order"] ** 2, r["prof"], hbm_peak,
                                     fp32=mode != "fp64")
        d5["modes"][mode] = line
        log(f"extra M_5 {mode}: {r['ms'] / 5:.1f} ms/step")
    ref5 = res5["fp64"]["u"][:, 0]
    for mode in ("mixed_tf32", "learned"):
        d5["modes"][mode]["u0_rel_l2_vs_fp64"] = float(
            np.linalg.norm(res5[mode]["u"][:, 0] - ref5) / np.linalg.norm(ref5))
    d5["learned_training"] = net5.info
    ex["d5_m5_blocks_1m"] = d5
    return ex


def hbm_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # fallback figure of an earlier GB300 measurement


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        # the reference arm is the CPU oracle (rank 0 only)
        if rank != 0:
            return
        W = make_workload(args.workload)
        import oracle as O
        O.build()
        cps, cores, el, ncells = oracle_timing(W, args.steps, args.warmup,
                                               None if W["C"] <= 200_000 else 20_000)
        line = {"impl": "reference", "metric": METRIC, "value": cps, "unit": UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "mesh_cells": W["C"], "nmom": W["n"],
                           "quad_points": 2 * W["order"] ** 2, "mode": "oracle_fp64"},
                "cpu_baseline": {"value": cps, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"{args.steps} oracle steps after {args.warmup} "
                                           f"untimed on {ncells} cells of the mesh, OpenMP "
                                           f"over cells"},
                "e2e": {"value": cps, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2205_08417_gb300 import build, kitrt as K
    build.build()
    W = make_workload(args.workload)

    modes = [args.mode] + [m for m in args.compare.split(",") if m and m not in (args.mode, "none")]
    peak = fp64_peak_tflops(torch)
    results = {}
    clocks = None
    log(f"workload {args.workload}: {W['C']} cells, modes {modes}")
    net = train_network(K, torch, W, args.train_samples) if "learned" in modes else None
    if net is not None:
        log(f"learned closure trained: {net.info}")
    for mode in modes:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        cs = ClockSampler(local) if mode == args.mode else None
        tau = args.tau if mode == "fp64" else args.tau_mixed
        try:
            r = run_mode(K, torch, W, mode, args.steps, args.warmup, args.t_start, tau,
                         e2e=not args.no_e2e, net=net if mode == "learned" else None)
        except K.KitrtError as exc:
            print(f"bench: mode {mode} (tau {tau}) failed: {exc}", file=sys.stderr, flush=True)
            raise
        r["tau"] = tau
        log(f"mode {mode}: {r['ms'] / args.steps:.3f} ms/step, stats {r['stats']}")
        if cs is not None:
            clocks = cs.stop()
        results[mode] = r
    sn = None
    if not args.no_sn:
        hp = hbm_peak_gbs()
        sn = {"sn_fp32": run_sn(K, torch, W, args.steps, args.warmup, True, hp, args.workload),
              "sn_fp64": run_sn(K, torch, W, args.steps, args.warmup, False, hp, args.workload)}
    extras = None
    if not args.no_extras and world == 1:
        extras = run_extras(K, torch, args, peak, hbm_peak_gbs(), results)
    head = results[args.mode]
    if world > 1:
        ms, e2e_ms = max_over_ranks([head["ms"], head.get("e2e_ms", float("nan"))], "cuda")
    else:
        ms, e2e_ms = head["ms"], head.get("e2e_ms", float("nan"))
    C = W["C"]
    value = replica_throughput(C, args.steps, ms, world)
    e2e_value = replica_throughput(C, args.steps, e2e_ms, world)

    n, Qf = W["n"], W["order"] ** 2  # folded points Q' = Q/2 = order^2
    work = head["solver"].work()
    fl = work["sweep_fp64_flops"]
    ops = work["sweep_fp64_ops"]
    ekey = "closure_eval_fp64" if args.mode == "fp64" else "closure_eval_mixed"
    pe = head["prof"][ekey]
    sweep_s = pe["total_ms"] / 1e3
    # the sweep is bound by the FP64 pipe: every FP64 instruction (FMA, add, multiply, and the
    # eight of each table-driven exp) takes one issue slot of it; the pipe's sustained rate is the
    # measured DGEMM rate over 2 flops per FMA
    achieved = pe["units"] * ops / sweep_s / 1e12
    peak_ops = peak / 2.0
    closure_ms = sum(head["prof"][k]["total_ms"] for k in head["prof"] if k.startswith("closure"))
    closures_per_s = C * args.steps / (closure_ms / 1e3)

    errors = {}
    if "fp64" in results:
        ref = results["fp64"]["u"][:, 0]
        for mname, r in results.items():
            if mname != "fp64":
                errors[f"{mname}_vs_fp64_u0_rel_l2"] = float(
                    np.linalg.norm(r["u"][:, 0] - ref) / np.linalg.norm(ref))

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        import oracle as O
        O.build()
        sample = None if W["C"] <= 200_000 else 20_000
        cps, cores, el, ncells = oracle_timing(W, 3, 1, sample)
        where = f"the full {ncells}-cell mesh" if sample is None else \
            f"a {ncells}-cell Morton-contiguous submesh around the pulse"
        cpu = {"value": cps, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"3 oracle steps after 1 untimed on {where}, OpenMP over cells ({el:.1f} s)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.mode == "fp64" else "f64+tf32",
        "data": "synthetic",
        "config": {"workload": args.workload, "mesh_cells": C, "nmom": n,
                   "quad_points": 2 * W["order"] ** 2, "quad_points_folded": Qf,
                   "mode": args.mode, "dt": head["dt"], "tau": head["tau"], "parallelism": f"replicas{world}",
                   "t_start": args.t_start, "setup_steps": head["setup"],
                   "l2": f"working set > L2: {'FP64' if args.mode == 'fp64' else 'FP32'} psi (C x Q'pad x "
                         f"{8 if args.mode == 'fp64' else 4} B = "
                         f"{C * ((Qf + 31) // 32 * 32) * (8 if args.mode == 'fp64' else 4) / 1e6:.0f} MB) "
                         "written and re-read every step; no flush"},
        "closures_per_s": closures_per_s,
        "evaluations_per_cell_step": head["stats"]["evaluations"] / (C * args.steps),
        "roofline": {"kernel": ekey,
                     "bound": "alu", "achieved": achieved, "peak": peak_ops,
                     "unit": "T FP64 instructions/s",
                     "frac": achieved / peak_ops, "traffic": None,
                     "peak_source": "FP64 pipe: measured cuBLAS DGEMM 4096^3 in this run "
                                    f"({peak:.3f} TFLOP/s) / 2 flops per FMA instruction; achieved "
                                    "counts the sweep's FP64 instructions per cell evaluation "
                                    "(sum-factorised exponent and moments; 2 per exp in the mixed "
                                    "modes, 8 in FP64 mode) x evaluations "
                                    "/ the sweep's CUDA-event time",
                     "fp64_ops_per_cell_eval": ops,
                     "fp64_flops_per_cell_eval": fl,
                     "fp64_tflops_achieved": pe["units"] * fl / sweep_s / 1e12,
                     "exps_per_cell_eval": work["exps"],
                     "sweep_grid": work["sweep_grid"], "sweep_items": work["sweep_items"],
                     "tensor_flops_per_cell_eval": work["tensor_flops"],
                     "tensor_tflops_achieved": pe["units"] * work["tensor_flops"] / (pe["total_ms"] / 1e3) / 1e12,
                     "newton_flops_per_cell_eval": work["newton_flops"],
                     "gaunt_nnz": work["gaunt_nnz"], "cell_evals": pe["units"],
                     "launches": pe["launches"], "avg_launch_ms": pe["total_ms"] / pe["launches"]},
        "kernels": {k: {"launches": v["launches"], "ms": v["total_ms"],
                        "share": v["total_ms"] / max(1e-9, sum(x["total_ms"] for x in head["prof"].values()))}
                    for k, v in head["prof"].items()},
        "learned_training": None if net is None else net.info,
        "modes": {m: dict(mode_line(W, r, args.steps), tau=r["tau"]) for m, r in results.items()},
        "flux_roofline": flux_roofline(W, n, Qf, head["prof"], hbm_peak_gbs(),
                                       fp32=args.mode != "fp64"),
        "extras": extras,
        "error": errors,
        "sn": sn,
        "e2e": None if args.no_e2e else {
            "value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": head["e2e_bytes"],
            "d2h_bytes_per_step": head["e2e_bytes"]},
        "gpu_launches": int(head["stats"]["launches"]),
        "launches_before_timed": int(head["launches_before"]),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
