#!/usr/bin/env python
"""Throughput of the localized extrapolated-regularization hot path (Siebor & Tlupova) on GB300.

Workload (fixed): unit sphere, lattice-crossing quadrature at h = 1/128 (N = 272,718 nodes),
M = 392,718 targets = every node + 100,000 near-band points (|b| <= 4h) + 20,000 points uniform
in [-2, 2]^3; degree-4 polynomial densities f, q; delta_k = rho_k h with rho = (2, 3, 4);
regularization only for r/delta <= 6.  One step = one pass of the whole path for both layers:
closest point, far field, near sums for three deltas and the extrapolation solve.

The headline arm is the precision variant (far field with FP32 operands and FP64 accumulation;
near sums, closest point and solve in FP64); the plain FP64 path is timed on the same
workload for the speedup.  Prints one JSON line (rank 0).

With --gpus N under torchrun the targets are cut into N contiguous slices of their Morton order
(one per GPU, every GPU holding the whole surface): the total work is fixed (strong scaling), no
collective runs on the data path, and the slices are gathered once after the timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "SL+DL target evals/s and Gpair-interactions/s at N~300k; speedup vs plain FP64"
UNIT = "target-evals/s"
WORKLOAD = "sphere128"
# Nominal non-tensor peaks at the 2070 MHz maximum SM clock: 152 SMs x 128 FP32 lanes x 2 flop,
# and the FP64 rate of 1.25 TFLOP/s; both are scaled by the median SM clock seen while timing.
SM_MAX_MHZ = 2070.0
FP32_PEAK_NOMINAL = 152 * 128 * 2 * SM_MAX_MHZ * 1e6
FP64_PEAK_NOMINAL = 1.25e12
# Algorithmic work per unit (convention: FMA = 2 flops, rsqrt = 1 op, erf/exp counted as calls):
# a far (target, node) pair costs 34 flops + 1 rsqrt for the single layer and 33 + 1 rsqrt for the
# double layer; a near (node, delta) evaluation with t <= cutoff_t costs 30 flops + 1 erf + 1 exp.
FAR_FLOPS_PER_PAIR = 34 + 1 + 33 + 1      # both layers, one far pair
NEAR_FLOPS_PER_DELTA_EVAL = 30 + 1 + 1    # one regularized (node, delta) term, both layers
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of
# the sphere128 workload, each with a fingerprint of the kernel's sources at capture time (comments
# and blank space removed).  When the sources no longer match, the kernel has changed since the
# counters were taken and the roofline reports traffic as null until they are captured again.
NCU_TRAFFIC = {
    ("sphere128", "k_near"): (232271360 + 173821184, "58eac48f48c82c5e"),
    ("sphere128", "k_far32"): (60701184 + 30923264, "1e0ef82f28b6f2bc"),
}
KERNEL_SOURCES = {"k_near": ("k_near.cu", "near_common.cuh", "ers_internal.h"),
                  "k_far32": ("k_far.cu", "ers_internal.h")}


def source_fingerprint(kernel: str) -> str:
    """sha256 (first 16 hex digits) of the kernel's source files with comments and blank space removed."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        text = open(os.path.join(ROOT, "paper_2507_00156_gb300", "csrc", name)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("".join(text.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, kernel: str):
    rec = NCU_TRAFFIC.get((workload, kernel))
    if rec is None or source_fingerprint(kernel) != rec[1]:
        return None
    return rec[0]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the plain FP64 path (and of its e2e)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="target wall time of the CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-launch leg")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-closure leg")
    ap.add_argument("--batched-small", action="store_true",
                    help="profiling only: the batched leg on two spheres at h = 1/32 and 4 bodies")
    ap.add_argument("--workload", default=WORKLOAD, help="profiling only: a smaller case (e.g. sphere64)")
    ap.add_argument("--no-two-drop", action="store_true", help="skip the two-drop (Sec. 4.3) leg")
    ap.add_argument("--two-drop-fine", action="store_true", help="two-drop leg: h = 1/128 with the FP64 treecode")
    ap.add_argument("--two-drop-control", action="store_true",
                    help="two-drop leg: also the same series with a gap of 0.1 instead of 1.5e-8")
    ap.add_argument("--tree", default=None,
                    help="treecode leg: theta,N0,p (default: the parameters of Eq. (optimal_params) for h)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        if args.impl == "ours":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def build_targets(wl, x):
    return np.ascontiguousarray(np.concatenate([x, wl.extra_targets]))


def morton_keys(y: np.ndarray, cell: float) -> np.ndarray:
    """Morton (Z-order) key of each point's cell of width `cell` (10 bits per axis)."""
    c = np.floor((y - y.min(axis=0)) / cell).astype(np.int64)
    c = np.clip(c, 0, 1023)
    key = np.zeros(len(y), dtype=np.int64)
    for bit in range(10):
        for a in range(3):
            key |= ((c[:, a] >> bit) & 1) << (3 * bit + a)
    return key


def shard_indices(y: np.ndarray, cell: float, world: int):
    """The targets in Morton order of their cells, cut into `world` contiguous slices of sizes
    differing by at most one: slice r (an index array into y, in that order) is rank r's share."""
    order = np.argsort(morton_keys(y, cell), kind="stable")
    return np.array_split(order, world)


def gather_rows(local, idx, M: int, world: int):
    """Every rank's rows (local[i] belongs to target idx[i]) assembled into one (M, k) array in the
    original target order, on every rank (one all_gather of slices padded to the largest)."""
    import torch
    import torch.distributed as dist
    if world == 1:
        out = torch.empty((M,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
        out[torch.as_tensor(idx, device=local.device)] = local
        return out
    n = torch.tensor([local.shape[0]], device=local.device)
    ns = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(ns, n)
    cap = int(max(int(v.item()) for v in ns))
    pad = torch.zeros((cap,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    ipad = torch.full((cap,), -1, dtype=torch.int64, device=local.device)
    ipad[: local.shape[0]] = torch.as_tensor(idx, dtype=torch.int64, device=local.device)
    rows = [torch.zeros_like(pad) for _ in range(world)]
    ids = [torch.zeros_like(ipad) for _ in range(world)]
    dist.all_gather(rows, pad)
    dist.all_gather(ids, ipad)
    out = torch.empty((M,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    for r, i, k in zip(rows, ids, ns):
        k = int(k.item())
        out[i[:k]] = r[:k]
    return out


def rel_max(a: np.ndarray, b: np.ndarray, world: int) -> float:
    """max |a - b| / max |b| over the targets of every rank (0 where a rank has none)."""
    num = float(np.abs(a - b).max()) if a.size else 0.0
    den = float(np.abs(b).max()) if b.size else 0.0
    num, den = max_over_ranks(num, world), max_over_ranks(den, world)
    return num / den if den > 0 else 0.0


def sum_over_ranks(x, world: int):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor(np.atleast_1d(np.asarray(x, dtype=np.float64)),
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    v = [int(z) for z in t.cpu().numpy()]
    return v if np.ndim(x) else v[0]


def cpu_baseline(wl, y, seconds: float, gpu_results=None):
    """The FP64 oracle (localized mode, OpenMP over targets) on a seeded sample of the same
    targets, sized from a short calibration run to about `seconds` of wall time."""
    import oracle
    x, n, w = oracle.quadrature(wl.shape, wl.h)
    f = workloads.poly_eval(wl.f_coef, x)
    q = workloads.poly_eval(wl.q_coef, x)

    def run(idx):
        yy = y[idx]
        x0, n0, b = oracle.closest_point(wl.shape, yy)
        f0, q0 = workloads.poly_eval(wl.f_coef, x0), workloads.poly_eval(wl.q_coef, x0)
        t0 = time.perf_counter()
        x0, n0, b = oracle.closest_point(wl.shape, yy)
        u, v, _ = oracle.evaluate(x, n, w, f, q, yy, x0, n0, b, f0, q0, wl.h, wl.rho, 6.0, oracle.LOCALIZED)
        return time.perf_counter() - t0, u, v

    cal = workloads.subsample(256, len(y), 11)
    t_cal, _, _ = run(cal)
    count = int(min(len(y), max(256, 256 * seconds / max(t_cal, 1e-3))))
    idx = workloads.subsample(count, len(y), 12)
    t, u, v = run(idx)
    out = {"value": count / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"{count} of {len(y)} targets (seeded, same node/band/far mix), FP64 oracle, localized "
                     f"far+near form, closest point included; {t:.1f} s wall"}
    errs = {}
    if gpu_results:
        for name, (ug, vg) in gpu_results.items():
            errs[name] = {"SL": float(np.abs(ug[idx] - u).max() / np.abs(u).max()),
                          "DL": float(np.abs(vg[idx] - v).max() / np.abs(v).max())}
    return out, errs


def batched_leg(ers, torch, steps: int, warmup: int, small: bool = False):
    """Two unit spheres 0.01 apart at h = 1/96 (each evaluated at the nodes of both) plus 16
    uneven bodies (own nodes + 5 % near band), 8 densities per surface, as ONE persistent launch
    replayed from a CUDA graph.  Unit: (target, density) evaluations of both layers per second.
    small (profiling only): the spheres at h = 1/32 and 4 bodies."""
    nrhs = 8
    pair, bodies = (workloads.batched_config(nrhs=nrhs, n_bodies=4, h_pair=1 / 32) if small
                    else workloads.batched_config(nrhs=nrhs))
    dev = torch.device("cuda")
    surfs = []

    def surface(body):
        s = ers.Surface(body.shape.center, body.shape.axes, body.h)
        x = s.nodes()[0].cpu().numpy()
        f = np.stack([workloads.poly_eval(c, x) for c in body.f_coefs])
        q = np.stack([workloads.poly_eval(c, x) for c in body.q_coefs])
        s.set_density_multi(torch.from_numpy(f).to(dev), torch.from_numpy(q).to(dev))
        surfs.append(s)
        return s, x

    def problem(s, body, y):
        yd = torch.from_numpy(np.ascontiguousarray(y)).to(dev)
        x0, n0, b = s.closest_point(yd)
        x0h = x0.cpu().numpy()
        f0 = np.stack([workloads.poly_eval(c, x0h) for c in body.f_coefs])
        q0 = np.stack([workloads.poly_eval(c, x0h) for c in body.q_coefs])
        M = len(y)
        return dict(s=s, y=yd, x0=x0, n0=n0, b=b, f0=torch.from_numpy(f0).to(dev),
                    q0=torch.from_numpy(q0).to(dev),
                    u=torch.empty((nrhs, M, 3), dtype=torch.float64, device=dev),
                    v=torch.empty((nrhs, M, 3), dtype=torch.float64, device=dev))

    (sA, xA), (sB, xB) = surface(pair[0]), surface(pair[1])
    yAB = np.concatenate([xA, xB])
    probs = [problem(sA, pair[0], yAB), problem(sB, pair[1], yAB)]
    for i, body in enumerate(bodies):
        s, x = surface(body)
        band = workloads.near_band_targets(body.shape, max(1, len(x) // 20), 4 * body.h,
                                           np.random.default_rng(2000 + i))[0]
        probs.append(problem(s, body, np.concatenate([x, band])))
    batch = ers.Batch(probs, nrhs, rho=(2.0, 3.0, 4.0))
    nitems, grid = batch.info()
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        batch.launch()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        batch.launch()
        b.record(stream)
        b.synchronize()
        total += a.elapsed_time(b) / 1e3
    targets = sum(int(p["y"].shape[0]) for p in probs)
    pairs = sum(int(p["y"].shape[0]) * p["s"].N for p in probs)
    ok = all(bool(torch.isfinite(p["u"]).all()) and bool(torch.isfinite(p["v"]).all()) for p in probs)
    return {"value": steps * targets * nrhs / total, "unit": "(target, density) evals/s, both layers",
            "ms_per_launch": total / steps * 1e3, "problems": len(probs), "nrhs": nrhs, "targets": targets,
            "surface_nodes": [s.N for s in surfs], "gpairs_x_rhs_per_s": steps * pairs * nrhs / total / 1e9,
            "work_items": nitems, "persistent_grid": grid, "launches_per_step": 1, "finite": ok,
            "workload": ("profiling case: two unit spheres gap 0.01 at h=1/32 + 4 bodies, 8 densities" if small else
                         "two unit spheres gap 0.01 at h=1/96 (self + neighbour nodes) + 16 bodies "
                         "(semi-axes U[0.6,1], h in {1/32,1/48,1/64,1/96}, own nodes + 5% band), 8 densities")}


def two_drop_leg(ers, torch, fine: bool, control: bool = False):
    """Two drops nearly touching (Sec. 4.3): GMRES on Eq. (IE-2Surf) at h = 1/16, 1/32, 1/64 in FP64
    with the direct far field, and h = 1/128 for the e_64 row: with the mixed direct far field (its
    solution agrees with the FP64 treecode's to 4e-8), or with fine the FP64 treecode at Table 2's
    theta = 0.6, N0 = 4000, p = 10.  Iterations, solve times and the self-convergence errors of
    Table 2 (max and L2 over the velocity components at the coarse nodes), the max also over the
    nodes farther than 4h from the contact point (1, 0, 0).  With control, the same for a second
    drop centred at (2, 0, 0.6403) (gap 0.1 instead of 1.5e-8)."""
    from paper_2507_00156_gb300 import two_drop as gtd

    def series(eps, levels):
        sol, rows = {}, []
        for inv, tree, prec in levels:
            P = gtd.TwoDrops(1 / inv, eps=eps, tree=tree, precision=prec)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, it, rel, conv = P.solve(tol=1e-10)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            u1, u2 = P.split(x)
            sol[inv] = ([u1.cpu().numpy(), u2.cpu().numpy()], [P.x[0].cpu().numpy(), P.x[1].cpu().numpy()])
            far = "treecode theta, N0, p = %s" % (tree,) if tree else "direct"
            rows.append({"inv_h": inv, "N": P.N, "iterations": it, "relres": rel, "converged": conv, "solve_s": secs,
                         "matvecs": P.matvecs, "far_field": far + (" (mixed precision)" if prec else "")})
            del P
        invs = [r["inv_h"] for r in rows]
        for i in range(len(invs) - 1):
            (uc, xc), (uf, xf) = sol[invs[i]], sol[invs[i + 1]]
            mx, l2 = gtd.self_convergence(uc, xc, uf, xf)
            far4 = [np.linalg.norm(xx - np.array([1.0, 0.0, 0.0]), axis=1) > 4.0 / invs[i] for xx in xc]
            mx4, _ = gtd.self_convergence([u[k] for u, k in zip(uc, far4)], [xx[k] for xx, k in zip(xc, far4)], uf, xf)
            rows[i]["max_err"], rows[i]["l2_err"], rows[i]["max_err_beyond_4h_of_contact"] = mx, l2, mx4
            if i > 0:
                rows[i]["max_order"] = float(np.log2(rows[i - 1]["max_err"] / mx))
                rows[i]["l2_order"] = float(np.log2(rows[i - 1]["l2_err"] / l2))
        return rows

    last = (128, (0.6, 4000, 10), ers.PREC_FP64) if fine else (128, None, ers.PREC_MIXED)
    levels = [(16, None, ers.PREC_FP64), (32, None, ers.PREC_FP64), (64, None, ers.PREC_FP64), last]
    out = {"rows": series(gtd.EPS, levels), "precision": "fp64 (h = 1/128: %s)" % ("fp64 treecode" if fine else
                                                                                   "mixed direct far field"),
           "rho": [3, 4, 5], "rho_sharp": 3, "gmres_tol": 1e-10,
           "note": "Table 2 (Sec. 4.3): errors e_h = u_h - u_{h/2} at the nodes of h; the paper's 1/16..1/64 rows: "
                   "iterations 13, 12, 12; max 3.17e-3, 1.07e-4, 4.06e-6; L2 1.19e-4, 6.11e-6, 2.11e-7"}
    if control:
        out["control_gap_0.1"] = series(0.6403, levels)
    return out


TRAIN_RADII = (1.0, 1.0, 1.0, 0.85, 0.7)  # one seeded density each
LEARNED_H = 1 / 96     # training spacing = the evaluation spacing
LEARNED_STEPS = 3000   # Adam steps per network


def learned_leg(ers, torch, s, wl, steps: int, warmup: int):
    """The learned near-field closure: networks trained on the GPU (own kernels) from five seeded
    densities on spheres at the evaluation spacing h = 1/96 (three on the unit sphere, one each on
    spheres of radius 0.85 and 0.7, so that the curvature input kappa h spans 1/96 .. 1/67; targets:
    the nodes and 200,000 band points |b| <= 6 rho_2 h, the two-delta closure's near radius), then
    evaluated on the two unit spheres 0.01 apart at h = 1/96: the integral over the first sphere at
    the nodes of both, with validation against the three-delta method (tolerance 1e-5, every 32nd
    target), the per-layer gate and fallback to the method.  Also timed with the closure accepted
    unconditionally (no fallback), against the plain mixed evaluation of the same problem."""
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rng = np.random.default_rng(5005)
    data = {1: [], 2: []}
    h_train = LEARNED_H
    band_w = 6.0 * wl.rho[1] * h_train
    t0 = time.perf_counter()
    surfs = {}
    for R in TRAIN_RADII:
        if R not in surfs:
            sh = workloads.Shape((0.0, 0.0, 0.0), (R, R, R))
            sR = ers.Surface(sh.center, sh.axes, h_train)
            xR = sR.nodes()[0].cpu().numpy()
            yd = t(np.concatenate([xR, workloads.near_band_targets(sh, 200000, band_w, rng)[0]]))
            x0, n0, b = sR.closest_point(yd)
            surfs[R] = (sR, xR, yd, x0, n0, b, x0.cpu().numpy())
        sR, x, yd, x0, n0, b, x0h = surfs[R]
        fc, qc = workloads.density_coeffs(rng), workloads.density_coeffs(rng)
        sR.set_density(t(workloads.poly_eval(fc, x)), t(workloads.poly_eval(qc, x)))
        f0, q0 = t(workloads.poly_eval(fc, x0h)), t(workloads.poly_eval(qc, x0h))
        u3, v3 = sR.eval(yd, f0, q0, rho=wl.rho, precision=ers.PREC_MIXED, x0=x0, n0=n0, b=b)
        for nd in (1, 2):
            out = ers.closure_data(sR, yd, x0, n0, b, f0, q0, u3, v3, rho=wl.rho, ndelta=nd)
            sel = out[4].bool()
            data[nd].append([z[sel] for z in out[:4]])
    del surfs
    t_data = time.perf_counter() - t0
    nets, losses = {}, {}
    t0 = time.perf_counter()
    for nd in (1, 2):
        Xs, Xd, Ts, Td = (torch.cat([d[i] for d in data[nd]]).contiguous() for i in range(4))
        nets[nd] = ers.Closure(seed=100 + nd)
        losses[nd] = [nets[nd].train(layer, X, T, steps=LEARNED_STEPS, batch=8192, lr=2e-3)
                      for layer, (X, T) in enumerate(((Xs, Ts), (Xd, Td)))]
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    nsamples = {nd: int(sum(d[0].shape[0] for d in data[nd])) for nd in (1, 2)}
    del data

    # evaluation problem: sphere A at the origin, targets = nodes of A and of B at (2.01, 0, 0)
    pair, _ = workloads.batched_config(gap=0.01, nrhs=1, n_bodies=0)
    A, B = pair
    sa = ers.Surface(A.shape.center, A.shape.axes, A.h)
    sb = ers.Surface(B.shape.center, B.shape.axes, B.h)
    xa, xb = sa.nodes()[0].cpu().numpy(), sb.nodes()[0].cpu().numpy()
    del sb
    fc, qc = A.f_coefs[0], A.q_coefs[0]
    sa.set_density(t(workloads.poly_eval(fc, xa)), t(workloads.poly_eval(qc, xa)))
    ye = np.concatenate([xa, xb])
    yed = t(ye)
    x0, n0, b = sa.closest_point(yed)
    x0h = x0.cpu().numpy()
    f0, q0 = t(workloads.poly_eval(fc, x0h)), t(workloads.poly_eval(qc, x0h))
    M = len(ye)
    u = torch.empty((M, 3), dtype=torch.float64, device=dev)
    v = torch.empty((M, 3), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(warmup):
            fn()
        total, out = 0.0, None
        for _ in range(steps):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = fn()
            e.record(stream)
            e.synchronize()
            total += a.elapsed_time(e) / 1e3
        return total / steps, out

    t_plain, _ = timed(lambda: sa.eval(yed, f0, q0, rho=wl.rho, precision=ers.PREC_MIXED, x0=x0, n0=n0, b=b,
                                       u=u, v=v))
    u_ref, v_ref = u.cpu().numpy(), v.cpu().numpy()
    # the plain FP64 path on the same problem (one step after one warm-up)
    sa.eval(yed, f0, q0, rho=wl.rho, precision=ers.PREC_FP64, x0=x0, n0=n0, b=b, u=u, v=v)
    a64, e64 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a64.record(stream)
    sa.eval(yed, f0, q0, rho=wl.rho, precision=ers.PREC_FP64, x0=x0, n0=n0, b=b, u=u, v=v)
    e64.record(stream)
    e64.synchronize()
    t_fp64 = a64.elapsed_time(e64) / 1e3
    res = {"workload": "train: spheres of radius 1, 1, 1, 0.85, 0.7 at h=1/96, one seeded density each, "
                       "nodes + 200k band points |b| <= 18h; evaluate: two unit spheres gap 0.01, h=1/96, "
                       "integral over the first at the nodes of both (a density not trained on)",
           "targets": M, "nodes": int(xa.shape[0]),
           "plain_fp64": {"value": M / t_fp64, "unit": UNIT, "ms_per_step": t_fp64 * 1e3},
           "plain_mixed": {"value": M / t_plain, "unit": UNIT, "ms_per_step": t_plain * 1e3},
           "training": {"samples_per_network": nsamples, "densities": len(TRAIN_RADII), "steps": LEARNED_STEPS,
                        "batch": 8192, "data_s": t_data, "train_s": t_train}}
    args = (yed, x0, n0, b, f0, q0)
    # an untrained closure predicts no correction: what the network gains over the one- or
    # two-delta sums alone
    zero = ers.Closure(seed=0)
    for nd in (2, 1):
        t_val, out = timed(lambda: ers.eval_learned(sa, nets[nd], *args, rho=wl.rho, precision=ers.PREC_MIXED,
                                                    tol=1e-5, vstride=32, ndelta=nd, u=u, v=v))
        _, _, verr, fb = out
        used, ew, eo = nets[nd].last_gate()
        t_acc, _ = timed(lambda: ers.eval_learned(sa, nets[nd], *args, rho=wl.rho, precision=ers.PREC_MIXED,
                                                  tol=1e30, vstride=1 << 20, ndelta=nd, u=u, v=v))
        ul, vl = u.cpu().numpy(), v.cpu().numpy()
        res[f"ndelta{nd}"] = {
            "value": M / t_val, "unit": UNIT, "ms_per_step": t_val * 1e3,
            "fell_back_at_tol_1e-5": bool(fb), "validation_rel_err": [float(z) for z in verr],
            "gate": {"network_kept": list(used), "validation_err_with_network": list(ew),
                     "validation_err_without_network": list(eo)},
            "targets_outside_training_extent": nets[nd].last_out_of_range(),
            "accepted": {"value": M / t_acc, "ms_per_step": t_acc * 1e3,
                         "speedup_vs_plain_mixed": t_plain / t_acc, "speedup_vs_plain_fp64": t_fp64 / t_acc,
                         "max_rel_err_vs_three_delta": {
                             "SL": float(np.abs(ul - u_ref).max() / np.abs(u_ref).max()),
                             "DL": float(np.abs(vl - v_ref).max() / np.abs(v_ref).max())}},
            "final_train_loss": losses[nd]}
        _, _, verr0, _ = ers.eval_learned(sa, zero, *args, rho=wl.rho, precision=ers.PREC_MIXED, tol=1e30,
                                          vstride=32, ndelta=nd, u=u, v=v)
        u0, v0 = u.cpu().numpy(), v.cpu().numpy()
        res[f"ndelta{nd}"]["without_network"] = {
            "validation_rel_err": [float(z) for z in verr0],
            "max_rel_err_vs_three_delta": {"SL": float(np.abs(u0 - u_ref).max() / np.abs(u_ref).max()),
                                           "DL": float(np.abs(v0 - v_ref).max() / np.abs(v_ref).max())}}
    return res


def run_reference(args, world, rank):
    """--impl reference: the FP64 oracle as the reference arm, on host cores, rank 0 only."""
    if rank != 0:
        return
    import oracle
    wl = workloads.config(WORKLOAD)
    x, n, w = oracle.quadrature(wl.shape, wl.h)
    f = workloads.poly_eval(wl.f_coef, x)
    q = workloads.poly_eval(wl.q_coef, x)
    y = build_targets(wl, x)
    per_step = 1024
    times = []
    for step in range(args.warmup + args.steps):
        idx = workloads.subsample(per_step, len(y), 100 + step)
        yy = y[idx]
        t0 = time.perf_counter()
        x0, n0, b = oracle.closest_point(wl.shape, yy)
        f0, q0 = workloads.poly_eval(wl.f_coef, x0), workloads.poly_eval(wl.q_coef, x0)
        oracle.evaluate(x, n, w, f, q, yy, x0, n0, b, f0, q0, wl.h, wl.rho, 6.0, oracle.LOCALIZED)
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = per_step / t
    sample = (f"{per_step} seeded targets per step out of {len(y)} (same mix), FP64 oracle, localized far+near "
              f"form; value is targets/s, i.e. extrapolated per target to the full workload")
    print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "strong",
                      "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                      "config": {"workload": WORKLOAD, "N": len(w), "M": len(y), "rho": list(wl.rho)},
                      "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch

    import paper_2507_00156_gb300 as ers
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = workloads.config(args.workload)
    s = ers.Surface(wl.shape.center, wl.shape.axes, wl.h)
    xd, _, _ = s.nodes()
    x = xd.cpu().numpy()
    fdev = torch.from_numpy(workloads.poly_eval(wl.f_coef, x)).to(dev)
    qdev = torch.from_numpy(workloads.poly_eval(wl.q_coef, x)).to(dev)
    s.set_density(fdev, qdev)
    y_all = build_targets(wl, x)
    M_all, N = len(y_all), s.N
    # N > 1: the targets are cut into contiguous slices of their Morton order (cells of 6h), one per
    # rank; every rank holds the whole surface, and no collective runs on the data path
    shard = shard_indices(y_all, 6.0 * wl.h, world)[rank] if world > 1 else np.arange(M_all)
    y = np.ascontiguousarray(y_all[shard])
    M = len(y)
    yd = torch.from_numpy(y).to(dev)
    x0, _, b0 = s.closest_point(yd)  # set-up only: the densities at the closest points are inputs
    on_surface = b0.cpu().numpy() == 0.0
    x0h = x0.cpu().numpy()
    f0h, q0h = workloads.poly_eval(wl.f_coef, x0h), workloads.poly_eval(wl.q_coef, x0h)
    f0, q0 = torch.from_numpy(f0h).to(dev), torch.from_numpy(q0h).to(dev)
    u = torch.empty((M, 3), dtype=torch.float64, device=dev)
    v = torch.empty((M, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step(prec, concurrent=False, sharp=False, rho=None, tree=None):
        s.eval(yd, f0, q0, rho=rho or wl.rho, precision=prec, u=u, v=v, concurrent=concurrent, sharp=sharp,
               tree=tree)

    def timed(prec, steps, warm, concurrent=False, sharp=False, rho=None, tree=None):
        for _ in range(warm):
            step(prec, concurrent, sharp, rho, tree)
        s.profile(True)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        evs = []
        kern = []
        for _ in range(steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(prec, concurrent, sharp, rho, tree)
            b.record(stream)
            evs.append((a, b))
            kern.append(s.last_profile())  # synchronizes; device times are unaffected
        torch.cuda.synchronize()
        barrier(world)
        s.profile(False)
        total = sum(a.elapsed_time(b) for a, b in evs) / 1e3
        kms = np.mean(np.array(kern), axis=0)
        return total, kms

    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    except Exception:
        gpu_id = None

    # headline: precision variant
    sampler = ClockSampler(gpu_id)
    t_mixed, k_mixed = timed(ers.PREC_MIXED, args.steps, args.warmup)
    clocks = sampler.stop()
    near_targets, near_pairs, far_pairs = s.last_counts()
    cls_counts = s.last_class_counts()
    cls_local = list(cls_counts)  # this rank's pairs, for this rank's roofline
    far_local = far_pairs
    defect_counts = s.last_defect_class_counts()
    u_mixed, v_mixed = u.cpu().numpy(), v.cpu().numpy()
    t_mixed = max_over_ranks(t_mixed, world)
    ms_step = t_mixed / args.steps * 1e3
    value = args.steps * M_all / t_mixed
    # the slices gathered once, outside the timed region: the whole result on every rank
    u_all = gather_rows(u, shard, M_all, world)
    gathered_finite = bool(torch.isfinite(u_all).all().item())
    del u_all
    near_targets, near_pairs, far_pairs = sum_over_ranks([near_targets, near_pairs, far_pairs], world)
    cls_counts = sum_over_ranks(list(cls_counts), world)
    defect_counts = sum_over_ranks(list(defect_counts), world)

    # the same mixed step with the on-surface option (ERS_OPT_SHARP, Sec. 2.1): node targets with
    # one delta# = rho_2 h and the s#_p, no extrapolation
    t_sh, k_sh = timed(ers.PREC_MIXED, args.steps, 1, sharp=True)
    t_sh = max_over_ranks(t_sh, world)
    nsh_pairs = s.last_sharp_pairs()
    u_sh, v_sh = u.cpu().numpy(), v.cpu().numpy()

    # the same mixed step with the O(delta^7) variant (ERS_OPT_FOUR_DELTA): a fourth delta
    # rho_3 = 2 rho_2 - rho_1, near radius cutoff_t rho_3 h
    rho4 = tuple(wl.rho) + (2 * wl.rho[2] - wl.rho[1],)
    t_fd, k_fd = timed(ers.PREC_MIXED, args.steps, 1, rho=rho4)
    t_fd = max_over_ranks(t_fd, world)
    fd_counts = s.last_counts()
    fd_cls = s.last_class_counts()
    u_fd, v_fd = u.cpu().numpy(), v.cpu().numpy()

    # the same mixed step with the far sums by the treecode of Sec. 3.4 (ERS_OPT_TREECODE) at the
    # parameters of Eq. (optimal_params) for this h; the modified weights are built in the warm-up
    # (they depend only on the densities) and timed separately after a density update
    tree = ers.treecode_defaults(wl.h)
    if args.tree:
        th, n0s, ps = args.tree.split(",")
        tree = (float(th), int(n0s), int(ps))
    t_tc, k_tc = timed(ers.PREC_MIXED, args.steps, 1, tree=tree)
    t_tc = max_over_ranks(t_tc, world)
    tc_stats = s.tree_stats()
    tc_counts = s.last_counts()
    u_tc, v_tc = u.cpu().numpy(), v.cpu().numpy()
    s.set_density(fdev, qdev)  # same densities, new version: the next treecode eval rebuilds the weights
    _, k_tcw = timed(ers.PREC_MIXED, 1, 0, tree=tree)

    # the same mixed step with the far and near fields on two streams (ERS_OPT_CONCURRENT)
    t_conc, k_conc = timed(ers.PREC_MIXED, args.steps, 1, concurrent=True)
    t_conc = max_over_ranks(t_conc, world)

    # plain FP64 path on the same workload
    t64, k64 = (None, None)
    if args.fp64_steps > 0:
        t64, k64 = timed(ers.PREC_FP64, args.fp64_steps, 1)
        t64 = max_over_ranks(t64, world)
    u64, v64 = u.cpu().numpy(), v.cpu().numpy()

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    yh = torch.from_numpy(y).pin_memory().numpy()
    f0p = torch.from_numpy(f0h).pin_memory().numpy()
    q0p = torch.from_numpy(q0h).pin_memory().numpy()
    uh = torch.empty((M, 3), dtype=torch.float64).pin_memory().numpy()
    vh = torch.empty((M, 3), dtype=torch.float64).pin_memory().numpy()

    def timed_host(prec, steps):
        s.eval_host(yh, f0p, q0p, rho=wl.rho, precision=prec, u=uh, v=vh)
        torch.cuda.synchronize()
        barrier(world)
        te = 0.0
        for _ in range(steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.eval_host(yh, f0p, q0p, rho=wl.rho, precision=prec, u=uh, v=vh)
            te += time.perf_counter() - t0
        barrier(world)
        return max_over_ranks(te, world)

    te = timed_host(ers.PREC_MIXED, args.steps)
    e2e = {"value": args.steps * M_all / te, "unit": UNIT, "h2d_bytes_per_step": 3 * M_all * 3 * 8,
           "d2h_bytes_per_step": 2 * M_all * 3 * 8, "api": "ers_eval_host (pinned host arrays, includes copies)"}
    e2e64 = None
    if args.fp64_steps > 0:
        te64 = timed_host(ers.PREC_FP64, args.fp64_steps)
        e2e64 = {"value": args.fp64_steps * M_all / te64, "unit": UNIT, "steps": args.fp64_steps,
                 "h2d_bytes_per_step": 3 * M_all * 3 * 8, "d2h_bytes_per_step": 2 * M_all * 3 * 8,
                 "api": "ers_eval_host, plain FP64 path (pinned host arrays, includes copies)"}

    # differences and counts over the targets of every rank
    diffs = {"sharp": (rel_max(u_sh[on_surface], u_mixed[on_surface], world),
                       rel_max(v_sh[on_surface], v_mixed[on_surface], world)),
             "fd": (rel_max(u_fd, u_mixed, world), rel_max(v_fd, v_mixed, world)),
             "tc": (rel_max(u_tc, u_mixed, world), rel_max(v_tc, v_mixed, world))}
    if t64 is not None:
        diffs["fp64"] = (rel_max(u_mixed, u64, world), rel_max(v_mixed, v64, world))
    n_on_surface = sum_over_ranks(int(on_surface.sum()), world)
    nsh_pairs = sum_over_ranks(nsh_pairs, world)
    fd_counts = sum_over_ranks(list(fd_counts), world)
    fd_cls = sum_over_ranks(list(fd_cls), world)
    tc_app, tc_dir, tc_near = sum_over_ranks([tc_stats["approximated"], tc_stats["direct"], tc_counts[1]], world)
    tc_stats = dict(tc_stats, approximated=tc_app, direct=tc_dir)

    if rank != 0:
        return
    # roofline of the dominant kernel of the headline step
    near_flops = None
    sm_mhz = clocks.get("sm_mhz") or SM_MAX_MHZ
    scale = sm_mhz / SM_MAX_MHZ
    ms_closest, ms_far, ms_near = (float(z) for z in k_mixed)
    # cls_counts[k] = near pairs with k deltas beyond the cutoff, i.e. 3 - k regularized terms
    near_flops = NEAR_FLOPS_PER_DELTA_EVAL * sum(c * (3 - k) for k, c in enumerate(cls_local))
    far_flops = far_local * FAR_FLOPS_PER_PAIR
    roof_near = {"kernel": "k_near (near sums + extrapolation: FP64 pair geometry, float-pair factors and "
                           "contractions)", "bound": "alu", "unit": "TFLOP/s",
                 "achieved": near_flops / (ms_near * 1e-3) / 1e12, "peak": FP64_PEAK_NOMINAL * scale / 1e12,
                 "peak_source": "nominal FP64 1.25 TFLOP/s x median SM clock / 2070 MHz (FP64-accurate flops; the "
                                "float-pair arithmetic runs on the FP32 pipe, bound by instruction issue)",
                 "units": "32 flops per regularized (node, delta) term: 30 flops, erf and exp counted as one op each"}
    roof_far = {"kernel": "k_far32 (FP32 far field, FP64 tile accumulation)", "bound": "alu", "unit": "TFLOP/s",
                "achieved": far_flops / (ms_far * 1e-3) / 1e12, "peak": FP32_PEAK_NOMINAL * scale / 1e12,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x median SM clock",
                "units": "69 flops per far (target, node) pair, both layers (FMA = 2, rsqrt = 1)"}
    for r in (roof_near, roof_far):
        r["frac"] = r["achieved"] / r["peak"]
        r["traffic"] = ncu_traffic(args.workload, r["kernel"].split()[0])
    # the dominant kernel by live time; the other one beside it
    roof, roof_other = (roof_near, roof_far) if ms_near >= ms_far else (roof_far, roof_near)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "shape": "unit sphere", "h": wl.h, "N": N, "M": M_all, "rho": list(wl.rho),
                   "parallelism": ("targets sharded over %d GPUs (contiguous Morton-order slices, %d-%d targets "
                                   "per GPU; surface on every GPU; no collective on the data path)"
                                   % (world, M_all // world, -(-M_all // world)) if world > 1 else "one GPU"),
                   "cutoff_t": 6.0, "precision": ("mixed (FP32 far field with FP64 tile sums; local sums in float-pair arithmetic, ~1e-14 relative; FP64 pair geometry, closest point and solve)"),
                   "l2": "flushed between timed steps (256 MiB write, outside the timed events)"},
        "gpairs_per_s": args.steps * M_all * N / t_mixed / 1e9,
        "kernels_ms": {"closest_point": ms_closest, "far_field": ms_far, "near_field_and_solve": ms_near},
        "sharp_option": {"ms_per_step": t_sh / args.steps * 1e3,
                         "speedup_vs_extrapolated": t_mixed / t_sh,
                         "kernels_ms": {"far_field": float(k_sh[1]), "near_field_and_solve": float(k_sh[2])},
                         "on_surface_targets": n_on_surface, "on_surface_near_pairs": nsh_pairs,
                         "max_rel_diff_vs_extrapolated_on_surface": {"SL": diffs["sharp"][0],
                                                                      "DL": diffs["sharp"][1]},
                         "note": "ERS_OPT_SHARP: on-surface targets with the s#_p of Sec. 2.1, delta# = 3h, "
                                 "no extrapolation; both methods are O(h^5)"},
        "four_delta_option": {"ms_per_step": t_fd / args.steps * 1e3, "rho": list(rho4),
                              "cost_vs_three_delta": t_fd / t_mixed,
                              "kernels_ms": {"far_field": float(k_fd[1]), "near_field_and_solve": float(k_fd[2])},
                              "near_targets": fd_counts[0], "near_pairs": fd_counts[1],
                              "near_pairs_by_unregularized_deltas": fd_cls,
                              "near_tflops": NEAR_FLOPS_PER_DELTA_EVAL * sum(c * (4 - k) for k, c in enumerate(fd_cls))
                              / (float(k_fd[2]) * 1e-3) / 1e12,
                              "max_rel_diff_vs_three_delta": {"SL": diffs["fd"][0], "DL": diffs["fd"][1]},
                              "note": "ERS_OPT_FOUR_DELTA: O(delta^7) extrapolation of Sec. 1 with the I4 "
                                      "column; the difference is the three-delta method's O(h^5) error"},
        "treecode_option": {"ms_per_step": t_tc / args.steps * 1e3, "theta": tree[0], "N0": tree[1], "p": tree[2],
                            "speedup_vs_direct": t_mixed / t_tc,
                            "kernels_ms": {"far_field_treecode": float(k_tc[1]), "near_field_and_solve": float(k_tc[2])},
                            "modified_weights_ms": float(k_tcw[1]) - float(k_tc[1]),
                            "tree": tc_stats,
                            "approximated_per_target": tc_stats["approximated"] / M_all,
                            "direct_far_pairs_per_target": tc_stats["direct"] / M_all,
                            "near_pairs": tc_near,
                            "max_rel_diff_vs_direct": {"SL": diffs["tc"][0], "DL": diffs["tc"][1]},
                            "note": "ERS_OPT_TREECODE: far sums by barycentric Lagrange interpolation at "
                                    "Chebyshev points for clusters meeting the MAC (Sec. 3.4), parameters of "
                                    "Eq. (optimal_params); weights cached between steps (densities unchanged)"},
        "concurrent_option": {"ms_per_step": t_conc / args.steps * 1e3,
                              "kernels_ms": {"far_field": float(k_conc[1]), "near_field_and_solve": float(k_conc[2])},
                              "note": "same step with ERS_OPT_CONCURRENT (far and near fields on two streams, "
                                      "both timed from the fork)"},
        "counts": {"near_targets": near_targets, "near_pairs": near_pairs, "far_pairs": far_pairs,
                   "near_pairs_by_unregularized_deltas": cls_counts,
                   "near_pairs_by_defect_path_deltas": defect_counts},
        "gpu_launches": 3 * args.steps,
        "gathered": {"targets": M_all, "finite": gathered_finite,
                     "note": "the per-rank slices gathered once after the timed steps (all_gather)"},
        "roofline": roof,
        "roofline_other_kernel": roof_other,
        "clocks": clocks,
        "e2e": e2e,
    }
    if t64 is not None:
        ms64 = t64 / args.fp64_steps * 1e3
        line["plain_fp64"] = {"value": args.fp64_steps * M_all / t64, "unit": UNIT, "ms_per_step": ms64,
                              "steps": args.fp64_steps, "e2e": e2e64,
                              "gpairs_per_s": args.fp64_steps * M_all * N / t64 / 1e9,
                              "kernels_ms": {"closest_point": float(k64[0]), "far_field": float(k64[1]),
                                             "near_field_and_solve": float(k64[2])},
                              "far_fp64_tflops": far_flops / (float(k64[1]) * 1e-3) / 1e12,
                              "fp64_peak_tflops": FP64_PEAK_NOMINAL * scale / 1e12}
        line["speedup_vs_plain_fp64"] = ms64 / ms_step
        line["mixed_vs_fp64_rel"] = {"SL": diffs["fp64"][0], "DL": diffs["fp64"][1]}
    if not args.no_batched:
        line["batched"] = batched_leg(ers, torch, steps=2, warmup=1, small=args.batched_small)
    if not args.no_learned and args.workload == WORKLOAD:
        line["learned"] = learned_leg(ers, torch, s, wl, steps=args.steps, warmup=1)
    if not args.no_two_drop and args.workload == WORKLOAD:
        line["two_drop"] = two_drop_leg(ers, torch, fine=args.two_drop_fine, control=args.two_drop_control)
    if world == 1 and not args.no_cpu_baseline:
        cb, errs = cpu_baseline(wl, y, args.cpu_seconds, {"mixed": (u_mixed, v_mixed), "fp64": (u64, v64)})
        line["cpu_baseline"] = cb
        line["max_rel_err_vs_oracle_on_cpu_sample"] = errs
    print(json.dumps(line))


if __name__ == "__main__":
    main()
