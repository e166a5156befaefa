#!/usr/bin/env python
"""Benchmark of the AB-/BA-GKB hot path on one B300.

Workload: the 512x512 flat fan-beam problem (720 angles over [0, 360), 725
bins, SOD 1024, SDD 2048, seeded 30-ellipse phantom, 2 % noise), FP32
projectors with FP64 GKB scalars, 150 iterations (the paper's fixed timing
length).  One step = one BA-GKB solve plus one AB-GKB solve of that problem,
run as one two-slice batched launch of the library (the two solves overlap
on the GPU; the line also reports them run one after another), so a step is
300 GKB iterations; the metric is GKB iterations per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Beside the headline the line carries: the roofline of the dominant kernel
against the shared-memory gather ceiling of a projector (one 4-byte word per
lane per clock: 32 matrix non-zeros per SM per clock), every projector's and
the reorthogonalisation's own fraction, the matched pair B = A^T run as
plain GKB on the same problem, AB-/BA-GMRES on the same problem, the 64x64 FP64 workload (iterations/s and
kernels per iteration), the multi-slice batch, the learned stop, and the
FP64 oracle timed on the host cores (1 thread and all threads).

Under torchrun every rank solves its own copy of the problem (independent
slices, no collective: weak scaling).  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import gkb_inputs as gi  # noqa: E402

K_ITERS = 150
VARIANTS = ("BA", "AB")
METRIC = "GKB iterations/s (512x512 fan, 720x725, FP32 projectors + FP64 scalars, k=150, BA+AB)"
PROFILE_CLASSES = ("A", "B", "AT", "BT", "reorth_dots", "reorth_update", "other")


def peaks():
    """(HBM GB/s, maximum SM MHz, which) from MEASURED_PEAKS.json, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2032.0)), "measured"
    except Exception:
        return 6400.0, 2032.0, "fallback"


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or "unknown"


# ---------------------------------------------------------------------------
# algorithmic work of the projectors (non-zeros of A and B), from the geometry

def taps_forward(g) -> int:
    """Non-zeros of Joseph's A: two interpolation taps per image row (or
    column) a ray crosses with at least one neighbour inside the grid."""
    total = 0
    hx, hy = (g.nx - 1) / 2.0, (g.ny - 1) / 2.0
    for a in range(g.n_angles):
        c, s = math.cos(g.angles[a]), math.sin(g.angles[a])
        u = (np.arange(g.n_det) - (g.n_det - 1) / 2.0) * g.det_width
        if g.beam == "parallel":
            px, py = u * c, u * s
            ex, ey = np.full_like(u, -s), np.full_like(u, c)
        else:
            px, py = np.full_like(u, g.sod * c), np.full_like(u, g.sod * s)
            bx, by = -(g.sdd - g.sod) * c - u * s, -(g.sdd - g.sod) * s + u * c
            lx, ly = bx - px, by - py
            L = np.hypot(lx, ly)
            ex, ey = lx / L, ly / L
        rows = np.abs(ey) >= np.abs(ex)
        for mask, (p0, p1, e0, e1, lim, cnt, h0, h1) in (
                (rows, (px, py, ex, ey, g.nx, g.ny, hx, hy)), (~rows, (py, px, ey, ex, g.ny, g.nx, hy, hx))):
            if not mask.any():
                continue
            k = np.arange(cnt)[None, :]
            if mask is rows:
                y = (h1 - k) * g.pixel
                xs = p0[mask, None] + (y - p1[mask, None]) / e1[mask, None] * e0[mask, None]
                f = xs / g.pixel + h0
            else:
                xx = (k - h1) * g.pixel
                ys = p0[mask, None] + (xx - p1[mask, None]) / e1[mask, None] * e0[mask, None]
                f = h0 - ys / g.pixel
            fl = np.floor(f)
            total += int(((fl >= 0) & (fl <= lim - 1)).sum() + ((fl + 1 >= 0) & (fl + 1 <= lim - 1)).sum())
    return total


def taps_back(g) -> int:
    """Non-zeros of the pixel-driven B: two bins per (pixel, angle) pair,
    counting only bins inside the detector."""
    X = ((np.arange(g.nx) - (g.nx - 1) / 2.0) * g.pixel)[None, :]
    Y = (((g.ny - 1) / 2.0 - np.arange(g.ny)) * g.pixel)[:, None]
    total = 0
    for a in range(g.n_angles):
        c, s = math.cos(g.angles[a]), math.sin(g.angles[a])
        if g.beam == "parallel":
            u = X * c + Y * s
        else:
            U = g.sod - (X * c + Y * s)
            u = g.sdd * (-X * s + Y * c) / U
        t = u / g.det_width + (g.n_det - 1) / 2.0
        d = np.floor(t)
        total += int(((d >= 0) & (d <= g.n_det - 1)).sum() + ((d + 1 >= 0) & (d + 1 <= g.n_det - 1)).sum())
    return total


def reorth_bytes(dim: int, k: int, passes: int = 1, elem: int = 4):
    """Algorithmic HBM bytes of the reorthogonalisation over a solve of k iterations: iteration
    j reads the j stored basis vectors and q~ for the dot products, and the j
    vectors plus q~ (read and written) for the update, per pass."""
    ldq = (dim + 7) // 8 * 8
    cols = k * (k + 1) // 2
    dots = passes * (cols + k) * ldq * elem
    update = passes * (cols + 2 * k) * ldq * elem
    return dots, update


def launches_per_solve(variant: str, k: int, reorth: int, a_kernels: int = 2, at_kernels: int = 2,
                       bt_kernels: int = 3) -> int:
    """Kernel launches of one gkb_plan_execute run to k iterations (no early
    stop) when no captured graph can be asked (--no-graph).  The banded A is
    an image transpose plus the band kernel; the scatter A^T is the scatter
    and the kernel that adds its two partial images; the scatter B^T is
    max|x|, the scatter and the finishing kernel."""
    # A^T (and B^T for AB and BA) in the initialisation
    init = {"BA": 5 + at_kernels + bt_kernels, "AB": 4 + at_kernels + bt_kernels, "matched": 4 + at_kernels}[variant]
    proj = {"BA": a_kernels + 1 + at_kernels + bt_kernels, "AB": a_kernels + 1 + at_kernels + bt_kernels,
            "matched": a_kernels + at_kernels}[variant]
    per_iter = proj + 1 + 1 + 3 * reorth + 1 + 1  # projectors, half1, stop check, reorth, half2, advance
    final = 1
    return init + k * per_iter + final


# the FP32 kernels each operator runs on the bench workload (default kernel families)
KERNEL_NAMES = {"A": "k_fwd", "B": "k_back_tile", "AT": "k_fadj_lines", "BT": "k_badj_scatter"}


# ---------------------------------------------------------------------------
# multi-rank timing rules (replicas: every rank solves its own problem)

def rank_max(x: float, dist, device) -> float:
    """The largest value over all ranks (the slowest rank sets the step time);
    x itself when there is one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Units processed by all ranks per second, from the slowest rank's time."""
    return units_per_rank * world / (ms / 1e3)


# ---------------------------------------------------------------------------
# clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, path: str | None):
        self.proc = None
        self.path = path or os.path.join("/tmp", f"gkb_clocks_{os.getpid()}.csv")
        self.index = index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# ---------------------------------------------------------------------------
# the oracle on the host cores (the reference arm and the CPU baseline)

def _oracle_problem(w):
    from oracle.projectors import Projectors
    g = w.geom
    P = Projectors(g)
    b, en = gi.add_noise(P.A(gi.phantom_of(w)), gi.noise_direction(g.m, w.noise_seed), w.eta)
    return P, b, en


def oracle_iteration_seconds(P, b, variant="BA"):
    """Seconds of one FP64 oracle GKB iteration: the initialisation and one
    pass of the loop with the oracle's explicit ||A x - b|| (setup included)."""
    from oracle import gkb as og
    t0 = time.perf_counter()
    og.gkb(variant, P, b, 1)
    return time.perf_counter() - t0


def cpu_baseline(full: bool, c4: bool = False):
    """The FP64 oracle timed on this host: per matrix-vector product (A, B,
    A^T, B^T) and per BA-GKB iteration on the 512 fan workload, and per
    iteration on the 64x64 workload, with one thread and with all threads.
    The headline value is the all-thread BA iteration rate on the 512 fan
    (about 10-30 s of CPU work in total).  With c4 also one matvec per
    operator at 2048^2 on all threads (about a minute more)."""
    from oracle import projectors as op
    nt_all = op.threads()
    out = {"cpu": cpu_model(), "threads_all": nt_all, "per_matvec_s": {}, "per_iteration_s": {}}
    w = gi.fan_512()
    P, b, _ = _oracle_problem(w)
    rng = np.random.default_rng(0)
    x = gi.phantom_of(w)
    y = np.abs(rng.standard_normal(w.geom.m))
    small = gi.small_parallel_64()
    Ps, bs_, _ = _oracle_problem(small)
    try:
        for nt in sorted({1, nt_all}):
            op.set_threads(nt)
            mv = {}
            for name, f, v in (("A", P.A, x), ("B", P.B, y), ("AT", P.AT, y), ("BT", P.BT, x)):
                t0 = time.perf_counter()
                f(v)
                mv[name] = time.perf_counter() - t0
            out["per_matvec_s"][f"{w.name}@{nt}t"] = mv
            if nt == nt_all or full:
                out["per_iteration_s"][f"{w.name}_BA@{nt}t"] = oracle_iteration_seconds(P, b)
            out["per_iteration_s"][f"{small.name}_BA@{nt}t"] = oracle_iteration_seconds(Ps, bs_)
    finally:
        op.set_threads(nt_all)
    if c4:
        # config 4 (2048^2, 1800 x 2897): one matvec per operator on all
        # threads; a BA iteration is about the four of them (the oracle's
        # explicit ||A x - b|| adds one more A)
        w4 = gi.parallel_2048()
        from oracle.projectors import Projectors
        P4 = Projectors(w4.geom)
        x4 = gi.phantom_of(w4)
        y4 = np.abs(rng.standard_normal(w4.geom.m))
        mv4 = {}
        for name, f, v in (("A", P4.A, x4), ("B", P4.B, y4), ("AT", P4.AT, y4), ("BT", P4.BT, x4)):
            t0 = time.perf_counter()
            f(v)
            mv4[name] = time.perf_counter() - t0
        out["per_matvec_s"][f"{w4.name}@{nt_all}t"] = mv4
        out["per_iteration_s"][f"{w4.name}_BA@{nt_all}t_estimate"] = sum(mv4.values()) + mv4["A"]
    it = out["per_iteration_s"][f"{w.name}_BA@{nt_all}t"]
    sample = (f"one FP64 oracle BA-GKB iteration (initialisation and one pass of the loop with its explicit ||Ax-b||) on "
              f"{w.name}, C projectors on {nt_all} threads ({out['cpu']}); per-matvec times at 1 and "
              f"{nt_all} threads and the {small.name} iteration in 'details'")
    return {"value": 1.0 / it, "unit": "iterations/s", "cores": nt_all, "kind": "oracle", "sample": sample,
            "details": out}


def cpu_c3_subset(n_slices: int = 16):
    """The FP64 oracle on the first n_slices slices of the multi-slice
    workload (the bench's batched subset: parallel N in {256..1024}, 180 to
    720 angles, discrepancy principle, k_max 150), every slice solved to its
    stop by BA-GKB one after another on all threads of this host; the
    timed region holds the solves only (problem set-up outside).  Several
    minutes of CPU work: behind its own flag."""
    from oracle import gkb as og
    from oracle import projectors as op
    ws = gi.batch_slices(256)[:n_slices]
    probs = [_oracle_problem(w) for w in ws]
    iters = 0
    t0 = time.perf_counter()
    for P, b, en in probs:
        r = og.gkb("BA", P, b, 150, stop=og.STOP_DP, noise_norm=float(np.linalg.norm(en)))
        iters += int(r["k_stop"])
    dt = time.perf_counter() - t0
    return {"slices": n_slices, "seconds": dt, "slices_per_s": n_slices / dt, "iterations": iters,
            "threads": op.threads(), "cpu": cpu_model(),
            "how": "FP64 oracle BA-GKB with the discrepancy principle (its explicit ||Ax-b|| each iteration), "
                   "slices one after another"}


def run_reference(args, rank):
    """The reference arm: the FP64 oracle (the paper has no released code) on
    the host cores, one BA-GKB iteration of the 512 fan workload per step."""
    if rank != 0:
        return 0
    from oracle import projectors as op
    w = gi.fan_512()
    P, b, _ = _oracle_problem(w)
    secs = [oracle_iteration_seconds(P, b) for _ in range(args.warmup + args.steps)]
    timed = secs[args.warmup:]
    per = statistics.mean(timed)
    value = 1.0 / per
    nt = op.threads()
    sample = (f"one FP64 oracle BA-GKB iteration (initialisation and one pass of the loop with its explicit ||Ax-b||) on "
              f"{w.name}, C projectors on {nt} threads ({cpu_model()})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded ellipse phantom)",
            "config": {"workload": w.name, "variants": ["BA"], "k_per_step": 1},
            "cpu_baseline": {"value": value, "unit": "iterations/s", "cores": nt, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm

def batched_section(gkb, torch, n_slices: int, rank: int):
    """The uneven multi-slice workload (the first n_slices of the 256-slice
    recipe: N in {256, 384, 512, 768, 1024}, 180/360/720 angles, ceil(sqrt(2) N)
    bins, noise 0.5-5 %, discrepancy principle, k_max 150): plain single-slice
    FP32 solves one after another against one batched graph launch in FP32,
    with 16-bit projector operands (FP32 Krylov vectors) and with FP16
    storage throughout; slices/s, iterations, and each batch's largest
    relative iterate difference from the plain FP32 solves (the criterion is
    1e-3)."""
    ws = gi.batch_slices(256)[:n_slices]
    geoms, bs, ens = [], [], []
    for w in ws:
        G = gkb.Geometry(w.geom)
        x = torch.tensor(gi.phantom_of(w), dtype=torch.float32, device="cuda")
        bt = G.A(x).double().cpu().numpy()
        b, en = gi.add_noise(bt, gi.noise_direction(w.geom.m, w.noise_seed + 10000 * rank), w.eta)
        geoms.append(G)
        bs.append(torch.tensor(b, dtype=torch.float32, device="cuda"))
        ens.append(en)
    sizes = {}
    for w in ws:
        key = f"{w.geom.nx}x{w.geom.n_angles}"
        sizes[key] = sizes.get(key, 0) + 1
    out = {"slices": n_slices, "workload": "parallel N in {256..1024}, 180/360/720 angles, DP stop, k_max 150",
           "mix": sizes}
    plans = [gkb.Plan(G, variant="BA", k_max=150, stop="dp", noise_norm=en) for G, en in zip(geoms, ens)]
    for P, b in zip(plans, bs):
        P.execute(b)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [P.execute(b) for P, b in zip(plans, bs)]
    torch.cuda.synchronize()
    out["plain_slices_per_s"] = n_slices / (time.perf_counter() - t0)
    out["plain_iterations"] = int(sum(r.k_stop for r in plain))
    for P in plans:
        P.close()
    modes = {"f32": dict(storage=gkb.F32), "f32_bf16_operands": dict(storage=gkb.F32, operands=gkb.BF16),
             "f32_f16_operands": dict(storage=gkb.F32, operands=gkb.F16), "f16": dict(storage=gkb.F16)}
    for name, kw in modes.items():
        B = gkb.Batch(geoms, [dict(variant="BA", k_max=150, stop="dp", noise_norm=en, **kw) for en in ens])
        B.execute(bs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, res = B.execute(bs)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        diffs = [float(torch.linalg.norm(r.x - q.x) / torch.linalg.norm(q.x)) for r, q in zip(res, plain)]
        kd = [abs(r.k_stop - q.k_stop) for r, q in zip(res, plain)]
        out[f"batched_{name}_slices_per_s"] = n_slices / dt
        out[f"batched_{name}_max_rel_diff_vs_plain"] = max(diffs)
        out[f"batched_{name}_median_rel_diff_vs_plain"] = float(np.median(diffs))
        out[f"batched_{name}_iterations"] = int(sum(r.k_stop for r in res))
        out[f"batched_{name}_k_dp_max_shift"] = int(max(kd))
        B.close()
        if name != "f32":
            # the same storage mode stopped at each slice's plain discrepancy
            # index: the iterate difference from precision alone, without the
            # shift of the stopping index
            B = gkb.Batch(geoms, [dict(variant="BA", k_max=q.k_stop, stop="none", noise_norm=en, **kw)
                                  for q, en in zip(plain, ens)])
            st, res = B.execute(bs)
            d_same = [float(torch.linalg.norm(r.x - q.x) / torch.linalg.norm(q.x)) for r, q in zip(res, plain)]
            out[f"batched_{name}_same_k_max_rel_diff_vs_plain"] = max(d_same)
            out[f"batched_{name}_same_k_median_rel_diff_vs_plain"] = float(np.median(d_same))
            out[f"batched_{name}_same_k_within_1e-3"] = float(np.mean(np.array(d_same) <= 1e-3))
            B.close()
    # the learned stop trained on the 256 fan, applied to this multi-geometry
    # batch (outside its training distribution; the discrepancy fallback guards it)
    from paper_2606_31153_b300 import learned
    if os.path.exists(learned.DEFAULT_WEIGHTS):
        mlp = learned.load()
        B = gkb.Batch(geoms, [dict(variant="BA", k_max=150, stop="learned", noise_norm=en) for en in ens])
        _, rl, li = B.execute_learned(mlp, bs)
        xt = [gi.phantom_of(w) for w in ws]
        rre_p = [float(np.linalg.norm(q.x.double().cpu().numpy() - x) / np.linalg.norm(x)) for q, x in zip(plain, xt)]
        rre_l = [float(np.linalg.norm(r.x.double().cpu().numpy() - x) / np.linalg.norm(x)) for r, x in zip(rl, xt)]
        out["learned_fan256_weights"] = {
            "accepted_fraction": float(np.mean([d["fallback"] == 0 for d in li])),
            "rre_plain_mean": float(np.mean(rre_p)), "rre_learned_mean": float(np.mean(rre_l)),
            "improved_fraction": float(np.mean(np.array(rre_l) < np.array(rre_p))),
            "iters_plain": int(sum(q.k_stop for q in plain)), "iters_learned": int(sum(r.k_stop for r in rl))}
        B.close()
    return out


def learned_section(torch, n: int):
    """Learned stopping against the plain discrepancy principle on held-out
    problems of the training geometry (256 fan)."""
    from paper_2606_31153_b300 import learned
    if not os.path.exists(learned.DEFAULT_WEIGHTS):
        return None
    return learned.evaluate(learned.load(), n=n)


def timed_solves(torch, plan, b, reps):
    """Device milliseconds per solve of a captured plan (CUDA events on the stream)."""
    stream = torch.cuda.current_stream()
    plan.execute(b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        res = plan.execute(b)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps, res


def matched_section(gkb, torch, G, b, reps):
    """The matched pair B = A^T run as plain GKB (Algorithm 3) on the same
    problem and iteration count: iterations/s against BA/AB on this GPU."""
    plan = gkb.Plan(G, variant="matched", k_max=K_ITERS, stop="none", reorth=1, storage=gkb.F32)
    ms, res = timed_solves(torch, plan, b, reps)
    outer, body = plan.kernel_counts()
    plan.close()
    return {"iterations_per_s": K_ITERS / (ms / 1e3), "ms_per_solve": ms, "k": K_ITERS,
            "kernels_per_iteration": body, "kernels_outside_loop": outer}


def gmres_section(gkb, torch, G, b, reps):
    """The paper's comparison methods (Algorithms 1-2) on the same problem and
    iteration count: AB- and BA-GMRES (full Arnoldi, two classical
    Gram-Schmidt passes), iterations/s against AB/BA-GKB on this GPU."""
    out = {}
    for v in ("AB-GMRES", "BA-GMRES"):
        plan = gkb.Plan(G, variant=v, k_max=K_ITERS, stop="none", reorth=2, storage=gkb.F32)
        ms, res = timed_solves(torch, plan, b, reps)
        outer, body = plan.kernel_counts()
        plan.close()
        out[v] = {"iterations_per_s": K_ITERS / (ms / 1e3), "ms_per_solve": ms, "k": res.k_stop,
                  "kernels_per_iteration": body, "kernels_outside_loop": outer}
    return out


def small_section(gkb, torch, reps):
    """The 64x64 parallel workload (90 angles, 91 bins, 10 ellipses, 1 % noise)
    in FP64, AB- and BA-GKB with the discrepancy principle (k_max 30): a
    latency- and launch-bound case; iterations/s and kernels per iteration."""
    w = gi.small_parallel_64()
    G = gkb.Geometry(w.geom)
    x = torch.tensor(gi.phantom_of(w), dtype=torch.float64, device="cuda")
    bt = G.A(x).cpu().numpy()
    b_np, en = gi.add_noise(bt, gi.noise_direction(w.geom.m, w.noise_seed), w.eta)
    b = torch.tensor(b_np, dtype=torch.float64, device="cuda")
    out = {"workload": w.name, "dtype": "f64"}
    for v in VARIANTS:
        plan = gkb.Plan(G, variant=v, k_max=w.k_max, stop="dp", noise_norm=en, storage=gkb.F64)
        ms, res = timed_solves(torch, plan, b, reps)
        outer, body = plan.kernel_counts()
        out[v] = {"k_dp": res.k_stop, "ms_per_solve": ms, "iterations_per_s": res.k_stop / (ms / 1e3),
                  "kernels_per_iteration": body, "kernels_outside_loop": outer,
                  "us_per_kernel": 1e3 * ms / (outer + res.k_stop * body)}
        plan.close()
    G.close()
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2606_31153_b300 as gkb

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    w = gi.fan_512()
    g = w.geom
    G = gkb.Geometry(g)
    # data with the library's own forward projector (rank-specific phantom seed: independent slices)
    x_true = torch.tensor(gi.ellipse_phantom(g.nx, w.n_ellipses, w.phantom_seed + 1000 * rank), dtype=torch.float32,
                          device=dev)
    b_true = G.A(x_true).double().cpu().numpy()
    b_np, en = gi.add_noise(b_true, gi.noise_direction(g.m, w.noise_seed + 1000 * rank), w.eta)
    b = torch.tensor(b_np, dtype=torch.float32, device=dev)
    plans = {v: gkb.Plan(G, variant=v, k_max=K_ITERS, stop="none", reorth=1, storage=gkb.F32, use_graph=not args.no_graph)
             for v in VARIANTS}
    xs = {v: torch.empty(g.n, dtype=torch.float32, device=dev) for v in VARIANTS}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step_seq(bb, xo):
        res = {}
        for v in VARIANTS:
            res[v] = plans[v].execute(bb, xo[v])
        return res

    # the step: both solves as one two-slice batched launch (one graph, a
    # chain per solve), so BA and AB overlap -- one solve's small kernels and
    # each projector's last wave share the GPU with the other's work; with
    # --no-graph (profilers) the solves run one after another by direct launches
    pair = None if args.no_graph else gkb.Batch(
        [G, G], [dict(variant=v, k_max=K_ITERS, stop="none", reorth=1, storage=gkb.F32) for v in VARIANTS])

    def step(bb, xo):
        if pair is None:
            return step_seq(bb, xo)
        _, rs = pair.execute([bb, bb], [xo[v] for v in VARIANTS])
        return dict(zip(VARIANTS, rs))

    def timed(fn, xo, nvtx=False):
        out, last_res = [], None
        for _ in range(args.steps):
            flush.fill_(1.0)  # evict L2 (126 MB) between timed steps; not timed
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if nvtx:
                torch.cuda.nvtx.range_push("bench_timed_step")   # lets a profiler select the timed kernels
            e0.record(stream)
            last_res = fn(b, xo)
            e1.record(stream)
            if nvtx:
                torch.cuda.nvtx.range_pop()
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return out, last_res

    for _ in range(max(args.warmup, 0)):
        step(b, xs)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank, os.environ.get("GKB_CLOCKS_CSV"))
    clocks.start()
    times, last = timed(step, xs, nvtx=True)
    torch.cuda.synchronize()
    ck = clocks.stop()
    if dist:
        dist.barrier()
    ms = rank_max(sum(times) / len(times), dist, dev)
    iters_per_step = K_ITERS * len(VARIANTS)
    value = whole_job_rate(iters_per_step, world, ms)

    # the same solves one after another (single-solve plans), for comparison
    if pair is not None:
        xseq = {v: torch.empty(g.n, dtype=torch.float32, device=dev) for v in VARIANTS}
        step_seq(b, xseq)
        torch.cuda.synchronize()
        seq_times, _ = timed(step_seq, xseq)
        seq_ms = sum(seq_times) / len(seq_times)
        sequential = {"iterations_per_s": iters_per_step / (seq_ms / 1e3), "ms_per_step": seq_ms,
                      "bitwise_equal_to_the_step": bool(all(torch.equal(xseq[v], xs[v]) for v in VARIANTS)),
                      "how": "BA then AB, each one gkb_plan_execute (one graph per solve)"}
    else:
        sequential = {"iterations_per_s": value, "ms_per_step": ms, "how": "the step itself (--no-graph)"}

    # end to end through the public API from pinned host memory: the data's
    # host-to-device copy, the step, the two iterates' device-to-host copies
    bh = b.cpu().pin_memory()
    xh = {v: torch.empty(g.n, dtype=torch.float32).pin_memory() for v in VARIANTS}
    bd = torch.empty_like(b)

    def step_e2e():
        bd.copy_(bh, non_blocking=True)
        step(bd, xs)
        for v in VARIANTS:
            xh[v].copy_(xs[v], non_blocking=True)
        stream.synchronize()

    step_e2e()
    e2e_times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step_e2e()
        e2e_times.append(time.perf_counter() - t0)
    e2e_ms = rank_max(1e3 * sum(e2e_times) / len(e2e_times), dist, dev)
    e2e_value = whole_job_rate(iters_per_step, world, e2e_ms)
    if pair is not None:
        pair.close()

    # per-kernel times of the projectors (standalone launches on the same stream, CUDA events)
    rng = np.random.default_rng(0)
    xin = torch.tensor(rng.random(g.n), dtype=torch.float32, device=dev)
    yin = torch.tensor(rng.random(g.m), dtype=torch.float32, device=dev)
    xo, yo = torch.empty_like(xin), torch.empty_like(yin)
    ops = {"A": (G.A, xin, yo), "B": (G.B, yin, xo), "AT": (G.AT, yin, xo), "BT": (G.BT, xin, yo)}
    kt = {}
    for name, (f, i, o) in ops.items():
        for _ in range(3):
            f(i, out=o)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_rep = 20
        e0.record(stream)
        for _ in range(n_rep):
            f(i, out=o)
        e1.record(stream)
        e1.synchronize()
        kt[name] = e0.elapsed_time(e1) / n_rep

    # the same solves with an event between kernel groups: time per kernel class
    prof = {c: 0.0 for c in PROFILE_CLASSES}
    groups = {c: 0 for c in PROFILE_CLASSES}
    for v in VARIANTS:
        for c, (t_ms, n_g) in plans[v].profile(b).items():
            prof[c] += t_ms
            groups[c] += n_g
    prof_total = sum(prof.values())

    hbm, sm_max, peak_kind = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    nnzA, nnzB = taps_forward(g), taps_back(g)
    taps = {"A": nnzA, "AT": nnzA, "B": nnzB, "BT": nnzB}
    # the projectors' binding ceiling: one 4-byte shared-memory word per lane
    # per clock, i.e. 32 matrix non-zeros per SM per clock at the maximum clock
    ceiling_nz = sms * 32 * sm_max * 1e6
    ceiling_gbs = ceiling_nz * 4 / 1e9
    per_kernel = {}
    for k in ("A", "B", "AT", "BT"):
        nz_s = taps[k] / (kt[k] * 1e-3)
        per_kernel[k] = {"kernel": KERNEL_NAMES[k], "ms_per_launch": kt[k], "nonzeros": taps[k],
                         "nonzeros_per_s": nz_s, "frac_gather_ceiling": nz_s / ceiling_nz,
                         "ms_per_launch_in_solve": prof[k] / max(groups[k], 1),
                         "share_of_solve": prof[k] / prof_total}
    dims = {"BA": g.n, "AB": g.m}
    d_bytes = sum(reorth_bytes(dims[v], K_ITERS)[0] for v in VARIANTS)
    u_bytes = sum(reorth_bytes(dims[v], K_ITERS)[1] for v in VARIANTS)
    for cls, nbytes in (("reorth_dots", d_bytes), ("reorth_update", u_bytes)):
        gbs = nbytes / (prof[cls] * 1e-3) / 1e9
        per_kernel[cls] = {"kernel": {"reorth_dots": "k_dots + k_dots_reduce", "reorth_update": "k_update"}[cls],
                           "ms_per_solve_pair": prof[cls], "algorithmic_bytes": nbytes, "achieved_gbs": gbs,
                           "frac_hbm": gbs / hbm, "share_of_solve": prof[cls] / prof_total}
    per_kernel["other"] = {"ms_per_solve_pair": prof["other"], "share_of_solve": prof["other"] / prof_total}
    dom = max(("A", "B", "AT", "BT"), key=lambda k: prof[k])
    # DRAM bytes per launch of the dominant kernel from the last ncu capture,
    # only while the kernel sources are those the counters were taken from
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        try:
            import hashlib
            rec = json.load(open(tp))
            csrc = os.path.join(ROOT, "paper_2606_31153_b300", "csrc")
            src = open(os.path.join(csrc, "projectors_fast.cu"), "rb").read() + open(os.path.join(csrc, "common.cuh"), "rb").read()
            if rec.get("source_sha1") == hashlib.sha1(src).hexdigest():
                traffic = rec["dram_bytes_per_launch"].get(KERNEL_NAMES[dom])
        except Exception:
            traffic = None
    achieved_gbs = 4 * taps[dom] / (kt[dom] * 1e-3) / 1e9
    fp32_peak_tflops = sms * 128 * 2 * sm_max * 1e6 / 1e12
    roof = {"bound": "smem", "achieved": achieved_gbs, "peak": ceiling_gbs, "unit": "GB/s",
            "frac": achieved_gbs / ceiling_gbs, "traffic": traffic, "kernel": KERNEL_NAMES[dom], "operator": dom,
            "peak_kind": f"derived: {sms} SMs x 32 lanes x 4 B x {sm_max:.0f} MHz (shared-memory gather ceiling)",
            "algorithmic_bytes_per_launch": 4 * taps[dom],
            "note": ("algorithmic bytes = 4 B per matrix non-zero (one shared-memory word per interpolation tap); "
                     "frac = non-zeros/s / (SMs x 32 x max SM clock). The FP32 FMA view: "
                     f"{2 * taps[dom] / (kt[dom] * 1e-3) / 1e12:.2f} TFLOP/s of {fp32_peak_tflops:.1f} derived "
                     "(2 flops per non-zero); HBM moves about (n+m) x 4 B per launch, far below its roofline")}

    matched = matched_section(gkb, torch, G, b, max(args.steps, 2)) if not args.no_extras else None
    gmres = gmres_section(gkb, torch, G, b, max(args.steps, 2)) if not args.no_extras else None
    small = small_section(gkb, torch, max(args.steps, 3)) if not args.no_extras else None
    batched = batched_section(gkb, torch, args.batch_slices, rank) if args.batch_slices > 0 else None
    learned_eval = learned_section(torch, args.learned_n) if (args.learned_n > 0 and rank == 0) else None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_full, args.cpu_c4)
    if args.no_graph:
        launches = sum(launches_per_solve(v, K_ITERS, 1) for v in VARIANTS) * args.steps
    else:   # kernel nodes of each captured graph: outside the loop + k x one iteration
        launches = 0
        for v in VARIANTS:
            outer, body = plans[v].kernel_counts()
            launches += (outer + last[v].k_stop * body) * args.steps
    ref_rre = float(torch.linalg.norm(last["BA"].x.double() - x_true.double()) / torch.linalg.norm(x_true.double()))
    line = {"metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded 30-ellipse phantom, 2 % noise)",
            "config": {"workload": w.name, "variants": list(VARIANTS), "k_per_solve": K_ITERS,
                       "iterations_per_step": iters_per_step, "reorth": "CGS, 1 pass", "scalars": "f64",
                       "graph": ("direct launches, BA then AB" if args.no_graph else
                                 "BA and AB as one two-slice batched graph launch (a WHILE-node chain per solve)"),
                       "l2": "flushed (256 MB write) before each step",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e_value, "unit": "iterations/s", "h2d_bytes_per_step": g.m * 4,
                    "d2h_bytes_per_step": len(VARIANTS) * g.n * 4},
            "gpu_launches": launches,
            "roofline": roof,
            "per_kernel": per_kernel,
            "profile_ms_per_step": prof,
            "hbm_peak_gbs": hbm, "peak_kind": peak_kind, "sms": sms,
            "rre_BA_k150": ref_rre,
            "clocks": ck,
            "sequential_BA_then_AB": sequential,
            "matched": matched,
            "gmres": gmres,
            "small_f64": small,
            "batched": batched,
            "learned_stop": learned_eval,
            "cpu_baseline": cpu}
    if rank == 0:
        print(json.dumps(line), flush=True)
    for p in plans.values():
        p.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-full", action="store_true", help="also time the 512 fan oracle iteration on one thread")
    ap.add_argument("--cpu-c4", action="store_true", help="also time the oracle's matvecs at 2048^2 (about a minute)")
    ap.add_argument("--cpu-c3", action="store_true",
                    help="only time the oracle's DP-stopped solves of the 16-slice batch subset on this host "
                         "(no GPU; tens of minutes) and print them as one JSON line")
    ap.add_argument("--no-extras", action="store_true", help="skip the matched-pair and 64x64 FP64 sections")
    ap.add_argument("--batch-slices", type=int, default=16, help="slices of the multi-slice workload (0: skip)")
    ap.add_argument("--learned-n", type=int, default=64, help="held-out problems for the learned stop (0: skip)")
    ap.add_argument("--no-graph", action="store_true", help="launch kernels directly (profilers cannot see kernels inside graphs with conditional nodes)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.cpu_c3:
        if rank == 0:
            print(json.dumps({"cpu_c3_subset": cpu_c3_subset()}), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args, rank)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
