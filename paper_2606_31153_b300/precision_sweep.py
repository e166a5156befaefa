"""Storage-precision study of BA-GKB: the Krylov vectors and projector
operands stored as FP32, BF16 or FP16, or FP32 Krylov vectors with 16-bit
projector operands (FP32 accumulation in the projectors, FP64 scalars),
against the FP64 path, iteration by iteration.

    python -m paper_2606_31153_b300.precision_sweep --workload parallel512 --k 200
    python -m paper_2606_31153_b300.precision_sweep --workload parallel2048 --k 200 --reference f32

Prints one JSON line: per storage type the relative difference
||x_k - x_k^ref|| / ||x_k^ref|| at sampled k, the relative reconstruction
error against the phantom (Eq. RE), the discrepancy-principle index, and the
time per iteration.  The FP64 reference path is itself checked against the
FP64 CPU oracle by the test suite.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gkb_inputs as gi  # noqa: E402

WORKLOADS = {
    # the 2048 precision-sweep workload and a reduced copy the FP64 path finishes quickly;
    # the 451-angle copy has no four-fold symmetry (no degenerate singular-value pairs)
    "parallel2048": gi.parallel_2048,
    "parallel512": lambda: gi.Workload("parallel512_a450_d725", gi.parallel_geometry(512, 450, 725), 50, 4, 104, 0.01, 200),
    "parallel512_a451": lambda: gi.Workload("parallel512_a451_d725", gi.parallel_geometry(512, 451, 725), 50, 4, 104,
                                            0.01, 200),
}
# storage of the Krylov vectors and type of the projector operands
MODES = {"f64": ("F64", "F64"), "f32": ("F32", "F32"), "bf16": ("BF16", "BF16"), "f16": ("F16", "F16"),
         "f32+bf16": ("F32", "BF16"), "f32+f16": ("F32", "F16")}


def main(argv=None):
    import torch

    import paper_2606_31153_b300 as gkb
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="parallel512", choices=sorted(WORKLOADS))
    ap.add_argument("--k", type=int, default=200)
    ap.add_argument("--reference", default="f64", choices=["f64", "f32"])
    ap.add_argument("--every", type=int, default=10)
    ap.add_argument("--modes", default="f32,bf16,f16,f32+bf16,f32+f16",
                    help="storage[+operand type] of the compared runs")
    args = ap.parse_args(argv)
    w = WORKLOADS[args.workload]()
    g = w.geom
    G = gkb.Geometry(g)
    x_true = gi.phantom_of(w)
    xt = torch.tensor(x_true, dtype=torch.float64, device="cuda")
    b_true = G.A(xt).cpu().numpy()
    b, en = gi.add_noise(b_true, gi.noise_direction(g.m, w.noise_seed), w.eta)
    ks = sorted(set(list(range(args.every, args.k + 1, args.every)) + [1, 5]))
    runs = {}
    order = [args.reference] + [m for m in args.modes.split(",") if m != args.reference]
    ref_X = None
    for name in order:
        storage, operands = (getattr(gkb, c) for c in MODES[name])
        dt = torch.float64 if name == "f64" else torch.float32
        bd = torch.tensor(b, dtype=dt, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            res, X = gkb.solve_iterates(G, bd, variant="BA", k_max=args.k, storage=storage, operands=operands)
            status = res.status
        except gkb.GKBError as e:
            runs[name] = {"status": e.status, "error": str(e)}
            continue
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        kk = res.k_stop
        rre = {k: float(torch.linalg.norm(X[k - 1].double() - xt) / torch.linalg.norm(xt)) for k in ks if k <= kk}
        entry = {"status": int(status), "k_stop": kk, "ms_per_iteration": 1e3 * secs / max(kk, 1),
                 "k_dp": next((i + 1 for i, r in enumerate(res.resid) if r <= en), None), "rre": rre}
        if ref_X is None:
            ref_X = X.double()
        else:
            entry["rel_diff_vs_" + args.reference] = {
                k: float(torch.linalg.norm(X[k - 1].double() - ref_X[k - 1]) / torch.linalg.norm(ref_X[k - 1]))
                for k in ks if k <= kk}
        runs[name] = entry
        del X
        torch.cuda.empty_cache()
    print(json.dumps({"workload": w.name, "reference": args.reference, "k": args.k, "noise_norm": en, "runs": runs}))


if __name__ == "__main__":
    main()
