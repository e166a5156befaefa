"""Time the four projectors of one workload through the C ABI.

    python -m paper_2606_31153_b300.kernel_bench --workload fan512 --ops A,B,AT,BT --reps 20

Prints one line per operator: milliseconds per launch (CUDA events on the
launch stream, after warm-up launches) and the matrix non-zeros it applies per
second.  Used for per-kernel measurements and for profiler captures of a
single projector.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gkb_inputs as gi  # noqa: E402

WORKLOADS = {
    "parallel64": gi.small_parallel_64,
    "fan512": gi.fan_512,
    "parallel2048": gi.parallel_2048,
    "fan256": gi.fan_256_training,
}
DTYPES = {"f32": "float32", "bf16": "bfloat16", "f16": "float16", "f64": "float64"}


def main(argv=None):
    import torch

    import paper_2606_31153_b300 as gkb

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="fan512", choices=sorted(WORKLOADS))
    ap.add_argument("--ops", default="A,B,AT,BT")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--dtype", default="f32", choices=sorted(DTYPES))
    ap.add_argument("--no-tune", action="store_true", help="keep the default kernel shapes")
    ap.add_argument("--gather", action="store_true", help="run the transposes by the gather kernels")
    ap.add_argument("--shapes", default="", help="pin the kernel shapes of A,B,AT,BT (e.g. 2,2,0,2) instead of tuning")
    args = ap.parse_args(argv)
    w = WORKLOADS[args.workload]()
    g = w.geom
    G = gkb.Geometry(g)
    if args.gather:
        G.use_scatter(False)
    if args.shapes:
        G.set_shapes([int(v) for v in args.shapes.split(",")])
    elif not args.no_tune and args.dtype != "f64":
        G.autotune({"f32": gkb.F32, "bf16": gkb.BF16, "f16": gkb.F16}[args.dtype])
    dt = getattr(torch, DTYPES[args.dtype])
    rng = np.random.default_rng(0)
    x = torch.tensor(rng.random(g.n), device="cuda").to(dt)
    y = torch.tensor(rng.random(g.m), device="cuda").to(dt)
    xo, yo = torch.empty_like(x), torch.empty_like(y)
    table = {"A": (G.A, x, yo), "B": (G.B, y, xo), "AT": (G.AT, y, xo), "BT": (G.BT, x, yo)}
    stream = torch.cuda.current_stream()
    out = {}
    for op in args.ops.split(","):
        f, i, o = table[op]
        for _ in range(args.warmup):
            f(i, out=o)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.reps):
            f(i, out=o)
        e1.record(stream)
        e1.synchronize()
        out[op] = e0.elapsed_time(e1) / args.reps
    print(json.dumps({"workload": w.name, "dtype": args.dtype, "transposes": "gather" if args.gather else "scatter", "shapes": G.shapes()[0],
                      "ms_per_launch": out}))


if __name__ == "__main__":
    main()
