"""Semiconvergence and stopping rules of AB-, BA- and matched GKB.

    python -m paper_2606_31153_b300.semiconvergence --noise 0.04,0.07,0.10 --k 120

For one seeded synthetic problem per noise level (the paper's levels: 4, 7
and 10 % noise, Sec. 5) BA and matched GKB run to k_max with every iterate kept
(``gkb_solve_iterates``; AB's iterates are sampled by separate solves); the relative reconstruction error of each iterate
(Eq. RE) is computed on the device.  Printed, as one JSON line: per noise
level and variant the RRE curve at sampled k, the optimal index and its RRE,
the discrepancy-principle index (Eq. DP, tau = 1) with its RRE, and the
residual-norm-stagnation index (Eq. RNS) for a few tolerances with its RRE.
The stopping indices come from the same residual history the device
recurrences produce; the rules themselves are the solver's (``stop=dp`` and
``stop=rns`` give the same indices, which the test suite checks).
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


def problem(N: int, n_angles: int, eta: float, beam: str, seed: int):
    """Seeded phantom and geometry of the paper's size range (Sec. 5: 128^2-256^2
    images, 65-256 angles): parallel over 180 degrees or a flat fan over 360."""
    if beam == "parallel":
        g = gi.parallel_geometry(N, n_angles)
    else:
        g = gi.fan_geometry(N, n_angles, int(np.ceil(np.sqrt(2) * N)), 2.0 * N, 4.0 * N)
    w = gi.Workload(f"{beam}{N}_a{n_angles}", g, 20, seed, seed + 100, eta, 0)
    return w, g


def rns_index(res: np.ndarray, eps: float) -> int:
    """First k >= 2 with |r_{k-1} - r_k| < eps r_{k-1} (1-based), else len(res)."""
    for k in range(2, len(res) + 1):
        if abs(res[k - 2] - res[k - 1]) < eps * res[k - 2]:
            return k
    return len(res)


def main(argv=None):
    import torch

    import paper_2606_31153_b300 as gkb
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=256)
    ap.add_argument("--angles", type=int, default=180)
    ap.add_argument("--beam", default="parallel", choices=["parallel", "fan"])
    ap.add_argument("--noise", default="0.04,0.07,0.10")
    ap.add_argument("--k", type=int, default=120)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--rns", default="1e-2,5e-3,1e-3")
    args = ap.parse_args(argv)
    etas = [float(v) for v in args.noise.split(",")]
    rns_eps = [float(v) for v in args.rns.split(",")]
    out = {"N": args.N, "angles": args.angles, "beam": args.beam, "k_max": args.k, "levels": []}
    for eta in etas:
        w, g = problem(args.N, args.angles, eta, args.beam, args.seed)
        G = gkb.Geometry(g)
        x_true = gi.phantom_of(w)
        xt = torch.tensor(x_true, dtype=torch.float32, device="cuda")
        b_true = G.A(xt).double().cpu().numpy()
        b, en = gi.add_noise(b_true, gi.noise_direction(g.m, w.noise_seed), eta)
        bd = torch.tensor(b, dtype=torch.float32, device="cuda")
        level = {"eta": eta, "snr_db": gi.snr_db(eta), "variants": {}}
        for variant in ("AB", "BA", "matched"):
            if variant == "AB":
                # AB's iterate is B applied to a sinogram-space vector, which the
                # iterate recorder does not keep: one solve per sampled k instead
                res = gkb.solve(G, bd, variant=variant, k_max=args.k, stop="none", noise_norm=en, storage=gkb.F32)
                k_run = res.k_stop
                rre = np.full(k_run, np.inf)
                for k in sorted(set([1, 2, 3] + list(range(5, k_run + 1, 5)))):
                    rk = gkb.solve(G, bd, variant=variant, k_max=k, stop="none", noise_norm=en, storage=gkb.F32)
                    rre[k - 1] = float(torch.linalg.norm(rk.x - xt) / torch.linalg.norm(xt))
            else:
                res, X = gkb.solve_iterates(G, bd, variant=variant, k_max=args.k, stop="none", noise_norm=en,
                                            storage=gkb.F32)
                k_run = res.k_stop
                rre = (torch.linalg.norm(X[:k_run] - xt[None, :], dim=1) / torch.linalg.norm(xt)).cpu().numpy()
            resid = np.asarray(res.resid[:k_run], dtype=np.float64)
            k_opt = int(np.argmin(rre)) + 1
            dp = [k for k in range(1, k_run + 1) if resid[k - 1] <= en]
            k_dp = dp[0] if dp else None
            entry = {"k_run": k_run, "k_opt": k_opt, "rre_opt": float(rre[k_opt - 1]),
                     "k_dp": k_dp, "rre_dp": float(rre[k_dp - 1]) if k_dp else None,
                     "rns": {str(e): {"k": rns_index(resid, e), "rre": float(rre[rns_index(resid, e) - 1])}
                             for e in rns_eps},
                     "rre_curve": {str(k): float(rre[k - 1]) for k in range(5, k_run + 1, 5)}}
            if variant == "AB":   # the sampled curve only: report the stopping indices' RRE where sampled
                entry["note"] = "RRE sampled at k = 1, 2, 3 and every 5th k"
                for key in ("rre_dp",):
                    if entry[key] is not None and not np.isfinite(entry[key]):
                        entry[key] = None
            level["variants"][variant] = entry
        out["levels"].append(level)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
