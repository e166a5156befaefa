"""Learned stopping for BA-GKB: training data from the solver, training on the
device, evaluation against the plain discrepancy principle.

    python -m paper_2606_31153_b300.learned train --n 20000 --out paper_2606_31153_b300/learned_stop.npz
    python -m paper_2606_31153_b300.learned evaluate --weights paper_2606_31153_b300/learned_stop.npz --n 64

Training problems: the 512 fan geometry scaled to 256x256 (SOD 512, SDD 1024,
363 bins, 720 angles over 360 degrees), seeded phantoms of 5-40 ellipses,
noise levels U[0.5 %, 5 %].  Each problem is solved by the batched BA-GKB
solver without a stopping rule; the solver's own kernels extract the
features of the first 16 iterations and the labels (log k_DP, log lambda*),
and the network is trained by the library's forward/backward/Adam kernels.
Everything numeric runs on the GPU; this module only orchestrates.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gkb_inputs as gi  # noqa: E402

DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "learned_stop.npz")
N_PARAMS = 256 * 64 + 256 + 256 * 256 + 256 + 2 * 256 + 2


def init_params(seed: int) -> np.ndarray:
    """Kaiming-uniform weights (bound sqrt(6 / fan_in)), zero biases, flat layout W1 b1 W2 b2 W3 b3."""
    rng = np.random.default_rng(seed)
    parts = []
    for rows, cols in ((256, 64), (256, 256), (2, 256)):
        b = math.sqrt(6.0 / cols)
        parts.append(rng.uniform(-b, b, size=rows * cols))
        parts.append(np.zeros(rows))
    return np.concatenate(parts).astype(np.float32)


def problem_set(n: int, seed0: int):
    """(n_ellipses, eta, phantom seed, noise seed) of n training or test problems."""
    rng = np.random.default_rng(seed0)
    return [(int(rng.integers(5, 41)), float(rng.uniform(0.005, 0.05)), seed0 + 10 * i + 1, seed0 + 10 * i + 2)
            for i in range(n)]


def make_data(G, geom, probs):
    """Phantoms, data b = A x + e (A: the library's projector) and ||e||."""
    import torch
    xs, bs, ens = [], [], []
    for ne, eta, ps, ns in probs:
        x = gi.ellipse_phantom(geom.nx, ne, ps)
        xt = torch.tensor(x, dtype=torch.float32, device="cuda")
        bt = G.A(xt).double().cpu().numpy()
        b, en = gi.add_noise(bt, gi.noise_direction(geom.m, ns), eta)
        xs.append(x)
        bs.append(torch.tensor(b, dtype=torch.float32, device="cuda"))
        ens.append(en)
    return xs, bs, ens


def generate(n: int, seed0: int = 1_000_000, chunk: int = 64, k_max: int = 100, log=print):
    """Features, labels of n training solves (only the labelled ones are kept)."""
    import torch

    import paper_2606_31153_b300 as gkb
    geom = gi.fan_256_training().geom
    G = gkb.Geometry(geom)
    probs = problem_set(n, seed0)
    Xs, Ts = [], []
    t0 = time.time()
    for c0 in range(0, n, chunk):
        part = probs[c0:c0 + chunk]
        _, bs, ens = make_data(G, geom, part)
        batch = gkb.Batch([G] * len(part), [dict(variant="BA", k_max=k_max, stop="none", noise_norm=en) for en in ens])
        batch.execute(bs)
        X, T, V = batch.training_data()
        torch.cuda.synchronize()
        keep = V.bool()
        Xs.append(X[keep])
        Ts.append(T[keep])
        batch.close()
        log(f"  solves {min(c0 + chunk, n)}/{n}, labelled {int(sum(x.shape[0] for x in Xs))}, {time.time() - t0:.0f} s")
    return torch.cat(Xs), torch.cat(Ts)


def train(X, T, epochs: int = 200, batch: int = 256, lr: float = 1e-3, seed: int = 0, val_frac: float = 0.1,
          patience: int = 15, log=print):
    """Train on standardised features/targets with the library's Adam step,
    with early stopping on a held-out validation split: the weights of the
    epoch with the lowest validation loss are kept, and training ends after
    `patience` epochs without improvement.  Returns (mlp, norm, report)."""
    import torch

    import paper_2606_31153_b300 as gkb
    n = X.shape[0]
    gen = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(n, generator=gen).to(X.device)
    nv = max(1, int(val_frac * n))
    iv, it = perm[:nv], perm[nv:]
    mu_x, sd_x = X[it].mean(0), X[it].std(0).clamp_min(1e-3)
    mu_t, sd_t = T[it].mean(0), T[it].std(0).clamp_min(1e-3)
    Xs, Ts = ((X - mu_x) / sd_x).contiguous(), ((T - mu_t) / sd_t).contiguous()
    norm = torch.cat([mu_x, sd_x, mu_t, sd_t]).cpu().numpy().astype(np.float32)
    mlp = gkb.MLP()
    mlp.set_params(init_params(seed), norm)
    loss = torch.zeros(1, device=X.device)
    hist = []
    best = (float("inf"), -1, None)
    batch = min(batch, int(it.numel()))
    Xv, Tv = Xs[iv].contiguous(), Ts[iv].contiguous()
    for ep in range(epochs):
        order = it[torch.randperm(it.numel(), generator=gen).to(X.device)]
        tot = 0.0
        nb = 0
        for b0 in range(0, order.numel() - batch + 1, batch):
            idx = order[b0:b0 + batch]
            mlp.train_step(Xs[idx].contiguous(), Ts[idx].contiguous(), lr=lr, loss=loss)
            tot += float(loss)
            nb += 1
        yv = mlp.forward(Xv)
        vloss = float(0.5 * ((yv - Tv) ** 2).sum(1).mean())
        hist.append((tot / max(nb, 1), vloss))
        if vloss < best[0]:
            best = (vloss, ep, mlp.get_params()[0])
        if ep % 10 == 0 or ep == epochs - 1:
            log(f"  epoch {ep}: train {tot / max(nb, 1):.4f} val {vloss:.4f}")
        if ep - best[1] >= patience:
            log(f"  early stop at epoch {ep}: best validation loss {best[0]:.4f} at epoch {best[1]}")
            break
    mlp.set_params(best[2], norm)
    # train and validation error of the kept weights, in the original units
    yt = mlp.forward(Xs[it].contiguous())
    train_loss = float(0.5 * ((yt - Ts[it]) ** 2).sum(1).mean())
    y = mlp.forward(Xv) * sd_t + mu_t
    k_err = (torch.exp(y[:, 0]) - torch.exp(T[iv, 0])).abs()
    lam_err = (y[:, 1] - T[iv, 1]).abs()
    report = {"train_samples": int(it.numel()), "val_samples": int(nv), "epochs_run": len(hist),
              "best_epoch": best[1], "train_loss": train_loss, "val_loss": best[0],
              "val_k_abs_err_mean": float(k_err.mean()), "val_k_within_2": float((k_err <= 2).float().mean()),
              "val_loglambda_abs_err_mean": float(lam_err.mean())}
    return mlp, norm, report


def save(path, mlp, norm, report):
    theta, _ = mlp.get_params()
    np.savez(path, theta=theta, norm=norm, report=json.dumps(report))


def load(path=DEFAULT_WEIGHTS):
    import paper_2606_31153_b300 as gkb
    z = np.load(path)
    mlp = gkb.MLP()
    mlp.set_params(z["theta"], z["norm"])
    return mlp


def evaluate(mlp, n: int = 64, seed0: int = 9_000_000, k_max: int = 120):
    """Held-out problems: the learned batch against the plain discrepancy principle."""
    import torch

    import paper_2606_31153_b300 as gkb
    geom = gi.fan_256_training().geom
    G = gkb.Geometry(geom)
    probs = problem_set(n, seed0)
    xs, bs, ens = make_data(G, geom, probs)
    plain = gkb.Batch([G] * n, [dict(variant="BA", k_max=k_max, stop="dp", noise_norm=en) for en in ens])
    learned = gkb.Batch([G] * n, [dict(variant="BA", k_max=k_max, stop="learned", noise_norm=en) for en in ens])
    plain.execute(bs)
    learned.execute_learned(mlp, bs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, rp = plain.execute(bs)
    t_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, rl, li = learned.execute_learned(mlp, bs)
    t_learned = time.perf_counter() - t0

    def rre(x, xt):
        return float(np.linalg.norm(x.double().cpu().numpy() - xt) / np.linalg.norm(xt))
    rre_p = np.array([rre(r.x, x) for r, x in zip(rp, xs)])
    rre_l = np.array([rre(r.x, x) for r, x in zip(rl, xs)])
    k_p = np.array([r.k_stop for r in rp])
    k_l = np.array([r.k_stop for r in rl])
    khat = np.array([d["k_hat"] for d in li])
    fb = np.array([d["fallback"] for d in li])
    out = {"n": n, "rre_plain_mean": float(rre_p.mean()), "rre_learned_mean": float(rre_l.mean()),
           "rre_ratio_mean": float((rre_l / rre_p).mean()), "improved_fraction": float((rre_l < rre_p).mean()),
           "iters_plain_mean": float(k_p.mean()), "iters_learned_mean": float(k_l.mean()),
           "k_hat_abs_err_mean": float(np.abs(khat - k_p).mean()), "k_hat_within_2": float((np.abs(khat - k_p) <= 2).mean()),
           "accepted_fraction": float((fb == 0).mean()), "fallback_fraction": float((fb != 0).mean()),
           "seconds_plain": t_plain, "seconds_learned": t_learned}
    plain.close()
    learned.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("train")
    a.add_argument("--n", type=int, default=20000)
    a.add_argument("--epochs", type=int, default=200)
    a.add_argument("--seed", type=int, default=0)
    a.add_argument("--out", default=DEFAULT_WEIGHTS)
    a.add_argument("--eval-n", type=int, default=256)
    e = sub.add_parser("evaluate")
    e.add_argument("--weights", default=DEFAULT_WEIGHTS)
    e.add_argument("--n", type=int, default=64)
    args = ap.parse_args(argv)
    if args.cmd == "train":
        X, T = generate(args.n)
        mlp, norm, report = train(X, T, epochs=args.epochs, seed=args.seed)
        report["solves"] = args.n
        report["labelled"] = int(X.shape[0])
        save(args.out, mlp, norm, report)
        print(json.dumps(report), flush=True)
        print(json.dumps(evaluate(mlp, n=args.eval_n)), flush=True)
    else:
        print(json.dumps(evaluate(load(args.weights), n=args.n)))


if __name__ == "__main__":
    main()
