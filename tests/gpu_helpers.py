"""Shared helpers of the GPU parity tests (not collected as a test module)."""
import numpy as np

import gkb_inputs as gi


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(v, dtype):
    import torch
    return torch.as_tensor(np.asarray(v, dtype=np.float64)).to(device="cuda", dtype=dtype).contiguous()


def to_np(t):
    return t.detach().to("cpu", dtype=__import__("torch").float64).numpy()


def small_fan(N=96, na=120, nd=None):
    nd = nd if nd is not None else int(np.ceil(np.sqrt(2) * N))
    return gi.fan_geometry(N, na, nd, 2.0 * N, 4.0 * N)


def problem(w_or_geom, n_ell=6, seed=1, eta=0.02, oracle=None):
    """(x_true, b, ||e||) with b computed by the FP64 oracle."""
    g = w_or_geom
    x = gi.ellipse_phantom(g.nx, n_ell, seed, g.pixel) if g.nx == g.ny else gi.rasterize(
        gi.ellipse_params(min(g.nx, g.ny), n_ell, seed, g.pixel), g.nx, g.ny, g.pixel)
    bt = oracle.A(x)
    b, en = gi.add_noise(bt, gi.noise_direction(g.m, seed + 100), eta)
    return x, b, en
