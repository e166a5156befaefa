"""Learned stopping inside the batched BA-GKB solver."""
import os

import numpy as np
import pytest

import gkb_inputs as gi
from oracle import gkb as og
from oracle import mlp as om
from oracle.projectors import Projectors
from tests.gpu_helpers import rel, to_dev, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gkb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_31153_b300 as m
    return m


def _problems(n=4):
    """Fan beam without four-fold symmetry (91 angles) so the FP32 solver
    tracks the FP64 oracle iteration by iteration."""
    g = gi.fan_geometry(64, 91, 91, 128.0, 256.0)
    P = Projectors(g)
    out = []
    for i in range(n):
        rng = np.random.default_rng(50 + i)
        x = gi.ellipse_phantom(64, int(rng.integers(5, 12)), 60 + i)
        b, en = gi.add_noise(P.A(x), gi.noise_direction(g.m, 70 + i), float(rng.uniform(0.005, 0.02)))
        out.append((x, b, en))
    return g, P, out


def _oracle_labels(P, b, en, k_run, delta=8):
    ref = og.gkb("BA", P, b, k_run)
    kdp = og.dp_index(ref["resid"], en)
    k = kdp + delta
    Cd = og.lower_bidiagonal(ref["alpha"], ref["t"], kdp)
    rhs = np.zeros(kdp + 1)
    rhs[0] = ref["t"][0]
    target = np.linalg.norm(Cd @ og.solve_projected_svd(Cd, ref["t"][0]) - rhs)
    C = og.lower_bidiagonal(ref["alpha"], ref["t"], k)
    r0 = np.zeros(k + 1)
    r0[0] = ref["t"][0]
    lo, hi = np.log(ref["alpha"][0] * 1e-9), np.log(ref["alpha"][0] * 10)
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        r = np.linalg.norm(C @ og.tikhonov_projected(C, ref["t"][0], np.exp(mid)) - r0)
        lo, hi = (lo, mid) if r > target else (mid, hi)
    return kdp, 0.5 * (lo + hi)


def test_training_labels_match_oracle(gkb):
    g, P, probs = _problems(3)
    G = gkb.Geometry(g)
    bs = [to_dev(b, torch.float32) for _, b, _ in probs]
    batch = gkb.Batch([G] * 3, [dict(variant="BA", k_max=60, stop="none", noise_norm=en) for *_, en in probs])
    batch.execute(bs)
    X, T, V = batch.training_data()
    for i, (x, b, en) in enumerate(probs):
        kdp, loglam = _oracle_labels(P, b, en, 60)
        assert int(V[i]) == 1
        assert abs(float(T[i, 0]) - np.log(kdp)) < 1e-6
        assert abs(float(T[i, 1]) - loglam) <= 1e-3
        assert torch.isfinite(X[i]).all()


def test_learned_batch_hybrid_and_fallback(gkb):
    g, P, probs = _problems(4)
    G = gkb.Geometry(g)
    bs = [to_dev(b, torch.float32) for _, b, _ in probs]
    ens = [en for *_, en in probs]
    net = gkb.MLP()
    net.set_params(om.init_params(2).astype(np.float32))   # untrained: predictions are arbitrary
    learned = gkb.Batch([G] * 4, [dict(variant="BA", k_max=60, stop="learned", noise_norm=en) for en in ens])
    plain = gkb.Batch([G] * 4, [dict(variant="BA", k_max=60, stop="dp", noise_norm=en) for en in ens])
    _, rl, li = learned.execute_learned(net, bs)
    _, rp = plain.execute(bs)
    for i, (x, b, en) in enumerate(probs):
        assert li[i]["k_dp"] == rp[i].k_stop            # the discrepancy index is tracked exactly
        assert rl[i].k_stop >= max(17, li[i]["k_dp"])
        if li[i]["fallback"] == 1:                      # rejected: the discrepancy-principle iterate, bit for bit
            assert torch.equal(rl[i].x, rp[i].x)
        elif li[i]["fallback"] == 0:                    # accepted: x = Q_k u_lambda, within 5 % of tau ||e||
            k, lam = rl[i].k_stop, li[i]["lam"]
            ref = og.gkb("BA", P, b, k, keep_bases=True)
            C = og.lower_bidiagonal(ref["alpha"], ref["t"], k)
            xr = ref["Q"][:, :k] @ og.tikhonov_projected(C, ref["t"][0], lam)
            assert rel(to_np(rl[i].x), xr) <= 1e-3
            assert abs(li[i]["hybrid_resid"] - en) <= 0.05 * en


def test_trained_predictor_gains_over_plain_dp(gkb):
    """With the committed trained weights: on held-out problems of the training
    geometry, the learned mode's iterate is closer to the phantom than the
    plain discrepancy-principle iterate, on average."""
    from paper_2606_31153_b300 import learned
    if not os.path.exists(learned.DEFAULT_WEIGHTS):
        pytest.skip("no trained weights")
    res = learned.evaluate(learned.load(), n=32)
    print(res)
    assert res["accepted_fraction"] >= 0.5
    assert res["rre_learned_mean"] < res["rre_plain_mean"]
