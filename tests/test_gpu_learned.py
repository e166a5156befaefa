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
    """(k_DP, lambda*) of one problem from the FP64 oracle's BA-GKB run."""
    ref = og.gkb("BA", P, b, k_run)
    kdp = og.dp_index(ref["resid"], en)
    return kdp, float(np.log(og.tikhonov_label(ref["alpha"], ref["t"], kdp, delta)))


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


def _constant_net(gkb, log_k, log_lam):
    """A predictor whose output is the given (log k, log lambda) for every
    input: zero weights and biases, the targets' means set to the outputs."""
    net = gkb.MLP()
    norm = np.zeros(132, dtype=np.float32)
    norm[64:128] = 1.0
    norm[128:130] = (log_k, log_lam)
    norm[130:132] = 1.0
    net.set_params(np.zeros(net.n_params, dtype=np.float32), norm)
    return net


def test_learned_batch_hybrid_and_fallback(gkb):
    """The two outcomes of the learned stop.  Accepted: a predictor that
    returns the oracle's own labels (k_DP and lambda*) drives each slice to
    k_DP + 8 and the projected Tikhonov step; at least one slice must pass the
    5 % discrepancy check, and every accepted iterate equals the oracle's
    Q_k u_lambda to 1e-3.  Rejected: an untrained network's arbitrary
    prediction, where every fallback returns the discrepancy-principle iterate
    bit for bit."""
    g, P, probs = _problems(4)
    G = gkb.Geometry(g)
    ens = [en for *_, en in probs]
    accepted = 0
    for i, (x, b, en) in enumerate(probs):
        kdp, loglam = _oracle_labels(P, b, en, 60)
        net = _constant_net(gkb, float(np.log(kdp)), loglam)
        bs = [to_dev(b, torch.float32)]
        learned = gkb.Batch([G], [dict(variant="BA", k_max=60, stop="learned", noise_norm=en)])
        plain = gkb.Batch([G], [dict(variant="BA", k_max=60, stop="dp", noise_norm=en)])
        _, rl, li = learned.execute_learned(net, bs)
        _, rp = plain.execute(bs)
        li, rl, rp = li[0], rl[0], rp[0]
        assert li["k_dp"] == rp.k_stop == kdp            # the discrepancy index is tracked exactly
        assert li["k_hat"] == kdp and abs(np.log(li["lam"]) - loglam) <= 1e-2
        assert rl.k_stop == max(kdp + 8, 17)            # at least the 16 observed iterations + 1
        if li["fallback"] == 0:                          # accepted: x = Q_k u_lambda, within 5 % of tau ||e||
            accepted += 1
            k, lam = rl.k_stop, li["lam"]
            ref = og.gkb("BA", P, b, k, keep_bases=True)
            C = og.lower_bidiagonal(ref["alpha"], ref["t"], k)
            xr = ref["Q"][:, :k] @ og.tikhonov_projected(C, ref["t"][0], lam)
            assert rel(to_np(rl.x), xr) <= 1e-3
            assert abs(li["hybrid_resid"] - en) <= 0.05 * en
            assert abs(np.linalg.norm(P.A(xr) - b) - en) <= 0.05 * en
        else:
            assert torch.equal(rl.x, rp.x)
    assert accepted >= 1
    # an untrained network: arbitrary predictions, fallbacks bit for bit
    net = gkb.MLP()
    net.set_params(om.init_params(2).astype(np.float32))
    bs = [to_dev(b, torch.float32) for _, b, _ in probs]
    learned = gkb.Batch([G] * 4, [dict(variant="BA", k_max=60, stop="learned", noise_norm=en) for en in ens])
    plain = gkb.Batch([G] * 4, [dict(variant="BA", k_max=60, stop="dp", noise_norm=en) for en in ens])
    _, rl, li = learned.execute_learned(net, bs)
    _, rp = plain.execute(bs)
    for i in range(4):
        assert li[i]["k_dp"] == rp[i].k_stop
        assert rl[i].k_stop >= max(17, li[i]["k_dp"])
        if li[i]["fallback"] == 1:
            assert torch.equal(rl[i].x, rp[i].x)


def test_trained_predictor_gains_over_plain_dp(gkb):
    """With the committed trained weights (20k training solves, early
    stopping on a validation split): on held-out problems of the training
    geometry the predicted index is within 2 of the discrepancy index for
    almost every problem, the prediction is accepted by the 5 % discrepancy
    check, and the learned iterate is closer to the phantom than the plain
    discrepancy-principle iterate on almost every problem -- bought with the
    8 extra iterations the method runs past the predicted index."""
    from paper_2606_31153_b300 import learned
    if not os.path.exists(learned.DEFAULT_WEIGHTS):
        pytest.skip("no trained weights")
    res = learned.evaluate(learned.load(), n=64)
    print(res)
    assert res["k_hat_within_2"] >= 0.9
    assert res["accepted_fraction"] >= 0.9
    assert res["improved_fraction"] >= 0.9
    assert res["rre_learned_mean"] < res["rre_plain_mean"]
    assert res["iters_learned_mean"] <= res["iters_plain_mean"] + 8 + 2
