"""The predictor's device kernels against the FP64 oracle: forward pass,
gradients (<= 1e-4 relative), Adam steps, BF16 inference."""
import numpy as np
import pytest

from oracle import mlp as om
from tests.gpu_helpers import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gkb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_31153_b300 as m
    return m


def _setup(gkb, B=37, seed=3):
    rng = np.random.default_rng(seed)
    theta = om.init_params(seed) + 0.02 * rng.standard_normal(om.n_params())
    X = rng.standard_normal((B, 64))
    T = rng.standard_normal((B, 2))
    net = gkb.MLP()
    net.set_params(theta.astype(np.float32))
    th32 = theta.astype(np.float32).astype(np.float64)  # the parameters the device holds
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    Td = torch.tensor(T, dtype=torch.float32, device="cuda")
    return net, th32, X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64), Xd, Td


def test_forward_and_gradient_match_oracle(gkb):
    net, th, X, T, Xd, Td = _setup(gkb)
    Y = net.forward(Xd).double().cpu().numpy()
    assert rel(Y, om.forward(th, X)[0]) <= 1e-5
    g, loss = net.gradient(Xd, Td)
    assert rel(g.double().cpu().numpy(), om.gradient(th, X, T)) <= 1e-4
    assert abs(float(loss) - om.loss(th, X, T)) <= 1e-5 * om.loss(th, X, T)


def test_adam_steps_match_oracle(gkb):
    net, th, X, T, Xd, Td = _setup(gkb, B=64, seed=5)
    m, v = np.zeros_like(th), np.zeros_like(th)
    for step in (1, 2, 3):
        net.train_step(Xd, Td, lr=1e-3)
        th, m, v = om.adam_step(th, m, v, om.gradient(th, X, T), step, lr=1e-3)
    got, _ = net.get_params()
    assert rel(got.astype(np.float64), th) <= 1e-5


def test_bf16_inference_close_to_fp64(gkb):
    net, th, X, T, Xd, Td = _setup(gkb, B=50, seed=7)
    Y = net.forward(Xd, bf16=True).double().cpu().numpy()
    assert rel(Y, om.forward(th, X)[0]) <= 3e-2


def test_training_reduces_loss_deterministically(gkb):
    rng = np.random.default_rng(0)
    X = rng.standard_normal((256, 64)).astype(np.float32)
    W = rng.standard_normal((64, 2)).astype(np.float32) / 8
    T = np.tanh(X @ W)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    losses = []
    for _ in range(2):
        net = gkb.MLP()
        net.set_params(om.init_params(1).astype(np.float32))
        loss = torch.zeros(1, device="cuda")
        hist = []
        for _ in range(200):
            net.train_step(Xd, Td, lr=3e-3, loss=loss)
            hist.append(float(loss))
        losses.append(hist)
    assert losses[0] == losses[1]
    assert losses[0][-1] < 0.1 * losses[0][0]
