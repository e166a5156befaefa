"""Batched solves: every slice of one graph launch equals the same slice solved
alone (bit for bit: each slice runs the same deterministic kernels on its own
workspace), and slices agree with the FP64 oracle."""
import numpy as np
import pytest

import gkb_inputs as gi
from oracle import gkb as og
from oracle.projectors import Projectors
from tests.gpu_helpers import rel, to_dev, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

gkb = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global gkb
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_31153_b300 as m
    gkb = m


def _slices(n, seed=7):
    """An uneven batch with the recipe of the multi-slice workload, scaled down:
    N in {32, 48, 64, 80}, angles in {31, 45, 61} over [0, 180), bins
    ceil(sqrt(2) N), 3-8 ellipses, noise U[0.5 %, 5 %]."""
    ws = gi.scaled_batch_slices(n, sizes=[32, 48, 64, 80], angles=[31, 45, 61], seed=seed, k_max=40)
    out = []
    for w in ws:
        P = Projectors(w.geom)
        x = gi.phantom_of(w)
        b, en = gi.add_noise(P.A(x), gi.noise_direction(w.geom.m, w.noise_seed), w.eta)
        out.append((w, P, x, b, en))
    return out


@pytest.mark.parametrize("variant", ["BA", "AB"])
def test_batch_equals_individual_solves(variant):
    data = _slices(9)
    geoms = [gkb.Geometry(w.geom) for w, *_ in data]
    bs = [to_dev(b, torch.float32) for *_, b, _ in data]
    params = [dict(variant=variant, k_max=40, stop="dp", noise_norm=en) for *_, en in data]
    batch = gkb.Batch(geoms, params)
    st, res = batch.execute(bs)
    for i, (G, b, p) in enumerate(zip(geoms, bs, params)):
        one = gkb.solve(G, b, **p)
        assert res[i].k_stop == one.k_stop and res[i].reason == one.reason
        assert torch.equal(res[i].x, one.x)
        assert np.array_equal(res[i].resid, one.resid)
    # a second launch of the same graph gives the same answers
    st2, res2 = batch.execute(bs)
    assert all(torch.equal(a.x, b2.x) for a, b2 in zip(res, res2))
    batch.close()


def test_batched_slices_match_oracle():
    data = _slices(4, seed=11)
    geoms = [gkb.Geometry(w.geom) for w, *_ in data]
    bs = [to_dev(b, torch.float64) for *_, b, _ in data]
    st, res = gkb.solve_batched(geoms, bs, variant="BA", k_max=25, storage=gkb.F64)
    for (w, P, x, b, en), r in zip(data, res):
        ref = og.gkb("BA", P, b, 25)
        assert r.k_stop == 25
        assert rel(to_np(r.x), ref["x"]) <= 1e-6
        assert rel(r.resid, ref["resid"]) <= 1e-8
