"""AB-GMRES and BA-GMRES (Algorithms 1-2) on the device against the FP64 oracle."""
import numpy as np
import pytest

import gkb_inputs as gi
from oracle import gkb as og
from oracle import gmres as gm
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


# odd angle counts: no four-fold symmetry, so the spectra have no degenerate
# pairs and the iterations are well determined by the data
GEOMS = {
    "parallel64_a91": lambda: gi.parallel_geometry(64, 91, 91),
    "fan64_a91": lambda: gi.fan_geometry(64, 91, 91, 128.0, 256.0),
}


def _data(g, seed=1, eta=0.02):
    P = Projectors(g)
    x = gi.rasterize(gi.ellipse_params(min(g.nx, g.ny), 10, seed), g.nx, g.ny)
    b, en = gi.add_noise(P.A(x), gi.noise_direction(g.m, seed + 100), eta)
    return P, x, b, en


@pytest.mark.parametrize("gname", list(GEOMS))
@pytest.mark.parametrize("variant", ["AB", "BA"])
def test_fp64_gmres_matches_oracle(gname, variant):
    """FP64: the Hessenberg entries, the data residuals and the iterate after
    25 iterations, with two classical Gram-Schmidt passes against the
    oracle's modified Gram-Schmidt."""
    g = GEOMS[gname]()
    P, x, b, en = _data(g)
    k = 25
    ref = gm.gmres(variant, P, b, k)
    res = gkb.solve(gkb.Geometry(g), to_dev(b, torch.float64), variant=f"{variant}-GMRES", k_max=k, reorth=2,
                    storage=gkb.F64)
    assert res.k_stop == k and res.reason == "k_max"
    H = ref["H"]
    assert rel(res.alpha, np.diag(H)[:k]) <= 1e-10
    assert rel(res.t[1:], np.diag(H, -1)[:k]) <= 1e-10
    assert abs(res.t[0] - ref["beta"]) <= 1e-12 * ref["beta"]
    assert rel(res.resid, ref["resid"]) <= 1e-10
    assert rel(to_np(res.x), ref["x"]) <= 1e-9


@pytest.mark.parametrize("gname", list(GEOMS))
@pytest.mark.parametrize("variant", ["AB", "BA"])
def test_fp32_gmres_discrepancy_stop(gname, variant):
    """FP32 storage, the discrepancy principle: the same stopping index as the
    oracle (or one off where the oracle's residual is within 1e-6 of the
    threshold), and the iterate within 1e-3."""
    g = GEOMS[gname]()
    P, x, b, en = _data(g, eta=0.03)
    ref = gm.gmres(variant, P, b, 40, stop="dp", noise_norm=en)
    res = gkb.solve(gkb.Geometry(g), to_dev(b, torch.float32), variant=f"{variant}-GMRES", k_max=40, reorth=2,
                    stop="dp", noise_norm=en, storage=gkb.F32)
    kd = ref["k_stop"]
    margin = np.abs(ref["resid"][max(kd - 2, 0):kd] / en - 1.0).min()
    assert res.k_stop == kd or (abs(res.k_stop - kd) == 1 and margin <= 1e-6)
    ref_at = gm.gmres(variant, P, b, res.k_stop)
    assert rel(to_np(res.x), ref_at["x"]) <= 1e-3


def test_gmres_stops_earlier_than_gkb_on_the_same_data():
    """The paper's observation (Sec. 5): with the discrepancy principle the
    GMRES variants stop earlier than the GKB variants on the same data; the
    device shows the same ordering as the oracle."""
    g = gi.fan_geometry(64, 91, 91, 128.0, 256.0)
    P, x, b, en = _data(g, seed=3, eta=0.04)
    G = gkb.Geometry(g)
    bd = to_dev(b, torch.float64)
    k = {}
    for v in ("AB", "BA", "AB-GMRES", "BA-GMRES"):
        r = gkb.solve(G, bd, variant=v, k_max=60, reorth=2 if "GMRES" in v else 1, stop="dp", noise_norm=en,
                      storage=gkb.F64)
        k[v] = r.k_stop
    ko = {"AB-GMRES": gm.gmres("AB", P, b, 60, stop="dp", noise_norm=en)["k_stop"],
          "BA-GMRES": gm.gmres("BA", P, b, 60, stop="dp", noise_norm=en)["k_stop"],
          "AB": og.gkb("AB", P, b, 60, stop="dp", noise_norm=en)["k_stop"],
          "BA": og.gkb("BA", P, b, 60, stop="dp", noise_norm=en)["k_stop"]}
    assert k == ko
    assert k["AB-GMRES"] <= k["AB"] and k["BA-GMRES"] <= k["BA"]


def test_gmres_in_a_batch():
    """GMRES slices inside a batched graph return what single solves return,
    bit for bit."""
    g = gi.fan_geometry(64, 91, 91, 128.0, 256.0)
    P, x, b, en = _data(g)
    G = gkb.Geometry(g)
    bd = to_dev(b, torch.float32)
    params = [dict(variant=v, k_max=30, reorth=2, stop="dp", noise_norm=en) for v in ("AB-GMRES", "BA-GMRES", "BA")]
    single = [gkb.solve(G, bd, **p) for p in params]
    _, batch = gkb.solve_batched([G] * 3, [bd] * 3, params=params)
    for a, c in zip(single, batch):
        assert a.k_stop == c.k_stop
        assert torch.equal(a.x, c.x)
