"""Parity of the CUDA AB-/BA-/matched GKB solver with the FP64 oracle."""
import numpy as np
import pytest

import gkb_inputs as gi
from oracle import gkb as og
from oracle.projectors import Projectors
from tests.gpu_helpers import problem, rel, small_fan, to_dev, to_np

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


def tie_ok(k_gpu, resid_oracle, en, k_oracle, tau=1.0):
    """Identical stopping index, or a tie: the oracle's residual at k_DP or
    k_DP-1 lies within 1e-6 relative of tau ||e||."""
    if k_gpu == k_oracle:
        return True
    thr = tau * en
    near = [k for k in (k_oracle, k_oracle - 1) if 1 <= k <= len(resid_oracle)
            and abs(resid_oracle[k - 1] - thr) <= 1e-6 * thr]
    return bool(near) and k_gpu in (k_oracle, k_oracle - 1)


# Geometries without the four-fold rotational symmetry of the workload
# geometries (an odd number of angles): their GKB sequences are well
# conditioned, so every alpha_k, t_k and iterate can be compared tightly.
NONDEG = {
    "parallel64_a91": lambda: gi.parallel_geometry(64, 91, 91),
    "fan64_a91": lambda: gi.fan_geometry(64, 91, 91, 128.0, 256.0),
    "fanarc64_a91": lambda: gi.fan_geometry(64, 91, 91, 128.0, 256.0, detector="arc"),
}


def _data(g, seed=1, eta=0.01):
    P = Projectors(g)
    x = gi.rasterize(gi.ellipse_params(min(g.nx, g.ny), 10, seed), g.nx, g.ny)
    b, en = gi.add_noise(P.A(x), gi.noise_direction(g.m, seed + 100), eta)
    return P, x, b, en


@pytest.mark.parametrize("gname", list(NONDEG))
@pytest.mark.parametrize("variant", ["AB", "BA", "matched"])
def test_fp64_histories_match_oracle(gname, variant):
    g = NONDEG[gname]()
    P, x, b, en = _data(g)
    k = 40
    ref = og.gkb(variant, P, b, k)
    res = gkb.solve(gkb.Geometry(g), to_dev(b, torch.float64), variant=variant, k_max=k, storage=gkb.F64)
    assert res.k_stop == k and res.reason == "k_max"
    assert rel(res.alpha, ref["alpha"][:k]) <= 1e-10
    assert rel(res.t, ref["t"][:k + 1]) <= 1e-10
    assert rel(res.resid, ref["resid"]) <= 1e-10
    assert rel(to_np(res.x), ref["x"]) <= 1e-9


class _PerturbedOps:
    """The oracle's operators with every output perturbed by a seeded random
    vector of relative norm eps: a solve whose projector applications each
    carry an error of that size."""

    def __init__(self, P, eps, seed):
        self.P, self.eps, self.rng = P, eps, np.random.default_rng(seed)

    def _p(self, y):
        g = self.rng.standard_normal(y.size)
        return y + self.eps * np.linalg.norm(y) * g / np.linalg.norm(g)

    def A(self, x):
        return self._p(self.P.A(x))

    def B(self, y):
        return self._p(self.P.B(y))

    def AT(self, y):
        return self._p(self.P.AT(y))

    def BT(self, x):
        return self._p(self.P.BT(x))


def _fp32_envelope(P, b, variant, k, eps=1e-6, seeds=(1, 2, 3), floor=2e-5):
    """How far an FP32 solve may move the scalar histories from the FP64
    oracle: the oracle rerun with its vectors stored in FP32 (og.gkb's
    storage model) and every projector application perturbed by eps relative
    (the FP32 per-matrix-vector error level measured against the oracle on
    these geometries, 1e-7 - 1e-6), the running maximum of the relative
    spread over a few seeds.  The recurrences amplify such errors at a rate
    set by the spectrum (on the arc-detector fan by orders of magnitude late
    in the run), which a fixed bound cannot follow.  Returns (reference,
    envelopes of alpha, t and ||A x_k - b|| per iteration)."""
    ref = og.gkb(variant, P, b, k)
    runs = [og.gkb(variant, _PerturbedOps(P, eps, s), b, k, storage=np.float32) for s in seeds]
    env = []
    for key, n in (("alpha", k), ("t", k + 1), ("resid", k)):
        spread = np.max([np.abs(r[key][:n] - ref[key][:n]) / np.abs(ref[key][:n]) for r in runs], axis=0)
        env.append(np.maximum(floor, np.maximum.accumulate(spread)))
    return (ref, *env)


@pytest.mark.parametrize("gname", list(NONDEG))
@pytest.mark.parametrize("variant", ["AB", "BA", "matched"])
def test_fp32_histories_match_oracle(gname, variant):
    """FP32 storage against the FP64 oracle over 40 iterations: the iterate to
    1e-3, and alpha_k, t_k and ||A x_k - b|| element by element within the
    envelope of an FP32-storage oracle run whose projector applications each
    carry a 1e-6 relative error (_fp32_envelope): the recurrences amplify
    rounding at a rate set by the spectrum, so a fixed bound would be either
    loose early or wrong late."""
    g = NONDEG[gname]()
    P, x, b, en = _data(g)
    k = 40
    ref, env_a, env_t, env_r = _fp32_envelope(P, b, variant, k)
    res = gkb.solve(gkb.Geometry(g), to_dev(b, torch.float32), variant=variant, k_max=k, storage=gkb.F32)
    assert res.k_stop == k
    da = np.abs(res.alpha - ref["alpha"][:k]) / np.abs(ref["alpha"][:k])
    dt = np.abs(res.t - ref["t"][:k + 1]) / np.abs(ref["t"][:k + 1])
    dr = np.abs(res.resid - ref["resid"]) / np.abs(ref["resid"])
    print(f"{gname} {variant}: max alpha dev {da.max():.2e} (envelope max {env_a.max():.2e}), "
          f"t {dt.max():.2e}, resid {dr.max():.2e}")
    assert np.all(da <= env_a), (np.argmax(da - env_a), da.max())
    assert np.all(dt <= env_t)
    assert np.all(dr <= env_r)
    assert rel(to_np(res.x), ref["x"]) <= 1e-3


@pytest.mark.parametrize("variant", ["AB", "BA", "matched"])
def test_parallel64_workload_fp64_dp(variant):
    """The 64x64 parallel workload (90 angles over [0,180), 91 bins, 10
    ellipses, 1 % noise, FP64, 30 iterations, discrepancy principle).  Its
    geometry is invariant under 90-degree rotation, so M has degenerate
    singular-value pairs and alpha_k, t_k beyond k ~ 15 depend on rounding
    (the oracle itself moves by ~1e-5 under a 1e-15 change of b); the
    comparison is on the stopping index (tie rule), on the first twelve
    alpha_k and t_k, and on the iterate."""
    w = gi.small_parallel_64()
    g = w.geom
    P = Projectors(g)
    x_true = gi.phantom_of(w)
    b, en = gi.add_noise(P.A(x_true), gi.noise_direction(g.m, w.noise_seed), w.eta)
    ref = og.gkb(variant, P, b, w.k_max, stop="dp", noise_norm=en)
    full = og.gkb(variant, P, b, w.k_max)
    res = gkb.solve(gkb.Geometry(g), to_dev(b, torch.float64), variant=variant, k_max=w.k_max, stop="dp",
                    noise_norm=en, storage=gkb.F64)
    assert tie_ok(res.k_stop, full["resid"], en, ref["k_stop"])
    assert res.reason == ref["reason"]
    k = min(res.k_stop, 12)
    assert rel(res.alpha[:k], ref["alpha"][:k]) <= 1e-10
    assert rel(res.t[:k], ref["t"][:k]) <= 1e-10
    if res.k_stop == ref["k_stop"]:
        assert rel(to_np(res.x), ref["x"]) <= 1e-3


@pytest.mark.parametrize("variant", ["AB", "BA"])
def test_fan_fp32_iterate_at_k100_and_dp_index(variant):
    """Fan beam shaped like the 512 workload (SOD 2N, SDD 4N, bins ceil(sqrt(2)N))
    at 96x96 with 121 angles over 360 degrees: FP32 projectors with FP64
    scalars, iterate relative difference <= 1e-3 at k = 100 and the oracle's
    discrepancy-principle index (tie rule)."""
    g = small_fan(96, 121)
    P = Projectors(g)
    x_true, b, en = problem(g, n_ell=8, seed=2, eta=0.02, oracle=P)
    ref = og.gkb(variant, P, b, 100)
    G = gkb.Geometry(g)
    bd = to_dev(b, torch.float32)
    res = gkb.solve(G, bd, variant=variant, k_max=100, storage=gkb.F32)
    assert res.k_stop == 100
    assert rel(to_np(res.x), ref["x"]) <= 1e-3
    k_dp = og.dp_index(ref["resid"], en)
    dp = gkb.solve(G, bd, variant=variant, k_max=100, stop="dp", noise_norm=en, storage=gkb.F32)
    assert k_dp is not None and tie_ok(dp.k_stop, ref["resid"], en, k_dp)
    margin = np.min(np.abs(ref["resid"] / en - 1.0))
    print(f"{variant}: k_DP={k_dp} gpu={dp.k_stop} margin={margin:.3e}")


@pytest.mark.parametrize("variant", ["AB", "BA"])
def test_fan_symmetric_geometry_iterate_at_k100(variant):
    """The same fan problem with 120 angles (four-fold symmetric, like the
    720-angle workload): degenerate singular-value pairs make the k = 100
    iterate depend on rounding, so FP32 against FP64 is compared at 1e-2."""
    g = small_fan(96, 120)
    P = Projectors(g)
    x_true, b, en = problem(g, n_ell=8, seed=2, eta=0.02, oracle=P)
    ref = og.gkb(variant, P, b, 100)
    res = gkb.solve(gkb.Geometry(g), to_dev(b, torch.float32), variant=variant, k_max=100, storage=gkb.F32)
    err = rel(to_np(res.x), ref["x"])
    print(f"{variant}: symmetric fan, k=100 iterate rel diff {err:.2e}")
    assert err <= 1e-2


def test_graph_and_direct_launches_agree_bitwise():
    g = small_fan(64, 90)
    P = Projectors(g)
    _, b, en = problem(g, n_ell=5, seed=4, oracle=P)
    G = gkb.Geometry(g)
    bd = to_dev(b, torch.float32)
    r1 = gkb.solve(G, bd, variant="BA", k_max=25, use_graph=True)
    r2 = gkb.solve(G, bd, variant="BA", k_max=25, use_graph=False)
    r3 = gkb.solve(G, bd, variant="BA", k_max=25, use_graph=True)
    assert torch.equal(r1.x, r2.x) and torch.equal(r1.x, r3.x)
    assert np.array_equal(r1.alpha, r2.alpha) and np.array_equal(r1.resid, r3.resid)


def test_plan_reuse_and_host_buffers():
    g = small_fan(64, 90)
    P = Projectors(g)
    _, b, en = problem(g, n_ell=5, seed=4, oracle=P)
    G = gkb.Geometry(g)
    plan = gkb.Plan(G, variant="AB", k_max=20, stop="dp", noise_norm=en)
    bd = to_dev(b, torch.float32)
    r1 = plan.execute(bd)
    bh = bd.cpu().pin_memory()
    xh = torch.empty(g.n, dtype=torch.float32).pin_memory()
    r2 = plan.execute(bh, xh)
    assert r1.k_stop == r2.k_stop
    assert torch.equal(r1.x.cpu(), xh)


@pytest.mark.parametrize("variant", ["AB", "BA"])
def test_rns_stop_matches_oracle_history(variant):
    g = NONDEG["parallel64_a91"]()
    P, x, b, en = _data(g)
    ref = og.gkb(variant, P, b, 40, stop="rns", rns_eps=0.03)
    res = gkb.solve(gkb.Geometry(g), to_dev(b, torch.float64), variant=variant, k_max=40, stop="rns",
                    rns_eps=0.03, storage=gkb.F64)
    assert ref["reason"] == "rns"
    assert res.k_stop == ref["k_stop"] and res.reason == "rns"


def test_breakdown_reaches_pseudoinverse():
    """Matched GKB on a 5x5 image with 72 rays: the Krylov space is exhausted
    by k = 25 and the iterate is the least-squares solution A^+ b."""
    g = gi.parallel_geometry(5, 8, 9)
    P = Projectors(g)
    from oracle import dense
    A = dense.dense_A(g)
    b = A @ gi.ellipse_phantom(5, 2, 0) + 0.01 * gi.noise_direction(g.m, 5)
    res = gkb.solve(gkb.Geometry(g), to_dev(b, torch.float64), variant="matched", k_max=60, storage=gkb.F64)
    assert res.status == gkb.STATUS_BREAKDOWN and res.reason == "breakdown" and res.k_stop <= 25
    assert rel(to_np(res.x), np.linalg.pinv(A) @ b) <= 1e-7


def test_zero_and_nonfinite_data():
    g = gi.parallel_geometry(16, 8, 23)
    G = gkb.Geometry(g)
    z = torch.zeros(g.m, device="cuda")
    res = gkb.solve(G, z, variant="BA", k_max=5)
    assert res.k_stop == 0 and res.status == gkb.STATUS_BREAKDOWN and float(res.x.abs().max()) == 0.0
    bad = torch.ones(g.m, device="cuda")
    bad[3] = float("nan")
    with pytest.raises(gkb.GKBError) as ei:
        gkb.solve(G, bad, variant="AB", k_max=5)
    assert ei.value.status == gkb.ERR_NONFINITE


def test_full_size_fan512_properties():
    """The 512x512 fan workload at k = 150 (the benchmark's launch
    configuration): t_1 and alpha_1 against the oracle, the carried residual
    against an explicit ||A x - b|| with the library's own A, and the AB data
    residual decreasing monotonically."""
    w = gi.fan_512()
    g = w.geom
    P = Projectors(g)
    x_true = gi.phantom_of(w)
    b, en = gi.add_noise(P.A(x_true), gi.noise_direction(g.m, w.noise_seed), w.eta)
    G = gkb.Geometry(g)
    bd = to_dev(b, torch.float32)
    for variant in ("BA", "AB"):
        res = gkb.solve(G, bd, variant=variant, k_max=150)
        M, MT, first, _ = og.operators(variant, P)
        r0 = first(b)
        t1 = np.linalg.norm(r0)
        a1 = np.linalg.norm(MT(r0 / t1))
        assert abs(res.t[0] - t1) <= 1e-5 * t1 and abs(res.alpha[0] - a1) <= 1e-5 * a1
        explicit = float(torch.linalg.norm(G.A(res.x).double() - bd.double()))
        assert abs(explicit - res.resid[-1]) <= 1e-4 * res.resid[-1]
        if variant == "AB":
            assert np.all(np.diff(res.resid) <= 1e-5 * res.resid[:-1])
        rre = float(torch.linalg.norm(res.x.cpu().double() - torch.from_numpy(x_true)) / np.linalg.norm(x_true))
        assert rre < 0.5


def test_fan512_size_twin_dp_index_and_iterate():
    """The 512x512 fan workload's size and detector (725 bins, SOD 1024, SDD
    2048, 30 ellipses, 2 % noise) with 721 angles over 360 degrees: an odd
    count removes the four-fold symmetry of the 720-angle geometry (whose
    degenerate singular-value pairs make late iterations depend on rounding
    in FP64 as well).  FP32 BA-GKB with the discrepancy principle: the same
    stopping index as the FP64 oracle (tie rule: or one off where the
    oracle's residual is within 1e-6 of the threshold) and the iterate within
    1e-3 of the oracle's."""
    w = gi.fan_512()
    g = gi.fan_geometry(512, 721, 725, 1024.0, 2048.0)
    P = Projectors(g)
    x_true = gi.phantom_of(w)
    b, en = gi.add_noise(P.A(x_true), gi.noise_direction(g.m, w.noise_seed), w.eta)
    ref = og.gkb("BA", P, b, 80, stop="dp", noise_norm=en)
    kd = ref["k_stop"]
    assert ref["reason"] == "dp"
    res = gkb.solve(gkb.Geometry(g), to_dev(b, torch.float32), variant="BA", k_max=80, stop="dp", noise_norm=en)
    margin = np.abs(ref["resid"][max(kd - 2, 0):kd] / en - 1.0).min()
    print(f"k_DP oracle {kd}, device {res.k_stop}, margin {margin:.2e}")
    assert res.k_stop == kd or (abs(res.k_stop - kd) == 1 and margin <= 1e-6)
    xo = ref["x"] if res.k_stop == kd else og.gkb("BA", P, b, res.k_stop)["x"]
    err = rel(to_np(res.x), xo)
    print(f"iterate relative difference at k_DP: {err:.2e}")
    assert err <= 1e-3


@pytest.mark.parametrize("variant", ["BA", "matched"])
def test_iterate_history_matches_oracle(variant):
    g = NONDEG["fan64_a91"]()
    P, x, b, en = _data(g)
    ref = og.gkb(variant, P, b, 25, keep_iterates=True)
    res, X = gkb.solve_iterates(gkb.Geometry(g), to_dev(b, torch.float64), variant=variant, k_max=25, storage=gkb.F64)
    assert res.k_stop == 25
    for k in (1, 2, 7, 25):
        assert rel(to_np(X[k - 1]), ref["xs"][k - 1]) <= 1e-9


def test_graph_kernel_counts():
    """The captured graph reports its kernels: a fixed number outside the
    iteration loop and per iteration (used for launch accounting)."""
    g = NONDEG["fan64_a91"]()
    P = gkb.Plan(gkb.Geometry(g), variant="BA", k_max=10, stop="none", storage=gkb.F32)
    outer, body = P.kernel_counts()
    assert outer >= 3 and body >= 8
    P.close()
    Q = gkb.Plan(gkb.Geometry(g), variant="BA", k_max=10, stop="none", storage=gkb.F32, use_graph=False)
    with pytest.raises(gkb.GKBError):
        Q.kernel_counts()
    Q.close()


@pytest.mark.parametrize("variant", ["BA", "AB"])
@pytest.mark.parametrize("operands", ["bf16", "f16"])
def test_mixed_precision_operands_converge(variant, operands):
    """FP32 Krylov vectors with 16-bit projector operands (the projectors read
    and write images and sinograms in BF16 or FP16, FP32 accumulation): the
    discrepancy principle is met within two iterations of the FP64 oracle's
    index, and the iterate there is within the 16-bit operands' error scale
    of the oracle's (BF16 rounds operands to 2^-9 relative, FP16 to 2^-12; an
    iterate combines k ~ 20-40 such products)."""
    g = NONDEG["fan64_a91"]()
    P, x, b, en = _data(g, eta=0.02)
    ref = og.gkb(variant, P, b, 80, stop="dp", noise_norm=en)
    code = {"bf16": gkb.BF16, "f16": gkb.F16}[operands]
    res = gkb.solve(gkb.Geometry(g), to_dev(b, torch.float32), variant=variant, k_max=80, stop="dp", noise_norm=en,
                    storage=gkb.F32, operands=code)
    assert res.reason == "dp"
    assert abs(res.k_stop - ref["k_stop"]) <= 2
    xo = og.gkb(variant, P, b, res.k_stop)["x"]
    err = rel(to_np(res.x), xo)
    print(f"{variant} {operands}: k_DP {res.k_stop} (oracle {ref['k_stop']}), iterate difference {err:.2e}")
    assert err <= {"bf16": 3e-2, "f16": 5e-3}[operands]
    # the reconstruction error against the phantom stays that of the FP64 solve
    rre_mixed = rel(to_np(res.x), x)
    rre_ref = rel(ref["x"], x)
    assert rre_mixed <= 1.05 * rre_ref


@pytest.mark.parametrize("variant", ["AB", "matched"])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_hybrid_regularisation_matches_oracle(variant, storage):
    """Hybrid regularisation (projected Tikhonov with the discrepancy
    principle on the projected residual, stopping once lambda settles):
    lambda_k per iteration, the stopping index and the iterate against the
    FP64 oracle.  The device finds lambda to ~2e-8 relative (six rounds of a
    32-point bracket) where the oracle bisects to 1e-10."""
    g = NONDEG["fan64_a91"]()
    P, x, b, en = _data(g, eta=0.03)
    ref = og.hybrid(variant, P, b, 60, en, lam_tol=1e-3)
    dt, code = (torch.float64, gkb.F64) if storage == "f64" else (torch.float32, gkb.F32)
    res = gkb.solve(gkb.Geometry(g), to_dev(b, dt), variant=variant, k_max=60, stop="hybrid", noise_norm=en,
                    rns_eps=1e-3, storage=code)
    print(f"{variant} {storage}: k_stop {res.k_stop} ({res.reason}), oracle {ref['k_stop']} ({ref['reason']})")
    lam_tol, x_tol = (1e-6, 1e-6) if storage == "f64" else (2e-3, 2e-3)
    assert res.reason == "hybrid" and ref["reason"] == "lambda"
    if storage == "f64":
        assert res.k_stop == ref["k_stop"]
    k = min(res.k_stop, ref["k_stop"])
    on = ref["lam"][:k] > 0
    assert np.array_equal(res.lam[:k] > 0, on)
    assert np.all(np.abs(res.lam[:k][on] - ref["lam"][:k][on]) <= lam_tol * ref["lam"][:k][on])
    xo = ref["x"] if res.k_stop == ref["k_stop"] else og.hybrid(variant, P, b, res.k_stop, en, lam_tol=0.0)["x"]
    assert rel(to_np(res.x), xo) <= x_tol
    # the hybrid iterate meets the discrepancy principle on the data
    r = np.linalg.norm(P.A(to_np(res.x)) - b)
    assert abs(r - en) <= 1e-3 * en


@pytest.mark.parametrize("kw", [
    dict(variant="BA", stop="hybrid", noise_norm=1.0),            # hybrid: projected residual != data residual
    dict(variant="AB", stop="hybrid", noise_norm=0.0),            # hybrid needs ||e||
    dict(variant="AB", stop="hybrid", noise_norm=1.0, storage=3),  # hybrid with FP16 storage (scaled data)
    dict(variant="AB-GMRES", k_max=3000),                          # GMRES keeps at most 2048 columns of H
    dict(variant="BA-GMRES", stop="learned", noise_norm=1.0, k_max=40),
    dict(variant="AB-GMRES", operands=2),                          # mixed operands only for the GKB variants
    dict(variant="BA", stop="learned", noise_norm=1.0, k_max=40, operands=2),
    dict(variant="AB", stop="learned", noise_norm=1.0, k_max=40),  # learned stop: BA only
    dict(variant="BA", k_max=0),
    dict(variant="BA", k_max=5000),
    dict(variant="BA", stop=9),
    dict(variant="BA", reorth=3),
    dict(variant="BA", tau=-1.0),
    dict(variant="BA", stop="dp", noise_norm=float("nan")),
    dict(variant="BA", stop="rns", rns_eps=0.0),
    dict(variant="BA", storage=7),
])
def test_invalid_solve_parameters_are_rejected(kw):
    """Every parameter combination the header declares invalid is refused by
    gkb_plan_create with GKB_ERR_INVALID_ARG before any work."""
    G = gkb.Geometry(NONDEG["parallel64_a91"]())
    with pytest.raises(gkb.GKBError) as ei:
        gkb.Plan(G, **kw)
    assert ei.value.status == gkb.ERR_INVALID_ARG
