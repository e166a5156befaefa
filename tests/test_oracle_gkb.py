"""Pins of the FP64 GKB oracle (Algorithms 3-5) against library routines,
closed forms and brute force on tiny problems."""
import math

import numpy as np
import pytest
from scipy.sparse.linalg import lsqr

import gkb_inputs as gi
from oracle import dense, gkb as og
from oracle.projectors import Projectors


def tiny_problem(beam="parallel", N=8, na=6, nd=11, seed=0, eta=0.02):
    if beam == "parallel":
        g = gi.parallel_geometry(N, na, nd)
    else:
        g = gi.fan_geometry(N, na, nd, 3.0 * N, 6.0 * N)
    x = gi.ellipse_phantom(N, 3, seed)
    A, B = dense.dense_A(g), dense.dense_B(g)
    bt = A @ x
    b, en = gi.add_noise(bt, gi.noise_direction(g.m, seed + 50), eta)
    return g, x, A, B, b, en


@pytest.mark.parametrize("k", [1, 3, 8])
def test_matched_gkb_equals_scipy_lsqr(k):
    """Algorithm 3 is LSQR in exact arithmetic (Sec. 3.1)."""
    g, x, A, B, b, en = tiny_problem(N=10, na=9, nd=15)
    res = og.gkb("matched", og.DenseOps(A, B), b, k)
    xl = lsqr(A, b, atol=0, btol=0, conlim=0, iter_lim=k)[0]
    assert np.linalg.norm(res["x"] - xl) <= 1e-9 * np.linalg.norm(xl)


def test_matched_gkb_reaches_pseudoinverse():
    g, x, A, B, b, en = tiny_problem(N=5, na=8, nd=9)   # m = 72 > n = 25
    res = og.gkb("matched", og.DenseOps(A, B), b, g.n)
    xp = np.linalg.pinv(A) @ b
    assert np.linalg.norm(res["x"] - xp) <= 1e-7 * np.linalg.norm(xp)


def test_ba_gkb_reaches_ba_normal_equation_solution():
    """BA-GKB at full dimension: x = (BA)^+ B b (Eq. over UN NE)."""
    g, x, A, B, b, en = tiny_problem(N=5, na=8, nd=9)
    res = og.gkb("BA", og.DenseOps(A, B), b, g.n)
    xs = np.linalg.pinv(B @ A) @ (B @ b)
    assert np.linalg.norm(res["x"] - xs) <= 1e-6 * np.linalg.norm(xs)


def test_ab_gkb_reaches_ab_normal_equation_solution():
    """AB-GKB at full dimension: x = B (AB)^+ b (Eq. under UN NE)."""
    g, x, A, B, b, en = tiny_problem(N=6, na=3, nd=7)    # m = 21 < n = 36
    res = og.gkb("AB", og.DenseOps(A, B), b, g.m)
    xs = B @ (np.linalg.pinv(A @ B) @ b)
    assert np.linalg.norm(res["x"] - xs) <= 1e-6 * np.linalg.norm(xs)


@pytest.mark.parametrize("variant", ["AB", "BA"])
@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_krylov_optimality(variant, k):
    """u_k minimises ||M y - r0|| over K_k(M^T M, M^T r0): checked with an
    independently built, orthonormalised power basis and lstsq."""
    g, x, A, B, b, en = tiny_problem(N=7, na=7, nd=11, seed=2)
    M = A @ B if variant == "AB" else B @ A
    r0 = b if variant == "AB" else B @ b
    res = og.gkb(variant, og.DenseOps(A, B), b, k)
    v = M.T @ r0
    basis = []
    for _ in range(k):
        w = v.copy()
        for u in basis:
            w -= (u @ w) * u
        for u in basis:
            w -= (u @ w) * u
        basis.append(w / np.linalg.norm(w))
        v = M.T @ (M @ basis[-1])
    V = np.column_stack(basis)
    y = V @ np.linalg.lstsq(M @ V, r0, rcond=None)[0]
    xk = B @ y if variant == "AB" else y
    assert np.linalg.norm(res["x"] - xk) <= 1e-8 * np.linalg.norm(xk)


@pytest.mark.parametrize("variant", ["matched", "AB", "BA"])
def test_bidiagonal_relations_and_orthogonality(variant):
    g, x, A, B, b, en = tiny_problem(N=9, na=10, nd=13, seed=3)
    k = 12
    res = og.gkb(variant, og.DenseOps(A, B), b, k, keep_bases=True)
    M = {"matched": A, "AB": A @ B, "BA": B @ A}[variant]
    Q, S = res["Q"][:, :k], res["S"]
    C = og.lower_bidiagonal(res["alpha"], res["t"], k)
    assert np.linalg.norm(M @ Q - S @ C) <= 1e-12 * np.linalg.norm(M, 2)
    Qf = res["Q"]
    assert np.abs(Qf.T @ Qf - np.eye(Qf.shape[1])).max() <= 1e-14
    # second relation: M^T S_{k+1} = Q_{k+1} C~ with C~ upper bidiagonal (alpha diag, t super-diag)
    Ct = np.zeros((k + 1, k + 1))
    for i in range(k + 1):
        Ct[i, i] = res["alpha"][i]
        if i + 1 <= k:
            Ct[i, i + 1] = res["t"][i + 1]
    assert np.linalg.norm(M.T @ S - res["Q"] @ Ct) <= 1e-10 * np.linalg.norm(M, 2)


@pytest.mark.parametrize("variant", ["AB", "BA"])
def test_reorthogonalisation_keeps_basis_orthogonal_over_many_steps(variant):
    """The one-sided reorthogonalisation runs over every earlier q_i, the newest included; without it the
    loss of orthogonality reaches ~1e-13 here, with it it stays at ~1e-15."""
    g = gi.parallel_geometry(12, 30, 17)
    A, B = dense.dense_A(g), dense.dense_B(g)
    b = A @ gi.ellipse_phantom(12, 3, 1)
    Q = og.gkb(variant, og.DenseOps(A, B), b, 60, keep_bases=True)["Q"]
    assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() <= 1e-14


@pytest.mark.parametrize("variant", ["matched", "AB"])
def test_projected_residual_is_data_residual(variant):
    """For M = A and M = AB: A x_k - b = S_{k+1}(C_k u_k - t1 e1), so the two
    norms agree while S stays orthonormal."""
    g, x, A, B, b, en = tiny_problem(N=10, na=12, nd=15, seed=4)
    res = og.gkb(variant, og.DenseOps(A, B), b, 10)
    assert np.allclose(res["resid"], res["proj_resid"], rtol=1e-9)


def test_projected_svd_solve_equals_lstsq():
    rng = np.random.default_rng(8)
    for k in (1, 2, 5, 20):
        alpha, t = rng.uniform(0.1, 2, k + 1), rng.uniform(0.1, 2, k + 2)
        C = og.lower_bidiagonal(alpha, t, k)
        rhs = np.zeros(k + 1)
        rhs[0] = t[0]
        u = og.solve_projected_svd(C, t[0])
        assert np.allclose(u, np.linalg.lstsq(C, rhs, rcond=None)[0], rtol=1e-11, atol=1e-13)


def test_tikhonov_filter_limits():
    rng = np.random.default_rng(9)
    k = 6
    C = og.lower_bidiagonal(rng.uniform(0.1, 2, k), rng.uniform(0.1, 2, k + 1), k)
    t1 = 1.7
    u0 = og.tikhonov_projected(C, t1, 0.0)
    assert np.allclose(u0, og.solve_projected_svd(C, t1), rtol=1e-11)
    lam = 0.3
    rhs = np.zeros(k + 1)
    rhs[0] = t1
    aug = np.vstack([C, lam * np.eye(k)])
    ref = np.linalg.lstsq(aug, np.concatenate([rhs, np.zeros(k)]), rcond=None)[0]
    assert np.allclose(og.tikhonov_projected(C, t1, lam), ref, rtol=1e-11)


def test_discrepancy_principle_and_rns_stop():
    g, x, A, B, b, en = tiny_problem(N=12, na=12, nd=17, seed=5, eta=0.05)
    full = og.gkb("BA", og.DenseOps(A, B), b, 25)
    kdp = og.dp_index(full["resid"], en)
    assert kdp is not None and kdp > 1
    res = og.gkb("BA", og.DenseOps(A, B), b, 25, stop="dp", noise_norm=en)
    assert res["k_stop"] == kdp and res["reason"] == "dp"
    assert res["resid"][-1] <= en < res["resid"][-2]
    rns = og.gkb("BA", og.DenseOps(A, B), b, 25, stop="rns", rns_eps=0.01)
    r = full["resid"]
    expect = next(k for k in range(2, 26) if abs(r[k - 2] - r[k - 1]) / r[k - 2] < 0.01)
    assert rns["k_stop"] == expect


def test_matrix_free_oracle_equals_dense_route():
    g = gi.fan_geometry(12, 15, 19, 36.0, 72.0)
    x = gi.ellipse_phantom(12, 3, 1)
    P = Projectors(g)
    b, en = gi.add_noise(P.A(x), gi.noise_direction(g.m, 3), 0.02)
    D = og.DenseOps(dense.dense_A(g), dense.dense_B(g))
    for v in ("matched", "AB", "BA"):
        r1 = og.gkb(v, P, b, 8)
        r2 = og.gkb(v, D, b, 8)
        assert np.allclose(r1["alpha"], r2["alpha"], rtol=1e-10)
        assert np.allclose(r1["x"], r2["x"], rtol=1e-8, atol=1e-10)


def test_four_projector_applications_per_iteration():
    """Sec. 4: every iteration applies AB / BA and their transposes once: 4 projector
    applications per AB-/BA-GKB iteration (the oracle's own residual adds more)."""
    g = gi.parallel_geometry(10, 8, 15)
    P = Projectors(g)
    b = P.A(gi.ellipse_phantom(10, 2, 0))
    k = 5
    M, MT, first, _ = og.operators("BA", P)
    before = dict(P.calls)
    s = first(b)
    q = MT(s)
    for _ in range(k):
        s = M(q)
        q = MT(s)
    used = {key: P.calls[key] - before[key] for key in P.calls}
    assert used == {"A": k, "B": k + 1, "AT": k + 1, "BT": k + 1}


def _k1_label(a, b, c, target):
    """Closed form of the learned stop's lambda label on a one-column C.

    C = [a; b], rhs = [c; 0]: u_lambda = a c / (a^2 + b^2 + lambda^2) and
    ||C u - rhs||^2 = s u^2 - 2 a c u + c^2 with s = a^2 + b^2.  Setting that to
    target^2 and taking the root below the least-squares u* = a c / s gives
    u, and then lambda^2 = a c / u - s."""
    s = a * a + b * b
    u = (a * c - math.sqrt(a * a * c * c - s * (c * c - target * target))) / s
    return math.sqrt(a * c / u - s)


def test_tikhonov_lambda_closed_form_on_one_column():
    """The bisection for lambda against the closed form of a one-column
    projected problem, for targets between the least-squares residual and t1."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        a, b, c = rng.uniform(0.2, 3.0, 3)
        r_ls = c * b / math.sqrt(a * a + b * b)          # least-squares residual of [a; b] u ~ [c; 0]
        target = r_ls + rng.uniform(0.05, 0.95) * (c - r_ls)
        lam = _k1_label(a, b, c, target)
        C = og.lower_bidiagonal([a], [c, b], 1)
        assert abs(og.projected_residual(C, c, og.tikhonov_projected(C, c, lam)) - target) <= 1e-12 * c
        got = og.tikhonov_lambda(C, c, target, 1e-9 * a, 1e3 * a)
        assert abs(got - lam) <= 1e-9 * lam, (got, lam)


def test_tikhonov_label_hits_the_target_and_is_monotone():
    """On solver histories of a small BA problem: the projected Tikhonov
    residual grows monotonically in lambda from the least-squares residual
    (lambda = 0) towards t1, and the label reproduces the plain iterate's
    projected residual at k_dp to 1e-10."""
    g = gi.fan_geometry(32, 37, 47, 64.0, 128.0)
    P = Projectors(g)
    x = gi.ellipse_phantom(32, 5, 9)
    b, en = gi.add_noise(P.A(x), gi.noise_direction(g.m, 19), 0.02)
    ref = og.gkb("BA", P, b, 60)
    kdp = og.dp_index(ref["resid"], en)
    assert kdp is not None and kdp + 8 <= 60
    al, t = ref["alpha"], ref["t"]
    t1 = t[0]
    C = og.lower_bidiagonal(al, t, kdp + 8)
    lams = np.exp(np.linspace(np.log(al[0] * 1e-9), np.log(al[0] * 10), 200))
    rs = [og.projected_residual(C, t1, og.tikhonov_projected(C, t1, lam)) for lam in lams]
    assert np.all(np.diff(rs) >= -1e-12 * t1)
    r_ls = og.projected_residual(C, t1, og.solve_projected_svd(C, t1))
    assert abs(rs[0] - r_ls) <= 1e-8 * t1
    lam = og.tikhonov_label(al, t, kdp)
    Cd = og.lower_bidiagonal(al, t, kdp)
    target = og.projected_residual(Cd, t1, og.solve_projected_svd(Cd, t1))
    assert abs(og.projected_residual(C, t1, og.tikhonov_projected(C, t1, lam)) - target) <= 1e-10 * t1
    assert lams[0] < lam < lams[-1]


def test_storage_model_rounds_only_the_stored_vectors():
    """The FP32 storage model of the oracle: with storage=float64 it is the
    plain oracle bit for bit; with float32 every basis vector is exactly a
    float32 vector, and the scalars move away from the FP64 run by more than
    FP64 rounding but far less than the quantities themselves."""
    g = gi.fan_geometry(24, 29, 37, 48.0, 96.0)
    P = Projectors(g)
    x = gi.ellipse_phantom(24, 4, 3)
    b, en = gi.add_noise(P.A(x), gi.noise_direction(g.m, 13), 0.01)
    ref = og.gkb("BA", P, b, 12, keep_bases=True)
    same = og.gkb("BA", P, b, 12, keep_bases=True, storage=np.float64)
    assert np.array_equal(ref["alpha"], same["alpha"]) and np.array_equal(ref["x"], same["x"])
    f32 = og.gkb("BA", P, b, 12, keep_bases=True, storage=np.float32)
    assert np.array_equal(f32["Q"], f32["Q"].astype(np.float32).astype(np.float64))
    assert np.array_equal(f32["S"], f32["S"].astype(np.float32).astype(np.float64))
    dev = np.abs(f32["alpha"] - ref["alpha"]) / ref["alpha"]
    assert 1e-12 < dev.max() < 1e-3


@pytest.mark.parametrize("variant", ["AB", "matched"])
def test_hybrid_meets_the_discrepancy_principle_exactly(variant):
    """Every hybrid iterate with lambda_k > 0 has data residual ||A x - b|| =
    tau ||e|| (checked with the operators, not the projected problem), and
    lambda_k is zero exactly while the plain iterate's residual is above it."""
    g, x, A, B, b, en = tiny_problem("fan", N=9, na=7, nd=13, eta=0.05)
    ops = og.DenseOps(A, B)
    ref = og.gkb(variant, ops, b, 25)
    M, MT, first, to_image = og.operators(variant, ops)
    for k in (3, 6, 10, 14):
        h = og.hybrid(variant, ops, b, k, en, lam_tol=0.0)
        assert h["k_stop"] == k
        lam = h["lam"][-1]
        r = np.linalg.norm(A @ h["x"] - b)
        if ref["resid"][k - 1] > en:
            assert lam == 0.0 and np.allclose(h["x"], og.gkb(variant, ops, b, k)["x"], rtol=1e-12)
        else:
            assert lam > 0.0 and abs(r - en) <= 1e-8 * en


def test_hybrid_at_full_dimension_is_tikhonov():
    """Matched hybrid at k = n: the Krylov space is the whole image space, so
    the iterate is the full Tikhonov solution (A^T A + lambda^2 I)^-1 A^T b for
    its lambda (a dense solve), and that lambda meets the discrepancy
    principle for the full problem."""
    g, x, A, B, b, en = tiny_problem(N=5, na=8, nd=9, eta=0.05)   # n = 25 < m = 72
    h = og.hybrid("matched", og.DenseOps(A, B), b, g.n, en, lam_tol=0.0)
    lam = h["lam"][-1]
    assert lam > 0.0
    xt = np.linalg.solve(A.T @ A + lam * lam * np.eye(g.n), A.T @ b)
    assert np.linalg.norm(h["x"] - xt) <= 1e-7 * np.linalg.norm(xt)
    assert abs(np.linalg.norm(A @ xt - b) - en) <= 1e-7 * en
