"""Pins of the FP64 GMRES oracle (Algorithms 1-2) against library routines,
closed forms and independent constructions on tiny problems."""
import numpy as np
import pytest
from scipy.sparse.linalg import lsmr, lsqr

from oracle import gkb as og
from oracle import gmres as gm
from tests.test_oracle_gkb import tiny_problem


@pytest.mark.parametrize("variant", ["AB", "BA"])
def test_arnoldi_relation_and_orthogonality(variant):
    """M Q_k = Q_{k+1} H_k (Eq. Arn iter), Q orthonormal, H upper Hessenberg."""
    g, x, A, B, b, en = tiny_problem("fan", N=9, na=7, nd=13)
    res = gm.gmres(variant, og.DenseOps(A, B), b, 10, keep_bases=True)
    M = A @ B if variant == "AB" else B @ A
    Q, H = res["Q"], res["H"]
    k = res["k_stop"]
    assert np.linalg.norm(M @ Q[:, :k] - Q[:, :k + 1] @ H) <= 1e-12 * np.linalg.norm(M) * np.sqrt(k)
    assert np.linalg.norm(Q.T @ Q - np.eye(Q.shape[1])) <= 1e-13 * k
    assert np.all(np.tril(H, -2) == 0)


@pytest.mark.parametrize("k", [1, 3, 7])
def test_ab_gmres_with_matched_back_projector_is_lsqr(k):
    """With B = A^T, AB-GMRES minimises ||b - A x|| over x in A^T K_k(A A^T, b)
    = K_k(A^T A, A^T b): LSQR's problem, so the iterates agree."""
    g, x, A, B, b, en = tiny_problem(N=10, na=9, nd=15)
    res = gm.gmres("AB", og.DenseOps(A, A.T), b, k)
    xl = lsqr(A, b, atol=0, btol=0, conlim=0, iter_lim=k)[0]
    assert np.linalg.norm(res["x"] - xl) <= 1e-9 * np.linalg.norm(xl)


@pytest.mark.parametrize("k", [1, 3, 7])
def test_ba_gmres_with_matched_back_projector_is_lsmr(k):
    """With B = A^T, BA-GMRES minimises ||A^T (b - A x)|| over K_k(A^T A, A^T b):
    LSMR's problem (Fong and Saunders), so the iterates agree."""
    g, x, A, B, b, en = tiny_problem(N=10, na=9, nd=15)
    res = gm.gmres("BA", og.DenseOps(A, A.T), b, k)
    xl = lsmr(A, b, atol=0, btol=0, conlim=0, maxiter=k)[0]
    assert np.linalg.norm(res["x"] - xl) <= 1e-8 * np.linalg.norm(xl)


@pytest.mark.parametrize("variant", ["AB", "BA"])
@pytest.mark.parametrize("k", [1, 2, 5])
def test_minimal_residual_over_the_krylov_space(variant, k):
    """The unmatched case against an independent construction: the Krylov
    space spanned by explicit powers, orthonormalised by a library QR, and the
    minimiser by a library least-squares solve."""
    g, x, A, B, b, en = tiny_problem("fan", N=8, na=7, nd=11)
    res = gm.gmres(variant, og.DenseOps(A, B), b, k)
    M = A @ B if variant == "AB" else B @ A
    r0 = b if variant == "AB" else B @ b
    K = np.column_stack([np.linalg.matrix_power(M, i) @ r0 for i in range(k)])
    V, _ = np.linalg.qr(K)
    if variant == "AB":
        z = np.linalg.lstsq(A @ B @ V, b, rcond=None)[0]
        xs = B @ (V @ z)
    else:
        z = np.linalg.lstsq(B @ A @ V, B @ b, rcond=None)[0]
        xs = V @ z
    assert np.linalg.norm(res["x"] - xs) <= 1e-8 * np.linalg.norm(xs)


def test_ba_gmres_reaches_the_square_system_solution():
    """At full dimension BA-GMRES solves B A x = B b (Eq. over UN NE)."""
    g, x, A, B, b, en = tiny_problem(N=5, na=8, nd=9)   # n = 25
    res = gm.gmres("BA", og.DenseOps(A, B), b, g.n)
    xs = np.linalg.lstsq(B @ A, B @ b, rcond=None)[0]
    assert np.linalg.norm(res["x"] - xs) <= 1e-6 * np.linalg.norm(xs)


@pytest.mark.parametrize("variant", ["AB", "BA"])
def test_residuals_and_stopping(variant):
    """AB's projected residual is the data residual (orthonormal Q); both
    variants stop at the first k meeting Eq. DP, the tie-free index of the
    explicit residual history."""
    g, x, A, B, b, en = tiny_problem("fan", N=9, na=7, nd=13, eta=0.05)
    full = gm.gmres(variant, og.DenseOps(A, B), b, 12)
    if variant == "AB":
        assert np.allclose(full["proj_resid"], full["resid"], rtol=1e-10)
    kdp = og.dp_index(full["resid"], en)
    assert kdp is not None
    res = gm.gmres(variant, og.DenseOps(A, B), b, 12, stop="dp", noise_norm=en)
    assert res["k_stop"] == kdp and res["reason"] == "dp"
