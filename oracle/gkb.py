"""GKB with a matched transpose (Algorithm 3), AB-GKB (Algorithm 4) and
BA-GKB (Algorithm 5), step by step in FP64 -- TEST INFRASTRUCTURE.

Reading of the printed loop (its first pass refers to q_0 and alpha_0, which
the initialisation never defines): after the initialisation produces t_1,
s_1, alpha_1 and q_1, iteration k = 1, 2, ... computes

    s        = M q_k - alpha_k s_k
    t_{k+1}  = ||s||,  s_{k+1} = s / t_{k+1}
    q        = M^T s_{k+1} - t_{k+1} q_k
    q        = q - sum_{i<=k} (q_i^T q) q_i         (the one-sided
                                                     reorthogonalisation: one
                                                     pass, every coefficient
                                                     taken against the same q,
                                                     the printed classical
                                                     Gram-Schmidt form)
    alpha_{k+1} = ||q||, q_{k+1} = q / alpha_{k+1}

so that C_k is the (k+1) x k lower bidiagonal matrix with alpha_1..alpha_k
on its diagonal and t_2..t_{k+1} below it (Eq. lower bid), and
M Q_k = S_{k+1} C_k (Eq. GKB dec).  The projected problem
min ||C_k u - t_1 e_1|| (Eq. proj GKB) is solved through the SVD of C_k
(Sec. 3.2, last paragraph); the iterate is x_k = Q_k u_k (matched, BA) or
x_k = B Q_k u_k (AB).  The loop ends by the discrepancy principle (Eq. DP: the first k with
||A x_k - b|| <= tau ||e||) or residual-norm stagnation (Eq. RNS), both on the
data residual ||A x_k - b||, which this oracle forms explicitly.

  variant   M            M^T            first vector r_0   solution map
  matched   A            A^T            b                  x = Q u
  AB        A B          B^T A^T        b                  x = B (Q u)
  BA        B A          A^T B^T        B b                x = Q u
"""
from __future__ import annotations

import numpy as np

STOP_NONE, STOP_DP, STOP_RNS = "none", "dp", "rns"
REASON_MAX_ITER, REASON_DP, REASON_RNS, REASON_BREAKDOWN = "k_max", "dp", "rns", "breakdown"


def lower_bidiagonal(alpha, t, k):
    """C_k: (k+1) x k with alpha_1..alpha_k on the diagonal, t_2..t_{k+1} below.

    ``alpha[i]`` holds alpha_{i+1} and ``t[i]`` holds t_{i+1} (0-based lists).
    """
    C = np.zeros((k + 1, k))
    for i in range(k):
        C[i, i] = alpha[i]
        C[i + 1, i] = t[i + 1]
    return C


def solve_projected_svd(C, t1):
    """u = argmin ||C u - t1 e_1|| through the SVD of C (rank guard as LAPACK's rcond)."""
    U, sig, Vt = np.linalg.svd(C, full_matrices=False)
    beta = t1 * U[0, :]
    keep = sig > (C.shape[0]) * np.finfo(np.float64).eps * sig[0]
    return Vt[keep].T @ (beta[keep] / sig[keep])


def tikhonov_projected(C, t1, lam):
    """u_lambda = sum_i sigma_i/(sigma_i^2+lambda^2) (U_i^T t1 e1) V_i (SVD filter factors)."""
    U, sig, Vt = np.linalg.svd(C, full_matrices=False)
    beta = t1 * U[0, :]
    return Vt.T @ (sig / (sig * sig + lam * lam) * beta)


def projected_residual(C, t1, u):
    """||C u - t1 e_1|| (the residual of the projected problem)."""
    rhs = np.zeros(C.shape[0])
    rhs[0] = t1
    return float(np.linalg.norm(C @ u - rhs))


def tikhonov_lambda(C, t1, target, lo, hi, steps=100):
    """The lambda in [lo, hi] whose projected Tikhonov iterate u_lambda on C has
    ||C u_lambda - t1 e1|| = target, by bisection in log(lambda).  That
    residual grows monotonically with lambda (from the least-squares residual
    at lambda = 0 towards t1 as lambda -> infinity), so the root is unique
    when it lies in the bracket; otherwise the nearer end is returned."""
    a, b = np.log(lo), np.log(hi)
    for _ in range(steps):
        mid = 0.5 * (a + b)
        if projected_residual(C, t1, tikhonov_projected(C, t1, np.exp(mid))) > target:
            b = mid
        else:
            a = mid
    return float(np.exp(0.5 * (a + b)))


def tikhonov_label(alpha, t, k_dp, delta=8, lo_factor=1e-9, hi_factor=10.0):
    """Label of the learned stop's regularisation parameter (the paper has no
    learned part; this is the build's definition): lambda* such that the
    projected Tikhonov iterate on C_k, k = k_dp + delta, has the projected
    residual of the plain least-squares iterate at k_dp,

        ||C_k u_lambda - t1 e1|| = ||C_{k_dp} u_{k_dp} - t1 e1||,

    searched over [lo_factor, hi_factor] * alpha_1.  ``alpha`` and ``t`` are
    the 0-based histories (alpha_1.., t_1..) with at least k entries of alpha
    and k+1 of t."""
    t1 = t[0]
    Cd = lower_bidiagonal(alpha, t, k_dp)
    target = projected_residual(Cd, t1, solve_projected_svd(Cd, t1))
    C = lower_bidiagonal(alpha, t, k_dp + delta)
    return tikhonov_lambda(C, t1, target, alpha[0] * lo_factor, alpha[0] * hi_factor)


def operators(variant, ops):
    if variant == "matched":
        return ops.A, ops.AT, (lambda b: b), (lambda y: y)
    if variant == "AB":
        return (lambda v: ops.A(ops.B(v))), (lambda s: ops.BT(ops.AT(s))), (lambda b: b), ops.B
    if variant == "BA":
        return (lambda v: ops.B(ops.A(v))), (lambda s: ops.AT(ops.BT(s))), ops.B, (lambda y: y)
    raise ValueError(variant)


def gkb(variant, ops, b, k_max, stop=STOP_NONE, noise_norm=None, tau=1.0, rns_eps=None,
        reorth=True, breakdown_tol=1e-13, keep_iterates=False, x_true=None, keep_bases=False, storage=None):
    """Run Algorithm 3 ('matched'), 4 ('AB') or 5 ('BA') for at most k_max iterations.

    ``ops`` provides A, B, AT, BT as callables on FP64 vectors.  Returns a dict
    with alpha (alpha_1, alpha_2, ...), t (t_1, t_2, ...), resid[k-1] =
    ||A x_k - b||, proj_resid[k-1] = ||C_k u_k - t_1 e_1||, k_stop, reason and
    x (= x_{k_stop}); optionally every iterate, the RRE history and the bases.

    ``storage`` (e.g. numpy.float32) is a model of lower-precision storage:
    b, every vector the recurrences keep (s, q before and after
    normalisation, the basis) is rounded to that type after it is formed,
    while every operation still runs in FP64.  It shows how far the method
    itself moves when its vectors are stored in that type -- the scale
    against which a solve in that storage type is compared -- not a
    reference result.
    """
    M, MT, first, to_image = operators(variant, ops)
    b = np.asarray(b, dtype=np.float64)
    rnd = (lambda v: v) if storage is None else (lambda v: np.asarray(v).astype(storage).astype(np.float64))
    b = rnd(b)
    if stop == STOP_DP and noise_norm is None:
        raise ValueError("the discrepancy principle needs ||e||")
    # initialisation: t_1, s_1, alpha_1, q_1
    r0 = rnd(first(b))
    t = [np.linalg.norm(r0)]
    S = [rnd(r0 / t[0])]
    q = rnd(MT(S[0]))
    alpha = [np.linalg.norm(q)]
    Q = [rnd(q / alpha[0])]
    scale0 = max(t[0], alpha[0])
    resid, proj_resid, xs, rre = [], [], [], []
    x = None
    k_stop, reason = k_max, REASON_MAX_ITER
    for k in range(1, k_max + 1):
        # s = M q_k - alpha_k s_k, t_{k+1}, s_{k+1}
        s = rnd(M(Q[k - 1]) - alpha[k - 1] * S[k - 1])
        t.append(np.linalg.norm(s))
        broke = t[k] <= breakdown_tol * scale0
        if not broke:
            S.append(rnd(s / t[k]))
            # q = M^T s_{k+1} - t_{k+1} q_k, reorthogonalisation, alpha_{k+1}, q_{k+1}
            q = rnd(MT(S[k]) - t[k] * Q[k - 1])
            if reorth:
                coef = [Q[i] @ q for i in range(k)]
                for i in range(k):
                    q = q - coef[i] * Q[i]
                q = rnd(q)
            alpha.append(np.linalg.norm(q))
            if alpha[k] > breakdown_tol * scale0:
                Q.append(rnd(q / alpha[k]))
            else:
                broke = True
        # projected problem and iterate
        C = lower_bidiagonal(alpha, t, k)
        u = solve_projected_svd(C, t[0])
        x = to_image(np.column_stack(Q[:k]) @ u)
        rhs = np.zeros(k + 1)
        rhs[0] = t[0]
        proj_resid.append(np.linalg.norm(C @ u - rhs))
        resid.append(np.linalg.norm(ops.A(x) - b))
        if keep_iterates:
            xs.append(x.copy())
        if x_true is not None:
            rre.append(np.linalg.norm(x - x_true) / np.linalg.norm(x_true))
        # stopping rules
        if stop == STOP_DP and resid[-1] <= tau * noise_norm:
            k_stop, reason = k, REASON_DP
            break
        if stop == STOP_RNS and k >= 2 and abs(resid[-2] - resid[-1]) / resid[-2] < rns_eps:
            k_stop, reason = k, REASON_RNS
            break
        if broke:
            k_stop, reason = k, REASON_BREAKDOWN
            break
    out = dict(alpha=np.array(alpha), t=np.array(t), resid=np.array(resid),
               proj_resid=np.array(proj_resid), k_stop=k_stop, reason=reason, x=x)
    if keep_iterates:
        out["xs"] = xs
    if x_true is not None:
        out["rre"] = np.array(rre)
    if keep_bases:
        out["Q"] = np.column_stack(Q)
        out["S"] = np.column_stack(S)
    return out


def dp_index(resid, noise_norm, tau=1.0):
    """k_DP of Eq. (DP) from a residual history (1-based), or None."""
    hit = np.nonzero(np.asarray(resid) <= tau * noise_norm)[0]
    return int(hit[0]) + 1 if hit.size else None


def rre(x, x_true):
    """Relative reconstruction error, Eq. (RE)."""
    return float(np.linalg.norm(x - x_true) / np.linalg.norm(x_true))


class DenseOps:
    """The four operators as explicit matrices (for pins on tiny problems)."""

    def __init__(self, A, B):
        self.Am, self.Bm = A, B

    def A(self, x):
        return self.Am @ x

    def AT(self, y):
        return self.Am.T @ y

    def B(self, y):
        return self.Bm @ y

    def BT(self, x):
        return self.Bm.T @ x


def hybrid(variant, ops, b, k_max, noise_norm, tau=1.0, lam_tol=1e-3, lo_factor=1e-9, hi_factor=10.0):
    """Hybrid regularisation of AB-GKB or matched GKB (the paper's stated
    future work, Sec. 6: regularisation inside the projected problem): after
    every iteration k the projected Tikhonov problem

        u = argmin ||C_k u - t1 e1||^2 + lambda_k^2 ||u||^2

    is solved with lambda_k from the discrepancy principle on the projected
    residual: lambda_k = 0 while the least-squares residual is above
    tau ||e||, else the lambda with ||C_k u_lambda - t1 e1|| = tau ||e||
    (tikhonov_lambda over [lo_factor, hi_factor] * alpha_1).  For AB and
    matched GKB the basis S_{k+1} is orthonormal, so that projected residual
    is the data residual ||A x - b|| of x = B Q_k u (AB) or Q_k u (matched).
    The run stops at the first k >= 2 with lambda_{k-1} > 0 and
    |lambda_k - lambda_{k-1}| <= lam_tol lambda_{k-1} (the parameter has
    settled), else at k_max.  Returns the GKB run's histories with lam
    (lambda_1..), k_stop, reason ('lambda' or 'k_max') and x."""
    if variant not in ("AB", "matched"):
        raise ValueError("the projected residual is the data residual only for AB and matched GKB")
    run = gkb(variant, ops, b, k_max, keep_bases=True)
    _, _, _, to_image = operators(variant, ops)
    al, t = run["alpha"], run["t"]
    target = tau * noise_norm
    lams = []
    k_stop, reason = run["k_stop"], REASON_MAX_ITER
    for k in range(1, run["k_stop"] + 1):
        C = lower_bidiagonal(al, t, k)
        r_ls = projected_residual(C, t[0], solve_projected_svd(C, t[0]))
        lam = 0.0 if r_ls >= target else tikhonov_lambda(C, t[0], target, al[0] * lo_factor, al[0] * hi_factor)
        lams.append(lam)
        if k >= 2 and lams[-2] > 0.0 and abs(lam - lams[-2]) <= lam_tol * lams[-2]:
            k_stop, reason = k, "lambda"
            break
    C = lower_bidiagonal(al, t, k_stop)
    u = tikhonov_projected(C, t[0], lams[-1]) if lams[-1] > 0.0 else solve_projected_svd(C, t[0])
    x = to_image(run["Q"][:, :k_stop] @ u)
    return dict(alpha=al[:k_stop + 1], t=t[:k_stop + 2], lam=np.array(lams), k_stop=k_stop, reason=reason, x=x,
                resid_ls=run["resid"][:k_stop])
