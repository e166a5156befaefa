"""AB-GMRES (Algorithm 1) and BA-GMRES (Algorithm 2) step by step in FP64 --
TEST INFRASTRUCTURE.

Both methods run the Arnoldi process on a square product of the projector
pair from x_0 = 0:

  variant   M      r_0     iterate                      minimises
  AB        A B    b       x_k = B Q_k u_k              ||b - A x||      over x in B K_k(AB, b)
  BA        B A    B b     x_k = Q_k u_k                ||B (b - A x)|| over x in K_k(BA, B b)

Iteration k (Algorithms 1-2): w = M q_k; modified Gram-Schmidt against
q_1..q_k gives h_{i,k}; h_{k+1,k} = ||w||, q_{k+1} = w / h_{k+1,k}, so that
M Q_k = Q_{k+1} H_k with the
(k+1) x k upper Hessenberg H_k (Eq. Arn iter); u_k = argmin ||H_k u - ||r_0|| e_1||
(Eq. proj), solved here through the SVD as in Sec. 4's cost model (the
paper lists QR, LU or SVD); the iterate as in the table above.  The stopping
rules (Eq. DP, Eq. RNS) use the data residual ||A x_k - b|| for every
method, which this oracle forms explicitly.
"""
from __future__ import annotations

import numpy as np

from oracle.gkb import REASON_BREAKDOWN, REASON_DP, REASON_MAX_ITER, REASON_RNS, STOP_DP, STOP_NONE, STOP_RNS


def _lstsq_svd(H, beta):
    """u = argmin ||H u - beta e_1|| through the SVD of H (rank guard as LAPACK's rcond)."""
    U, sig, Vt = np.linalg.svd(H, full_matrices=False)
    rhs = beta * U[0, :]
    keep = sig > H.shape[0] * np.finfo(np.float64).eps * sig[0]
    return Vt[keep].T @ (rhs[keep] / sig[keep])


def gmres(variant, ops, b, k_max, stop=STOP_NONE, noise_norm=None, tau=1.0, rns_eps=None, breakdown_tol=1e-13,
          keep_bases=False, keep_iterates=False):
    """Run AB-GMRES ('AB', Algorithm 1) or BA-GMRES ('BA', Algorithm 2) for at
    most k_max iterations.  Returns a dict with H ((k+1) x k upper
    Hessenberg), resid[k-1] = ||A x_k - b||, proj_resid[k-1] =
    ||H_k u_k - ||r_0|| e_1||, k_stop, reason and x (= x_{k_stop}); optionally
    the basis Q and every iterate."""
    b = np.asarray(b, dtype=np.float64)
    if variant == "AB":
        M = lambda v: ops.A(ops.B(v))
        r0 = b.copy()
        to_image = ops.B
    elif variant == "BA":
        M = lambda v: ops.B(ops.A(v))
        r0 = ops.B(b)
        to_image = lambda y: y
    else:
        raise ValueError(variant)
    if stop == STOP_DP and noise_norm is None:
        raise ValueError("the discrepancy principle needs ||e||")
    beta = np.linalg.norm(r0)
    Q = [r0 / beta]
    H = np.zeros((k_max + 1, k_max))
    resid, proj_resid, xs = [], [], []
    x = None
    k_stop, reason = k_max, REASON_MAX_ITER
    for k in range(1, k_max + 1):
        w = M(Q[k - 1])
        for i in range(k):                                # modified Gram-Schmidt
            H[i, k - 1] = Q[i] @ w
            w = w - H[i, k - 1] * Q[i]
        H[k, k - 1] = np.linalg.norm(w)
        broke = H[k, k - 1] <= breakdown_tol * beta
        if not broke:
            Q.append(w / H[k, k - 1])
        Hk = H[:k + 1, :k]
        u = _lstsq_svd(Hk, beta)                          # projected problem
        x = to_image(np.column_stack(Q[:k]) @ u)          # iterate
        rhs = np.zeros(k + 1)
        rhs[0] = beta
        proj_resid.append(np.linalg.norm(Hk @ u - rhs))
        resid.append(np.linalg.norm(ops.A(x) - b))       # the data residual of Eq. DP
        if keep_iterates:
            xs.append(x.copy())
        if stop == STOP_DP and resid[-1] <= tau * noise_norm:
            k_stop, reason = k, REASON_DP
            break
        if stop == STOP_RNS and k >= 2 and abs(resid[-2] - resid[-1]) / resid[-2] < rns_eps:
            k_stop, reason = k, REASON_RNS
            break
        if broke:
            k_stop, reason = k, REASON_BREAKDOWN
            break
    out = dict(H=H[:k_stop + 1, :k_stop].copy(), beta=beta, resid=np.array(resid), proj_resid=np.array(proj_resid),
               k_stop=k_stop, reason=reason, x=x)
    if keep_bases:
        out["Q"] = np.column_stack(Q)
    if keep_iterates:
        out["xs"] = xs
    return out
