"""Oracle: the affine-normal direction of a level set (Sec. 5).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

At x with g = grad f(x), e = g/|g| and an orthonormal frame Q = [Q_T, e]:

    H_T = Q_T^T H Q_T,   h = Q_T^T H e,
    a_i = tr(H_T^{-1} d_{t_i} H_T),  i = 1..n-1,
    tau = H_T^{-1} (h - |g|/(n+1) a),
    nu  = Q [tau; -1] = Q_T tau - e.

d_{t_i} H_T = Q_T^T (sum_l T_l (Q_T)_{l i}) Q_T is the derivative of the tangent
Hessian block along the tangent axis q_i (T = third-derivative tensor).

Readings of the paper taken here, where it is silent or ambiguous:
* the regularisation r enters every tangent solve: H_T is replaced by
  H_T + r I both in the trace term and in tau (this is what reproduces the
  printed worked example of Sec. 5 to every shown digit);
* the returned direction is the paper's nu (its component along e is exactly
  -1), not a unit vector; ``unit`` is nu/|nu|;
* no orientation flip: if the Cholesky factorisation of H_T + r I fails the
  point is flagged NOT_PD; if |g| = 0 (or, unless ``assume_nonzero_x``,
  |g| <= 1e-14 * S with S the sum over all terms and coordinates of
  |gradient contributions|) it is flagged ZERO_GRAD;
  flagged points return NaN directions;
* work counters follow the paper's example: hv_evals = n, third_evals = n-1
  for the exact method.

The frame is any orthonormal basis of e-perp; the oracle completes e with a QR
factorisation, independently of the Householder frame the GPU uses (the
direction does not depend on the frame -- pinned by a test).
"""
from __future__ import annotations

import numpy as np

from . import derivs
from .rng import rademacher

FLAG_ZERO_GRAD = 1
FLAG_NOT_PD = 2
FLAG_KRYLOV_MAXIT = 4


def qr_frame(e: np.ndarray) -> np.ndarray:
    """Q_T: n x (n-1) orthonormal basis of the complement of unit vector e."""
    n = e.shape[0]
    M = np.column_stack([e, np.eye(n)])
    Q, _ = np.linalg.qr(M)
    return Q[:, 1:n]


def _grad_hess(exps, coef, x):
    F, G, H, SF, SG, SH = derivs.eval_derivs(exps, coef, x[None, :], order=2)
    return G[0], H[0], SG[0]


def _zero_grad(gn, sg, assume_nonzero_x):
    if gn == 0.0 or not np.isfinite(gn):
        return True
    return (not assume_nonzero_x) and gn <= 1e-14 * float(np.sum(sg))


def affine_normal_ad(exps, coef, x, r: float = 1e-6, assume_nonzero_x: bool = False, frame=None,
                     third: str = "tensor"):
    """The 'ad' reference route: full third tensor (``third='tensor'``), or the
    same trace term contracted term by term with W = Q_T (H_T+rI)^{-1} Q_T^T
    (``third='contract'``, for large n).  Returns (nu, unit, info dict)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    g, H, sg = _grad_hess(exps, coef, x)
    gn = float(np.linalg.norm(g))
    info = dict(grad_norm=gn, logdet=0.0, flags=0, hv_evals=n, third_evals=n - 1, krylov_iters=0)
    nan = np.full(n, np.nan)
    if _zero_grad(gn, sg, assume_nonzero_x):
        info["flags"] = FLAG_ZERO_GRAD
        return nan, nan, info
    e = g / gn
    QT = (frame or qr_frame)(e)
    HT = QT.T @ H @ QT + r * np.eye(n - 1)
    h = QT.T @ H @ e
    try:
        L = np.linalg.cholesky(HT) if n > 1 else np.zeros((0, 0))
    except np.linalg.LinAlgError:
        info["flags"] = FLAG_NOT_PD
        return nan, nan, info
    info["logdet"] = float(2.0 * np.sum(np.log(np.diag(L))))
    HTinv = np.linalg.inv(HT) if n > 1 else np.zeros((0, 0))
    if third == "tensor":
        T = derivs.third_tensor(exps, coef, x)
        a = np.array([np.trace(HTinv @ (QT.T @ np.einsum("ljk,l->jk", T, QT[:, i]) @ QT)) for i in range(n - 1)])
    else:
        W = QT @ HTinv @ QT.T
        c = derivs.third_contract(exps, coef, x, W, np.eye(n))
        a = QT.T @ c
    tau = HTinv @ (h - gn / (n + 1) * a)
    nu = QT @ tau - e
    return nu, nu / np.linalg.norm(nu), info


# ----------------------------------------------------------------- stochastic

def pcg(A, b, Minv, tol: float, maxit: int):
    """Preconditioned conjugate gradients from x0 = 0 (Saad, Alg. 9.1).

    Stops before an iteration when |r_k| <= tol |b| (recursively updated
    residual) or after ``maxit`` iterations.  Returns (x, iterations,
    converged).  Each iteration applies A once."""
    x = np.zeros_like(b)
    r = b.copy()
    bn = float(np.linalg.norm(b))
    z = Minv(r)
    p = z.copy()
    rz = float(r @ z)
    k = 0
    while True:
        if float(np.linalg.norm(r)) <= tol * bn:
            return x, k, True
        if k >= maxit:
            return x, k, False
        Ap = A(p)
        alpha = rz / float(p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        k += 1
        z = Minv(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new


def affine_normal_stochastic(exps, coef, x, r: float, q: int, tol: float, maxit: int, seed: int,
                             point_index: int, precond: str = "jacobi", assume_nonzero_x: bool = False,
                             frame=None, mlp_diag_lowrank=None, probes=None):
    """MF-logDet-Stochastic (Sec. 5): the trace term a is replaced by a
    Hutchinson estimate and every tangent solve by a Krylov (PCG) solve.

    Steps, in the paper's notation:
      1. g, H at x; e = g/|g|; frame Q_T; A = H_T + r I (applied as a matrix).
      2. For s = 1..q: ambient Rademacher w_s (SplitMix64, ``rng``), probe
         z_s = Q_T^T w_s (isotropic in the tangent space, E[z z^T] = I), solve
         A y_s = z_s by PCG; c^(s)_l = sum_jk T_ljk (Q_T y_s)_j (Q_T z_s)_k.
         (y_s^T d_{t_i}H_T z_s = (Q_T^T c^(s))_i, so the mean over s of
         Q_T^T c^(s) estimates a_i = tr(H_T^{-1} d_{t_i} H_T).)
      3. a = (1/q) sum_s Q_T^T c^(s); solve A tau = h - |g|/(n+1) a by PCG;
         nu = Q_T tau - e.
    Preconditioner (a reading; the paper names none): 'jacobi' applies Q_T^T D^{-1} Q_T with
    D = |diag(H)| + r (1 where that is 0; the Jacobi matrix of the ambient H + rI carried into the
    tangent space, so iterates do not depend on the frame); 'none' is the
    identity; 'lowrank' applies Q_T^T (D + U U^T) Q_T with (D, U) given by
    ``mlp_diag_lowrank``.  ``probes`` (q x n) replaces the generated ambient
    probes (used by a test that averages over all 2^n sign vectors).
    """
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    g, H, sg = _grad_hess(exps, coef, x)
    gn = float(np.linalg.norm(g))
    info = dict(grad_norm=gn, logdet=float("nan"), flags=0, hv_evals=0, third_evals=q, krylov_iters=0)
    nan = np.full(n, np.nan)
    if _zero_grad(gn, sg, assume_nonzero_x):
        info["flags"] = FLAG_ZERO_GRAD
        return nan, nan, info
    e = g / gn
    QT = (frame or qr_frame)(e)
    HT = QT.T @ H @ QT + r * np.eye(n - 1)
    h = QT.T @ (H @ e)
    A = lambda v: HT @ v
    if precond == "jacobi":
        d = np.abs(np.diag(H)) + r
        dinv = 1.0 / np.where(d > 0.0, d, 1.0)
        Minv = lambda v: QT.T @ (dinv * (QT @ v))
    elif precond == "none":
        Minv = lambda v: v.copy()
    elif precond == "lowrank":
        D, U = mlp_diag_lowrank
        Minv = lambda v: QT.T @ (D * (QT @ v) + U @ (U.T @ (QT @ v)))
    else:
        raise ValueError(precond)
    iters = 0
    maxed = False
    cbar = np.zeros(n)
    for s in range(q):
        w = rademacher(seed, point_index, s, q, n) if probes is None else np.asarray(probes[s], np.float64)
        z = QT.T @ w
        y, k, ok = pcg(A, z, Minv, tol, maxit)
        iters += k
        maxed |= not ok
        u = QT @ y
        v = QT @ z
        cbar += derivs.third_contract(exps, coef, x, u[:, None], v[:, None])
    a = QT.T @ (cbar / q)
    tau, k, ok = pcg(A, h - gn / (n + 1) * a, Minv, tol, maxit)
    iters += k
    maxed |= not ok
    info["krylov_iters"] = iters
    info["hv_evals"] = iters + 1
    if maxed:
        info["flags"] |= FLAG_KRYLOV_MAXIT
    nu = QT @ tau - e
    return nu, nu / np.linalg.norm(nu), info


def angle_deg(u: np.ndarray, v: np.ndarray) -> float:
    """Angle between two directions (the paper's 'Angle' column, Table "accuracy")."""
    c = float(u @ v) / (np.linalg.norm(u) * np.linalg.norm(v))
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


def unit_error(u: np.ndarray, v: np.ndarray) -> float:
    """Chord distance between unit directions (the 'Unit error' column)."""
    return float(np.linalg.norm(u / np.linalg.norm(u) - v / np.linalg.norm(v)))
