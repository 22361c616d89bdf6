"""Oracle: value, gradient, Hessian and third derivatives of a sparse polynomial.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Plain definition (Sec. 3.3 differentiates term by term): for a term c*x^alpha
and a multiset of variable indices I with multiplicity m_v of variable v,

    d^I x^alpha = prod_v falling(alpha_v, m_v) * x^(alpha - m),
    falling(a, k) = a (a-1) ... (a-k+1)   (zero when k > a).

So d_i x^a = a_i x^(a-e_i), d_ij x^a = a_i (a_j - delta_ij) x^(a-e_i-e_j) and
d_ijk likewise.  Powers are evaluated by repeated multiplication.  Alongside
every derivative the oracle accumulates sum |term contribution|, the scale
that the engine's tolerances are stated against ("relative to the sum of
|terms|").
"""
from __future__ import annotations

from itertools import combinations_with_replacement

import numpy as np


def falling(a: int, k: int) -> int:
    out = 1
    for i in range(k):
        out *= (a - i)
    return out


def ipow(x: np.ndarray, k: int) -> np.ndarray:
    """x**k by repeated multiplication (k >= 0)."""
    out = np.ones_like(x)
    for _ in range(k):
        out = out * x
    return out


def _monomial_derivative(alpha: dict, idx: tuple):
    """Coefficient factor and shifted exponents of d^idx x^alpha (alpha: var->exp)."""
    mult: dict[int, int] = {}
    for v in idx:
        mult[v] = mult.get(v, 0) + 1
    fac = 1
    for v, k in mult.items():
        fac *= falling(alpha.get(v, 0), k)
        if fac == 0:
            return 0, None
    shifted = {v: a - mult.get(v, 0) for v, a in alpha.items()}
    return fac, shifted


def eval_derivs(exps: np.ndarray, coef: np.ndarray, X: np.ndarray, order: int = 2):
    """F[P], G[P,n], H[P,n,n] and their |contribution| sums SF, SG, SH.

    ``order`` 0, 1 or 2 selects how many of F, G, H are formed (the others are
    returned as None)."""
    exps = np.asarray(exps)
    X = np.asarray(X, dtype=np.float64)
    P, n = X.shape
    F = np.zeros(P)
    SF = np.zeros(P)
    G = np.zeros((P, n)) if order >= 1 else None
    SG = np.zeros((P, n)) if order >= 1 else None
    H = np.zeros((P, n, n)) if order >= 2 else None
    SH = np.zeros((P, n, n)) if order >= 2 else None
    for t in range(exps.shape[0]):
        alpha = {int(v): int(exps[t, v]) for v in np.nonzero(exps[t])[0]}
        c = float(coef[t])
        sup = sorted(alpha)

        def value(shifted):
            out = np.full(P, 1.0)
            for v, a in shifted.items():
                out = out * ipow(X[:, v], a)
            return out

        val = c * value(alpha)
        F += val
        SF += np.abs(val)
        if order >= 1:
            for i in sup:
                fac, sh = _monomial_derivative(alpha, (i,))
                if fac:
                    contrib = (c * fac) * value(sh)
                    G[:, i] += contrib
                    SG[:, i] += np.abs(contrib)
        if order >= 2:
            for i in sup:
                for j in sup:
                    fac, sh = _monomial_derivative(alpha, (i, j))
                    if fac:
                        contrib = (c * fac) * value(sh)
                        H[:, i, j] += contrib
                        SH[:, i, j] += np.abs(contrib)
    return F, G, H, SF, SG, SH


def third_tensor(exps: np.ndarray, coef: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Full third-derivative tensor T[l, j, k] = d_l d_j d_k f(x) at one point."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    T = np.zeros((n, n, n))
    for t in range(exps.shape[0]):
        alpha = {int(v): int(exps[t, v]) for v in np.nonzero(exps[t])[0]}
        c = float(coef[t])
        sup = sorted(alpha)
        for l in sup:
            for j in sup:
                for k in sup:
                    fac, sh = _monomial_derivative(alpha, (l, j, k))
                    if fac:
                        val = 1.0
                        for v, a in sh.items():
                            val *= float(ipow(np.array(x[v]), a))
                        T[l, j, k] += c * fac * val
    return T


def third_contract(exps: np.ndarray, coef: np.ndarray, x: np.ndarray, U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """c[l] = sum_{j,k} d_l d_j d_k f(x) * sum_s U[j,s] V[k,s], term by term.

    With U = W (symmetric n x n) and V = I this is sum_jk T_ljk W_jk; with
    U = u, V = v (n x 1) it is sum_jk T_ljk u_j v_k.  The tensor is never formed,
    so this serves large n; it is pinned against ``third_tensor`` at small n."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    c = np.zeros(n)
    for t in range(exps.shape[0]):
        alpha = {int(v): int(exps[t, v]) for v in np.nonzero(exps[t])[0]}
        ct = float(coef[t])
        sup = sorted(alpha)
        for l in sup:
            for j in sup:
                for k in sup:
                    fac, sh = _monomial_derivative(alpha, (l, j, k))
                    if fac:
                        val = 1.0
                        for v, a in sh.items():
                            val *= float(ipow(np.array(x[v]), a))
                        c[l] += ct * fac * val * float(U[j] @ V[k])
    return c


def derivative_multisets(k: int, order: int):
    """All index multisets of a given order over k support slots (used by tests)."""
    return list(combinations_with_replacement(range(k), order))
