"""Seeded synthetic inputs shaped like the paper's benchmark families.

This module only *draws* inputs: variable ids, exponent rows, coefficients and
evaluation points.  It performs none of the method's arithmetic (no expansion,
merging, differentiation or linear algebra), which is why both the CUDA path
and the CPU oracle may consume it.

Conventions
-----------
* A polynomial is ``Poly(var_ids, exps, coef)``: ``var_ids`` uint64[n] (unique
  variable identities, the paper's ``vars.id``, Sec. 3.2), ``exps`` uint8[m, n]
  row-major exponent matrix and ``coef`` float64[m] (the ``(n, coef, pow)``
  data model of Sec. 2, Table "apisignature").
* Rows drawn by :func:`sparse_monomials` are distinct, so random operands are
  already simplified.  The "convexified" families of the affine-normal
  experiments concatenate ``sum x_i^4 + sum x_i^2`` with a scaled random part
  and may therefore repeat a monomial; every consumer must treat repeated rows
  as a sum (that is the polynomial's meaning).
* The paper fixes seed 20260321 for its experiments (Sec. 6.1); workload k
  uses ``SEED_BASE + k``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 20260321


@dataclass
class Poly:
    var_ids: np.ndarray  # uint64[n]
    exps: np.ndarray     # uint8[m, n]
    coef: np.ndarray     # float64[m]

    @property
    def n(self) -> int:
        return int(self.exps.shape[1])

    @property
    def m(self) -> int:
        return int(self.exps.shape[0])


def _count_monomials(n: int, max_deg: int, max_active: int) -> int:
    """How many exponent rows have 1..max_active nonzero entries and total
    degree <= max_deg (used only to cap a request; exact integer count)."""
    tot = 0
    for k in range(1, min(max_active, n) + 1):
        tot += math.comb(n, k) * sum(math.comb(d - 1, k - 1) for d in range(k, max_deg + 1))
    return tot


def _draw_compact(rng: np.random.Generator, n: int, B: int, max_deg: int, max_active: int,
                  support: int | None, degree: int | None, K: int) -> np.ndarray:
    """B candidate monomials in compact form int64[B, 2K]: the first K columns
    hold the support variables in ascending order (padding n), the last K the
    matching positive exponents (padding 0)."""
    kmax = min(max_active, n)
    k = rng.integers(1, kmax + 1, size=B) if support is None else np.full(B, support, dtype=np.int64)
    d = rng.integers(k, max_deg + 1) if degree is None else np.full(B, degree, dtype=np.int64)
    col = np.arange(K)[None, :]
    # k distinct variables per row: draw with replacement, redraw rows that repeat one
    vars_ = rng.integers(0, n, size=(B, K))
    while True:
        masked = np.where(col < k[:, None], vars_, -1 - col)  # unused slots never collide
        s = np.sort(masked, axis=1)
        bad = np.any(s[:, 1:] == s[:, :-1], axis=1)
        if not bad.any():
            break
        vars_[bad] = rng.integers(0, n, size=(int(bad.sum()), K))
    # uniform composition of d into k positive parts: k-1 distinct cut points in 1..d-1
    D1 = max(int(d.max()) - 1, 1)
    u = rng.random((B, D1))
    pos = np.arange(1, D1 + 1)[None, :]
    u = np.where(pos <= (d - 1)[:, None], u, np.inf)
    su = np.sort(u, axis=1)
    thr = np.where(k >= 2, su[np.arange(B), np.clip(k - 2, 0, D1 - 1)], -np.inf)
    cutpos = np.where(u <= thr[:, None], pos, np.iinfo(np.int64).max)
    cutpos = np.sort(cutpos, axis=1)[:, :max(K - 1, 1)]
    # part j spans units (c_{j-1}, c_j] with c_{-1} = 0 and c_{k-1} = d
    bounds = np.concatenate([np.zeros((B, 1), np.int64), cutpos[:, :K - 1]], axis=1) if K > 1 \
        else np.zeros((B, 1), np.int64)
    upper = np.concatenate([bounds[:, 1:], np.zeros((B, 1), np.int64)], axis=1)
    upper = np.where(col == (k - 1)[:, None], d[:, None], upper)
    parts = np.where(col < k[:, None], upper - bounds, 0)
    vars_ = np.where(col < k[:, None], vars_, n)
    order = np.argsort(vars_, axis=1, kind="stable")
    vars_ = np.take_along_axis(vars_, order, axis=1)
    parts = np.take_along_axis(parts, order, axis=1)
    return np.concatenate([vars_, parts], axis=1)


def sparse_monomials(rng: np.random.Generator, n: int, m: int, max_deg: int, max_active: int,
                     support: int | None = None, degree: int | None = None) -> np.ndarray:
    """Draw ``m`` distinct exponent rows (uint8[m, n]).

    Each row: support size k ~ U{1..max_active} (or fixed ``support``), a
    uniform k-subset of variables, total degree ~ U{k..max_deg} (or fixed
    ``degree``) split into k positive parts by a uniform composition.  Rows are
    drawn in batches and deduplicated keeping first occurrences, so the result
    is deterministic for a seed.  A request above the number of admissible rows
    is capped at that number.
    """
    if support is not None and degree is not None:
        cap = math.comb(n, support) * math.comb(degree - 1, support - 1)
    else:
        cap = _count_monomials(n, max_deg if degree is None else degree,
                               max_active if support is None else support)
    m = min(m, cap)
    K = min(max_active, n) if support is None else support
    if 2 * m > cap:
        # close to the admissible count rejection sampling stalls: enumerate
        # every admissible row and take a uniform random subset instead
        return _all_rows_subset(rng, n, m, max_deg, max_active, support, degree)
    out = np.zeros((0, 2 * K), dtype=np.int64)
    while out.shape[0] < m:
        B = max(4 * (m - out.shape[0]), 8192)
        cand = np.concatenate([out, _draw_compact(rng, n, B, max_deg, max_active, support, degree, K)])
        _, first = np.unique(cand, axis=0, return_index=True)
        out = cand[np.sort(first)]
    out = out[:m]
    rows = np.zeros((m, n + 1), dtype=np.uint8)
    np.put_along_axis(rows, out[:, :K], out[:, K:].astype(np.uint8), axis=1)
    return np.ascontiguousarray(rows[:, :n])


def _all_rows_subset(rng, n, m, max_deg, max_active, support, degree) -> np.ndarray:
    from itertools import combinations
    ks = range(1, min(max_active, n) + 1) if support is None else [support]
    ds = range(1, max_deg + 1) if degree is None else [degree]
    rows = []
    for k in ks:
        for d in ds:
            if d < k:
                continue
            comps = [np.diff((0,) + c + (d,)) for c in combinations(range(1, d), k - 1)]
            for vs in combinations(range(n), k):
                for c in comps:
                    r = np.zeros(n, dtype=np.uint8)
                    r[list(vs)] = c
                    rows.append(r)
    rows = np.array(rows, dtype=np.uint8).reshape(-1, n)
    pick = rng.permutation(rows.shape[0])[:m]
    return np.ascontiguousarray(rows[pick])


def monolist_rows(n: int, d: int) -> np.ndarray:
    """All exponent rows with total degree <= d, in the paper's internal order
    (graded, then ascending lexicographic order of the reversed row; Sec. 3.1,
    the monolist(3,2) example).  Enumerated by brute force, used for inputs."""
    rows = []

    def rec(prefix, left, i):
        if i == n:
            rows.append(tuple(prefix))
            return
        for a in range(left + 1):
            rec(prefix + [a], left - a, i + 1)

    rec([], d, 0)
    rows.sort(key=lambda r: (sum(r), r[::-1]))
    return np.array(rows, dtype=np.uint8).reshape(-1, n)


def shell_points(rng: np.random.Generator, n: int, P: int, r0: float = 0.5, r1: float = 1.5) -> np.ndarray:
    """P points uniform (by volume) in the shell r0 <= |x| <= r1 of R^n."""
    z = rng.standard_normal((P, n))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    # volume-uniform radius: r^n ~ U[r0^n, r1^n], written so that no power overflows
    u = rng.random(P)
    rad = r1 * (u + (1.0 - u) * (r0 / r1) ** n) ** (1.0 / n)
    return np.ascontiguousarray(z * rad[:, None])


def box_points(rng: np.random.Generator, n: int, P: int) -> np.ndarray:
    return np.ascontiguousarray(rng.uniform(-1.0, 1.0, size=(P, n)))


def convexified(rng: np.random.Generator, n: int, random_exps: np.ndarray, scale: float = 0.1,
                var_ids: np.ndarray | None = None) -> Poly:
    """sum_i x_i^4 + sum_i x_i^2 + scale * (random part with N(0,1) coefficients).
    Terms are concatenated, not merged."""
    eye = np.eye(n, dtype=np.uint8)
    exps = np.concatenate([4 * eye, 2 * eye, random_exps]).astype(np.uint8)
    coef = np.concatenate([np.ones(2 * n), scale * rng.standard_normal(random_exps.shape[0])])
    ids = np.arange(n, dtype=np.uint64) if var_ids is None else var_ids
    return Poly(ids, np.ascontiguousarray(exps), coef)


# ---------------------------------------------------------------- named workloads

def affine_small(seed_off: int = 0, P: int = 1024):
    """n=3: f = sum x_i^4 + sum x_i^2 + 0.1 q, q = all 35 monomials of degree
    <= 4 (coefficients N(0,1) drawn in monolist order); P points on the shell
    0.5 <= |x| <= 1.5."""
    rng = np.random.default_rng(SEED_BASE + 0 + seed_off)
    q = monolist_rows(3, 4)
    poly = convexified(rng, 3, q, 0.1)
    X = shell_points(rng, 3, P)
    return poly, X


def affine_small_stress(seed_off: int = 0, P: int = 1024):
    """The n=3 family made indefinite so that the NOT_PD and ZERO_GRAD flags
    occur: random part scaled x10 and a saddle x1^2 - x2^2 + x3 added; the
    first 8 points are placed where the gradient vanishes exactly (the
    gradient of an odd-free even polynomial is zero at the origin) or nearly."""
    rng = np.random.default_rng(SEED_BASE + 100 + seed_off)
    q = monolist_rows(3, 4)
    eye = np.eye(3, dtype=np.uint8)
    saddle = np.array([[2, 0, 0], [0, 2, 0], [0, 0, 1]], dtype=np.uint8)
    exps = np.concatenate([4 * eye, 2 * eye, q, saddle]).astype(np.uint8)
    coef = np.concatenate([np.ones(6), 1.0 * rng.standard_normal(q.shape[0]), [1.0, -1.0, 1.0]])
    poly = Poly(np.arange(3, dtype=np.uint64), exps, coef)
    X = shell_points(rng, 3, P)
    return poly, X


def product_pair(seed_off: int = 0, n: int = 20, m: int = 2000, overlap: int = 10, max_deg: int = 6,
                 max_active: int = 4):
    """Two random sparse operands over variable-id sets that overlap in
    ``overlap`` ids (A: 0..n-1, B: n-overlap..2n-overlap-1), N(0,1) coefficients."""
    rng = np.random.default_rng(SEED_BASE + 1 + seed_off)
    ea = sparse_monomials(rng, n, m, max_deg, max_active)
    eb = sparse_monomials(rng, n, m, max_deg, max_active)
    A = Poly(np.arange(n, dtype=np.uint64), ea, rng.standard_normal(ea.shape[0]))
    B = Poly(np.arange(n - overlap, 2 * n - overlap, dtype=np.uint64), eb, rng.standard_normal(eb.shape[0]))
    return A, B


def dense_power_base(d: int, n: int = 5) -> Poly:
    """p_d = sum_{|alpha| <= d} x^alpha in n variables, all coefficients 1
    (the heavy-simplify family of Sec. 6.3)."""
    rows = monolist_rows(n, d)
    return Poly(np.arange(n, dtype=np.uint64), rows, np.ones(rows.shape[0]))


def eval_batch(seed_off: int = 0, n: int = 30, m: int = 5000, P: int = 65536, max_deg: int = 4,
               max_active: int = 4):
    """n=30, 5,000 distinct terms of degree <= 4 with <= 4 active variables,
    N(0,1) coefficients, P points uniform in [-1,1]^n."""
    rng = np.random.default_rng(SEED_BASE + 2 + seed_off)
    e = sparse_monomials(rng, n, m, max_deg, max_active)
    poly = Poly(np.arange(n, dtype=np.uint64), e, rng.standard_normal(e.shape[0]))
    X = box_points(rng, n, P)
    return poly, X


def batched_uneven(seed_off: int = 0, n_polys: int = 256, n_lo: int = 5, n_hi: int = 60,
                   t_lo: int = 50, t_hi: int = 20000, p_lo: int = 128, p_hi: int = 4096, max_deg: int = 6,
                   max_active: int = 6):
    """256 convexified polynomials: n ~ U{5..60}, random-part term count
    log-uniform in [50, 20000] (capped at the admissible count), degree <= 6,
    point count log-uniform in [128, 4096] on the shell of each."""
    rng = np.random.default_rng(SEED_BASE + 3 + seed_off)
    polys, Xs = [], []
    for _ in range(n_polys):
        n = int(rng.integers(n_lo, n_hi + 1))
        t = int(round(math.exp(rng.uniform(math.log(t_lo), math.log(t_hi)))))
        P = int(round(math.exp(rng.uniform(math.log(p_lo), math.log(p_hi)))))
        e = sparse_monomials(rng, n, t, max_deg, max_active)
        polys.append(convexified(rng, n, e, 0.1))
        Xs.append(shell_points(rng, n, P))
    return polys, Xs


def large_sparse(n: int, seed_off: int = 0, P: int = 4096, terms_per_var: int = 20, max_deg: int = 4,
                 max_active: int = 4, shell: bool = False):
    """Convexified sparse polynomial in n variables with ~20n random terms of
    degree <= 4 and <= 4 active variables; P points in [-1,1]^n (or on the
    0.5..1.5 shell)."""
    rng = np.random.default_rng(SEED_BASE + 4 + seed_off + 7 * n)
    e = sparse_monomials(rng, n, terms_per_var * n, max_deg, max_active)
    poly = convexified(rng, n, e, 0.1)
    X = shell_points(rng, n, P) if shell else box_points(rng, n, P)
    return poly, X


def sparse_quartic(n: int, m: int, support: int, seed_off: int = 0, P: int = 4096, shell: bool = True):
    """Paper-shaped sparse quartics (Sec. 6.5/6.6 families): m random monomials
    with exactly ``support`` active variables and degree 4, convexified."""
    rng = np.random.default_rng(SEED_BASE + 5 + seed_off + 11 * n)
    e = sparse_monomials(rng, n, m, 4, support, support=support, degree=4)
    poly = convexified(rng, n, e, 0.1)
    X = shell_points(rng, n, P) if shell else box_points(rng, n, P)
    return poly, X


def clustered_sparse(n: int, seed_off: int = 0, P: int = 4096, couplings=(1.8, 1.3), cluster_size: int = 0):
    """The large sparse family with soft collective modes: ``large_sparse``'s
    convexified random part plus, for each coupling J_k, a cluster S_k of
    ``cluster_size`` variables (default n // 10, at least 8; disjoint, drawn at
    random) tied by the attractive mean-field term -(J_k/|S_k|) (sum_{i in S_k}
    x_i)^2, written out as its monomials (-J_k/|S_k|) x_i^2 and (-2 J_k/|S_k|)
    x_i x_j.  Each cluster lowers the curvature along its collective
    direction (near x = 0 the Jacobi-scaled curvature is about
    1 - 2 J_k mean_i 1/(12 x_i^2 + 2)): a few soft modes that a diagonal
    preconditioner cannot see.  P points in [-1, 1]^n."""
    rng = np.random.default_rng(SEED_BASE + 6 + seed_off + 13 * n)
    e = sparse_monomials(rng, n, 20 * n, 4, 4)
    base = convexified(rng, n, e, 0.1)
    s = cluster_size or max(8, n // 10)
    perm = rng.permutation(n)
    rows, coef = [], []
    for k, J in enumerate(couplings):
        S = np.sort(perm[k * s:(k + 1) * s])
        for a in range(s):
            r = np.zeros(n, np.uint8)
            r[S[a]] = 2
            rows.append(r)
            coef.append(-J / s)
            for b in range(a + 1, s):
                r = np.zeros(n, np.uint8)
                r[S[a]] = r[S[b]] = 1
                rows.append(r)
                coef.append(-2.0 * J / s)
    poly = Poly(base.var_ids, np.concatenate([base.exps, np.array(rows, np.uint8)]),
                np.concatenate([base.coef, np.array(coef)]))
    return poly, box_points(rng, n, P)
