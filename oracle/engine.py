"""Oracle: variable alignment, product expansion and simplify (plain definitions).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Polynomials are triples ``(var_ids, exps, coef)``: uint64[n] variable
identities, uint8[m, n] exponent rows, float64[m] coefficients -- the paper's
``(n, coef, pow)`` model carrying ``vars.id`` (Sec. 2 Table "apisignature",
Sec. 3.2).

Readings of the paper taken here, where it is silent or ambiguous:

* Alignment (Sec. 3.2): the merged variable space is the union of the operand
  ids in ascending id order; with ids assigned in creation order this yields
  the printed ``{x1, x2, y1, y2}``.
* ``simplify(p, zeroprec)`` (Sec. 2, Table "coresemantics"): coefficients of
  equal exponent rows are summed in input order; a merged term is dropped iff
  ``|c| <= zeroprec`` (default 0: exact zeros are removed).
* Output order: the paper's internal monomial order (Sec. 3.1, ``monolist``):
  total degree first, then ascending lexicographic order of the *reversed*
  exponent row.  The paper's displays are not consistent about term order, so
  order is a convention of this engine, fixed by the ``monolist(3,2)`` example.
* Exponents are uint8; a product exponent above 255 is an error.
"""
from __future__ import annotations

import numpy as np


class ExponentOverflow(ValueError):
    pass


def canonical_order(exps: np.ndarray) -> np.ndarray:
    """Permutation sorting rows by (total degree, reversed row) ascending."""
    exps = np.asarray(exps)
    if exps.shape[0] == 0:
        return np.zeros(0, dtype=np.int64)
    deg = exps.astype(np.int64).sum(axis=1)
    # np.lexsort: the LAST key is primary -> degree, then column n-1, ..., column 0
    keys = [exps[:, j] for j in range(exps.shape[1])] + [deg]
    return np.lexsort(keys)


def align(ids_a, ids_b):
    """Merged ascending id list and the column of every operand variable in it
    (Sec. 3.2: variable spaces are aligned by vars.id before combining)."""
    ids_a = [int(v) for v in ids_a]
    ids_b = [int(v) for v in ids_b]
    if len(set(ids_a)) != len(ids_a) or len(set(ids_b)) != len(ids_b):
        raise ValueError("duplicate variable id")
    merged = sorted(set(ids_a) | set(ids_b))
    pos = {v: i for i, v in enumerate(merged)}
    return (np.array(merged, dtype=np.uint64),
            np.array([pos[v] for v in ids_a], dtype=np.int64),
            np.array([pos[v] for v in ids_b], dtype=np.int64))


def _lift(exps, cols, n):
    out = np.zeros((exps.shape[0], n), dtype=np.uint16)
    out[:, cols] = exps
    return out


def simplify_rows(rows: np.ndarray, coef: np.ndarray, zeroprec: float = 0.0):
    """Merge equal rows (coefficients summed in input order), drop |c| <= zeroprec,
    return rows in canonical order.  Also returns sum |contributions| per merged
    row, the error scale for comparisons.  Raises ExponentOverflow above 255."""
    rows = np.asarray(rows)
    n = rows.shape[1]
    if rows.size and int(rows.max()) > 255:
        raise ExponentOverflow("exponent above 255")
    if rows.shape[0] == 0:
        return np.zeros((0, n), np.uint8), np.zeros(0), np.zeros(0)
    # group equal rows: each uint8 row is compared as one n-byte string (np.unique sorts them)
    rows8 = np.ascontiguousarray(rows, dtype=np.uint8)
    _, first, inv = np.unique(rows8.view(np.dtype((np.void, n))).reshape(-1), return_index=True,
                              return_inverse=True)
    uniq = rows8[first]
    inv = inv.reshape(-1)
    # np.bincount adds the weights in index order, i.e. in input order per group
    c = np.bincount(inv, weights=coef, minlength=uniq.shape[0])
    s = np.bincount(inv, weights=np.abs(coef), minlength=uniq.shape[0])
    keep = np.abs(c) > zeroprec
    uniq, c, s = uniq[keep], c[keep], s[keep]
    o = canonical_order(uniq)
    return uniq[o], c[o], s[o]


def simplify(var_ids, exps, coef, zeroprec: float = 0.0):
    """Sec. 2 ``simplify``: same variables, merged monomials, small terms removed."""
    e, c, s = simplify_rows(np.asarray(exps), np.asarray(coef, dtype=np.float64), zeroprec)
    return np.asarray(var_ids, dtype=np.uint64), e, c, s


def mul(a, b, zeroprec: float = 0.0):
    """Product of two polynomials ``(ids, exps, coef)``: align ids, form every
    pair (i, j) with exponent a_i + b_j and coefficient ca_i * cb_j (one IEEE
    multiply), then simplify.  Pairs are enumerated i-major, j-minor."""
    ids, ca_cols, cb_cols = align(a[0], b[0])
    n = len(ids)
    ea = _lift(np.asarray(a[1]), ca_cols, n)
    eb = _lift(np.asarray(b[1]), cb_cols, n)
    ma, mb = ea.shape[0], eb.shape[0]
    rows = (ea[:, None, :] + eb[None, :, :]).reshape(ma * mb, n)
    coefs = (np.asarray(a[2], np.float64)[:, None] * np.asarray(b[2], np.float64)[None, :]).reshape(-1)
    e, c, s = simplify_rows(rows, coefs, zeroprec)
    return ids, e, c, s


def add(a, b, zeroprec: float = 0.0):
    """Sum of two polynomials: align ids, concatenate terms, simplify (Sec. 3.2)."""
    ids, ca_cols, cb_cols = align(a[0], b[0])
    n = len(ids)
    rows = np.concatenate([_lift(np.asarray(a[1]), ca_cols, n), _lift(np.asarray(b[1]), cb_cols, n)])
    coefs = np.concatenate([np.asarray(a[2], np.float64), np.asarray(b[2], np.float64)])
    e, c, s = simplify_rows(rows, coefs, zeroprec)
    return ids, e, c, s


def coefficient_of(a, b, target_row_merged: np.ndarray) -> tuple[float, float]:
    """Coefficient (and sum of |contributions|) of one monomial of a*b, computed
    directly from the definition: the sum over pairs (i, j) whose exponent rows
    add up to the target, in i-major order.  Used to check single outputs of
    full-size products."""
    ids, ca_cols, cb_cols = align(a[0], b[0])
    n = len(ids)
    ea = _lift(np.asarray(a[1]), ca_cols, n).astype(np.int64)
    eb = _lift(np.asarray(b[1]), cb_cols, n).astype(np.int64)
    t = np.asarray(target_row_merged, dtype=np.int64)
    need = t[None, :] - ea                                  # b-row each a-term needs
    multi: dict[bytes, list[int]] = {}  # b rows may repeat: keep every index
    for j, row in enumerate(eb):
        multi.setdefault(row.tobytes(), []).append(j)
    tot, absum = 0.0, 0.0
    ca, cb = np.asarray(a[2], np.float64), np.asarray(b[2], np.float64)
    for i in range(ea.shape[0]):
        if need[i].min() < 0:
            continue
        for j in multi.get(need[i].tobytes(), ()):
            v = ca[i] * cb[j]
            tot += v
            absum += abs(v)
    return tot, absum


def sub(a, b, zeroprec: float = 0.0):
    """a - b (Table "coresemantics" "minus"): the sum of a and b with b's
    coefficients negated, simplified as ``add``."""
    return add(a, (b[0], b[1], -np.asarray(b[2], np.float64)), zeroprec)


def power(p, k: int, zeroprec: float = 0.0):
    """p^k (Table "coresemantics" "mpower"/"prod"): the left-to-right product
    p * p * ... * p of k factors, each partial product simplified as by
    ``mul``; k = 0 is the constant 1 over p's variables."""
    if k < 0:
        raise ValueError("negative power")
    ids = np.asarray(p[0], dtype=np.uint64)
    if k == 0:
        n = len(ids)
        one = np.ones(1)
        return ids, np.zeros((1, n), np.uint8), one, one.copy()
    acc = simplify(p[0], p[1], p[2], zeroprec)
    for _ in range(k - 1):
        acc = mul(acc[:3], p, zeroprec)
    return acc


def diff(p, var_id: int, zeroprec: float = 0.0):
    """d p / d x_v for the variable with id ``var_id`` (Sec. 3.3: term by term,
    c x^a -> a_v c x^(a - e_v); terms without x_v vanish), simplified; an id p
    does not have gives the zero polynomial."""
    ids = np.asarray(p[0], dtype=np.uint64)
    exps = np.asarray(p[1])
    coef = np.asarray(p[2], np.float64)
    hit = np.nonzero(ids == np.uint64(var_id))[0]
    if hit.size == 0:
        n = len(ids)
        return ids, np.zeros((0, n), np.uint8), np.zeros(0), np.zeros(0)
    v = int(hit[0])
    keep = exps[:, v] > 0
    rows = exps[keep].astype(np.int64)
    c = coef[keep] * rows[:, v]
    rows[:, v] -= 1
    e, cc, s = simplify_rows(rows.astype(np.uint8), c, zeroprec)
    return ids, e, cc, s

