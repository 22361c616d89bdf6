"""Pins for the algebra oracle (integer powers, differences, symbolic partial
derivatives): the paper's printed gradient of Sec. 3.3, binomial and
multinomial coefficients, the p_d^3 counts of Sec. 6.3, the identities of
subtraction, and symbolic derivatives evaluated against the numeric
derivative oracle on random polynomials."""
import math

import numpy as np
import pytest

from oracle import derivs, engine
from paper_2604_06575_b300 import workloads
from tests.golden_io import ints, parse_terms, read_kv


def as_map(p):
    return {tuple(int(v) for v in r): float(c) for r, c in zip(p[1], p[2])}


def rand_poly(rng, n, m, deg, act):
    e = workloads.sparse_monomials(rng, n, m, deg, act)
    return workloads.Poly(np.arange(n, dtype=np.uint64), e, rng.standard_normal(e.shape[0]))


def evaluate(exps, coef, X):
    """Plain monomial sums at the rows of X (no derivative formulas)."""
    return (coef[None, :] * np.prod(X[:, None, :] ** exps[None, :, :].astype(np.float64), axis=2)).sum(axis=1)


def test_paper_gradient_symbolic_sec33():
    g = read_kv("engine_examples.txt")
    ids = np.array([1, 2, 3], np.uint64)
    p = (ids, np.array([[3, 0, 0], [1, 1, 0], [0, 0, 1], [0, 0, 0]], np.uint8), np.array([1.0, 2.0, -1.0, 1.0]))
    for v in (1, 2, 3):
        e, c = parse_terms(g[f"grad.d{v}"])
        got = engine.diff(p, v)
        assert [int(x) for x in got[0]] == [1, 2, 3]
        assert as_map(got) == {tuple(int(x) for x in r): float(cc) for r, cc in zip(e, c)}


@pytest.mark.parametrize("k", range(9))
def test_binomial_powers(k):
    p = (np.array([5], np.uint64), np.array([[1], [0]], np.uint8), np.array([1.0, 1.0]))  # x + 1
    got = engine.power(p, k)
    assert as_map(got) == {(j,): float(math.comb(k, j)) for j in range(k + 1)}


def test_multinomial_fourth_power():
    p = (np.array([1, 2, 3], np.uint64), np.eye(3, dtype=np.uint8), np.ones(3))  # x1 + x2 + x3
    got = as_map(engine.power(p, 4))
    want = {}
    for a in range(5):
        for b in range(5 - a):
            c = 4 - a - b
            want[(a, b, c)] = float(math.factorial(4) // (math.factorial(a) * math.factorial(b) * math.factorial(c)))
    assert got == want


def test_pd_cube_by_power():
    g = read_kv("engine_examples.txt")
    for d, cnt in zip((2, 3), ints(g["pd3.base_counts"])):
        p = workloads.dense_power_base(d)
        cube = engine.power((p.var_ids, p.exps, p.coef), 3)
        assert cube[1].shape[0] == math.comb(5 + 3 * d, 3 * d)
        assert np.all(cube[2] == np.round(cube[2])) and cube[2].sum() == cnt ** 3


def test_power_zero_and_one():
    rng = np.random.default_rng(2)
    p = rand_poly(rng, 4, 9, 3, 2)
    t = (p.var_ids, p.exps, p.coef)
    z = engine.power(t, 0)
    assert z[1].shape == (1, 4) and not z[1].any() and z[2][0] == 1.0
    one = engine.power(t, 1)
    s = engine.simplify(*t)
    assert np.array_equal(one[1], s[1]) and np.array_equal(one[2], s[2])


def test_subtraction_identities():
    rng = np.random.default_rng(4)
    a = rand_poly(rng, 5, 30, 4, 3)
    b = rand_poly(rng, 5, 25, 4, 3)
    ta, tb = (a.var_ids, a.exps, a.coef), (b.var_ids, b.exps, b.coef)
    assert engine.sub(ta, ta)[1].shape[0] == 0  # a - a = 0
    x = np.array([9], np.uint64)
    assert as_map(engine.sub((x, np.array([[1], [0]], np.uint8), np.array([1.0, 1.0])),
                             (x, np.array([[1], [0]], np.uint8), np.array([1.0, -1.0])))) == {(0,): 2.0}
    back = engine.add(engine.sub(ta, tb)[:3], tb)  # (a - b) + b = a up to rounding
    ref = engine.simplify(*ta)
    gm, rm = as_map(back), as_map(ref)
    assert set(k for k, v in gm.items() if abs(v) > 1e-12) == set(rm)
    assert all(abs(gm[k] - v) <= 1e-12 * max(1.0, abs(v)) for k, v in rm.items())


@pytest.mark.parametrize("seed", range(3))
def test_diff_matches_numeric_gradient(seed):
    rng = np.random.default_rng(10 + seed)
    p = rand_poly(rng, 6, 40, 5, 4)
    X = rng.uniform(-1.2, 1.2, size=(5, 6))
    _, G, *_ = derivs.eval_derivs(p.exps, p.coef, X)
    for i, v in enumerate(p.var_ids):
        ids, e, c, _ = engine.diff((p.var_ids, p.exps, p.coef), int(v))
        assert np.array_equal(ids, p.var_ids)
        np.testing.assert_allclose(evaluate(e, c, X), G[:, i], rtol=1e-12, atol=1e-12)
    assert engine.diff((p.var_ids, p.exps, p.coef), 999)[1].shape[0] == 0  # an id p does not have


def test_wrong_derivative_coefficients_are_caught(monkeypatch):
    """Coefficients scaled down (as a diff that loses the a_v factor would
    leave them) fail the numeric-gradient pin."""
    real = engine.simplify_rows

    def no_factor(rows, coef, zeroprec=0.0):
        return real(rows, np.sign(coef) * np.abs(coef) / np.maximum(1.0, np.abs(np.round(coef))), zeroprec)
    monkeypatch.setattr(engine, "simplify_rows", no_factor)
    with pytest.raises(AssertionError):
        test_diff_matches_numeric_gradient(0)
