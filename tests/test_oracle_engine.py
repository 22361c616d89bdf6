"""Pins for the engine oracle (alignment, expansion, simplify, monomial order).

Each test ties ``oracle.engine`` to something other than itself: the paper's
printed examples (tests/golden/), brute force over tiny inputs written here
with plain dicts, and closed-form counts.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import engine
from paper_2604_06575_b300 import workloads
from tests.golden_io import ints, parse_terms, read_kv, read_rows


def P(ids, rows, coefs):
    return (np.array(ids, dtype=np.uint64), np.array(rows, dtype=np.uint8).reshape(len(coefs), len(ids)),
            np.array(coefs, dtype=np.float64))


def var(ids, k):
    """The polynomial x_k over variable ids ``ids``."""
    row = [0] * len(ids)
    row[ids.index(k)] = 1
    return P(ids, [row], [1.0])


def const(ids, c):
    return P(ids, [[0] * len(ids)], [c])


def scale(p, c):
    return (p[0], p[1], p[2] * c)


def as_set(p):
    return {tuple(int(v) for v in r): float(c) for r, c in zip(p[1], p[2])}


def test_monolist_order_matches_paper():
    rows = read_rows("monolist_3_2.txt")
    rng = np.random.default_rng(0)
    shuffled = rows[rng.permutation(len(rows))]
    assert np.array_equal(shuffled[engine.canonical_order(shuffled)], rows)
    assert len(rows) == math.comb(5, 2)


def test_canonical_order_is_graded_colex_on_all_small_rows():
    rows = np.array([r for r in itertools.product(range(4), repeat=3)], dtype=np.uint8)
    o = rows[engine.canonical_order(rows)]
    keys = [(int(r.sum()), tuple(int(v) for v in r[::-1])) for r in o]
    assert keys == sorted(keys)


def test_scalar_example_sec31():
    g = read_kv("engine_examples.txt")
    ids = ints(g["scalar.ids"])
    x1, x2, x3 = (var(ids, k) for k in ids)
    p = engine.mul(engine.mul(x1, x1)[:3], x1)[:3]
    p = engine.add(p, scale(engine.mul(x1, x2)[:3], 2.0))[:3]
    p = engine.add(p, scale(x3, -1.0))[:3]
    p = engine.add(p, const(ids, 1.0))[:3]
    e, c = parse_terms(g["scalar.expect"])
    assert as_set(p) == as_set(P(ids, e, c))
    assert int(p[1].astype(int).sum(axis=1).max()) == int(g["scalar.degree"])


def test_mixed_variable_alignment_sec32():
    g = read_kv("engine_examples.txt")
    pe, pc = parse_terms(g["mixed.p.terms"])
    qe, qc = parse_terms(g["mixed.q.terms"])
    p = P(ints(g["mixed.p.ids"]), pe, pc)
    q = P(ints(g["mixed.q.ids"]), qe, qc)
    ids, e, c, s = engine.add(p, q)
    assert [int(v) for v in ids] == ints(g["mixed.r.ids"])
    re_, rc = parse_terms(g["mixed.r.terms"])
    assert as_set((ids, e, c)) == as_set(P(ints(g["mixed.r.ids"]), re_, rc))


def test_substitution_example_sec33():
    g = read_kv("engine_examples.txt")
    ids = ints(g["subs.ids"])
    z1p1 = engine.add(var(ids, 1), const(ids, 1.0))[:3]
    u = engine.add(scale(engine.mul(z1p1, z1p1)[:3], 3.0), scale(var(ids, 2), 5.0))[:3]
    e, c = parse_terms(g["subs.expect"])
    assert as_set(u) == as_set(P(ids, e, c))


def test_quadprod_example_sec33():
    g = read_kv("engine_examples.txt")
    ids = ints(g["quadprod.ids"])
    b = [var(ids, 1), engine.mul(var(ids, 2), var(ids, 3))[:3]]
    Q = [[2.0, 1.0], [1.0, 3.0]]
    acc = const(ids, 0.0)
    for i in range(2):
        for j in range(2):
            acc = engine.add(acc, scale(engine.mul(b[i], b[j])[:3], Q[i][j]))[:3]
    e, c = parse_terms(g["quadprod.expect"])
    assert as_set(acc) == as_set(P(ids, e, c))


def test_trace_example_sec31():
    g = read_kv("engine_examples.txt")
    ids = ints(g["trace.ids"])
    t = engine.add(engine.add(var(ids, 1), const(ids, 1.0))[:3], engine.add(var(ids, 1), var(ids, 2))[:3])
    e, c = parse_terms(g["trace.expect"])
    assert as_set(t[:3]) == as_set(P(ids, e, c))


def brute_mul(a, b):
    """Plain dict expansion over named variables, written independently."""
    acc = {}
    for ra, ca in zip(a[1], a[2]):
        da = {int(a[0][k]): int(ra[k]) for k in range(len(a[0])) if ra[k]}
        for rb, cb in zip(b[1], b[2]):
            d = dict(da)
            for k in range(len(b[0])):
                if rb[k]:
                    d[int(b[0][k])] = d.get(int(b[0][k]), 0) + int(rb[k])
            key = tuple(sorted(d.items()))
            acc[key] = acc.get(key, 0.0) + float(ca) * float(cb)
    return {k: v for k, v in acc.items() if v != 0.0}


def named(p):
    out = {}
    for r, c in zip(p[1], p[2]):
        out[tuple(sorted((int(p[0][k]), int(r[k])) for k in range(len(p[0])) if r[k]))] = float(c)
    return out


@pytest.mark.parametrize("seed", range(6))
def test_mul_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    na, nb = int(rng.integers(1, 4)), int(rng.integers(1, 4))
    ids_a = sorted(rng.choice(6, na, replace=False).tolist())
    ids_b = rng.choice(6, nb, replace=False).tolist()  # unsorted on purpose
    ea = rng.integers(0, 3, size=(int(rng.integers(1, 6)), na))
    eb = rng.integers(0, 3, size=(int(rng.integers(1, 6)), nb))
    a = P(ids_a, ea, rng.integers(-3, 4, ea.shape[0]).astype(float))
    b = P(ids_b, eb, rng.integers(-3, 4, eb.shape[0]).astype(float))
    ids, e, c, s = engine.mul(a, b)
    assert [int(v) for v in ids] == sorted(set(ids_a) | set(ids_b))
    assert named((ids, e, c)) == brute_mul(a, b)
    assert np.array_equal(e, e[engine.canonical_order(e)])


def test_pd3_counts_and_coefficients():
    g = read_kv("engine_examples.txt")
    counts = ints(g["pd3.base_counts"])
    for d, cnt in zip((2, 3), counts):
        p = workloads.dense_power_base(d)
        assert p.m == cnt == math.comb(5 + d, d)
        t = (p.var_ids, p.exps, p.coef)
        ids, e, c, s = engine.mul(engine.mul(t, t)[:3], t)
        # the cube has every monomial of degree <= 3d
        assert e.shape[0] == math.comb(5 + 3 * d, 3 * d)
        # coefficients are exact integers; their sum is p(1,...,1)^3
        assert np.all(c == np.round(c)) and c.sum() == cnt ** 3
    # coefficient = number of ordered triples (a, b, c) of base monomials with a+b+c = target
    p = workloads.dense_power_base(2)
    base = [tuple(int(v) for v in r) for r in p.exps]
    cube = engine.mul(engine.mul((p.var_ids, p.exps, p.coef), (p.var_ids, p.exps, p.coef))[:3],
                      (p.var_ids, p.exps, p.coef))
    got = {tuple(int(v) for v in r): cc for r, cc in zip(cube[1], cube[2])}
    triples = {}
    for a in base:
        for b in base:
            for c in base:
                k = tuple(x + y + z for x, y, z in zip(a, b, c))
                triples[k] = triples.get(k, 0) + 1
    assert got == {k: float(v) for k, v in triples.items()}


def test_zeroprec_and_cancellation():
    ids = [1, 2]
    p = P(ids, [[1, 0], [1, 0], [0, 1], [0, 0]], [0.5, -0.5, 1e-9, 2.0])
    _, e, c, _ = engine.simplify(*p)
    assert as_set((ids, e, c)) == {(0, 0): 2.0, (0, 1): 1e-9}
    _, e, c, _ = engine.simplify(*p, zeroprec=1e-6)
    assert as_set((ids, e, c)) == {(0, 0): 2.0}


def test_exponent_overflow_raises():
    a = P([1], [[200]], [1.0])
    b = P([1], [[100]], [1.0])
    with pytest.raises(engine.ExponentOverflow):
        engine.mul(a, b)
    ok = engine.mul(P([1], [[155]], [1.0]), b)
    assert int(ok[1][0, 0]) == 255


def test_duplicate_ids_rejected():
    with pytest.raises(ValueError):
        engine.align([1, 1], [2])


def test_coefficient_of_matches_full_product():
    A, B = workloads.product_pair(n=6, m=40, overlap=3)
    a, b = (A.var_ids, A.exps, A.coef), (B.var_ids, B.exps, B.coef)
    ids, e, c, s = engine.mul(a, b)
    for k in range(0, e.shape[0], 17):
        v, av = engine.coefficient_of(a, b, e[k])
        assert v == pytest.approx(c[k], abs=1e-14 * av)
        assert av == pytest.approx(s[k], rel=1e-14)
