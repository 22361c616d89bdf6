"""Parity of simplify / mul / add (C ABI) against the engine oracle.

Bar: exponent rows bit-exact and in the same canonical order; coefficients
within 1e-12 of the oracle's sum of |contributions| per merged term; merged
terms whose oracle coefficient is within that bound of zero count as
cancelled on either side.  Exact-integer workloads (p_d^3) must match
bit-exactly in coefficients too.
"""
import numpy as np
import pytest
import torch

from oracle import engine
from paper_2604_06575_b300 import workloads
from tests.golden_io import ints, parse_terms, read_kv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pl(cuda_ok):
    from paper_2604_06575_b300 import polylab
    return polylab


def host(dp):
    return (np.asarray(dp.var_ids), dp.exps.cpu().numpy(), dp.coef.cpu().numpy())


def compare(got, ref, rel=1e-12, exact=False):
    gid, ge, gc = got
    rid, re_, rc, rs = ref
    assert [int(v) for v in gid] == [int(v) for v in rid]
    # drop near-cancelled terms on both sides before comparing
    r_keep = np.abs(rc) > rel * rs
    g_map = {r.tobytes(): c for r, c in zip(ge, gc)}
    r_map = {r.tobytes(): (c, s) for r, c, s in zip(re_, rc, rs)}
    for k, (c, s) in r_map.items():
        if abs(c) > rel * s:
            assert k in g_map, "missing term"
            if exact:
                assert g_map[k] == c
            else:
                assert abs(g_map[k] - c) <= rel * s
    for k, c in g_map.items():
        if k not in r_map:
            raise AssertionError("extra term")
    if exact or r_keep.all():
        assert np.array_equal(ge, re_), "order or rows differ"
    # canonical order of the GPU output on its own
    assert np.array_equal(ge, ge[engine.canonical_order(ge)])


def tup(p):
    return (p.var_ids, p.exps, p.coef)


@pytest.mark.parametrize("seed", range(8))
def test_mul_add_tiny_random(pl, seed):
    rng = np.random.default_rng(seed)
    na, nb = int(rng.integers(1, 5)), int(rng.integers(1, 5))
    ids_a = rng.choice(9, na, replace=False).astype(np.uint64)   # unsorted ids on purpose
    ids_b = rng.choice(9, nb, replace=False).astype(np.uint64)
    ea = rng.integers(0, 4, size=(int(rng.integers(1, 40)), na)).astype(np.uint8)
    eb = rng.integers(0, 4, size=(int(rng.integers(1, 40)), nb)).astype(np.uint8)
    a = workloads.Poly(ids_a, ea, rng.integers(-3, 4, ea.shape[0]).astype(float))
    b = workloads.Poly(ids_b, eb, rng.integers(-3, 4, eb.shape[0]).astype(float))
    da, db = pl.to_device(a), pl.to_device(b)
    compare(host(pl.mul(da, db)), engine.mul(tup(a), tup(b)), exact=True)
    compare(host(pl.add(da, db)), engine.add(tup(a), tup(b)), exact=True)
    compare(host(pl.simplify(da)), engine.simplify(*tup(a)), exact=True)


def test_paper_examples(pl):
    g = read_kv("engine_examples.txt")
    pe, pc = parse_terms(g["mixed.p.terms"])
    qe, qc = parse_terms(g["mixed.q.terms"])
    p = workloads.Poly(np.array(ints(g["mixed.p.ids"]), np.uint64), pe, pc)
    q = workloads.Poly(np.array(ints(g["mixed.q.ids"]), np.uint64), qe, qc)
    r = host(pl.add(pl.to_device(p), pl.to_device(q)))
    assert [int(v) for v in r[0]] == ints(g["mixed.r.ids"])
    re_, rc = parse_terms(g["mixed.r.terms"])
    assert {e.tobytes(): c for e, c in zip(r[1], r[2])} == {e.tobytes(): c for e, c in zip(re_, rc)}
    # (z1 + 1)^2 * 3 + 5 z2
    ids = np.array([1, 2], np.uint64)
    z1p1 = pl.to_device(workloads.Poly(ids, np.array([[1, 0], [0, 0]], np.uint8), np.array([1.0, 1.0])))
    sq = pl.mul(z1p1, z1p1)
    three = pl.to_device(workloads.Poly(ids, np.zeros((1, 2), np.uint8), np.array([3.0])))
    u = pl.add(pl.mul(sq, three), pl.to_device(workloads.Poly(ids, np.array([[0, 1]], np.uint8), np.array([5.0]))))
    e, c = parse_terms(g["subs.expect"])
    uh = host(u)
    assert {a.tobytes(): b for a, b in zip(uh[1], uh[2])} == {a.tobytes(): b for a, b in zip(e, c)}


@pytest.mark.parametrize("d,count", [(2, 462), (3, 2002), (4, 6188)])
def test_pd_cubed_exact(pl, d, count):
    p = workloads.dense_power_base(d)
    dp = pl.to_device(p)
    cube = pl.mul(pl.mul(dp, dp), dp)
    assert cube.m == count
    t = tup(p)
    ref = engine.mul(engine.mul(t, t)[:3], t)
    compare(host(cube), ref, exact=True)


def test_product_pair_full_size(pl):
    """Two 2,000-term operands in 20 variables sharing 10 ids: 4M-term expansion."""
    A, B = workloads.product_pair()
    got = host(pl.mul(pl.to_device(A), pl.to_device(B)))
    ref = engine.mul(tup(A), tup(B))
    compare(got, ref)


def test_simplify_with_repeats_and_zeroprec(pl):
    rng = np.random.default_rng(3)
    e = rng.integers(0, 3, size=(5000, 6)).astype(np.uint8)      # many repeated rows
    c = rng.standard_normal(5000)
    p = workloads.Poly(np.arange(6, dtype=np.uint64)[::-1].copy(), e, c)
    dp = pl.to_device(p)
    compare(host(pl.simplify(dp)), engine.simplify(*tup(p)))
    compare(host(pl.simplify(dp, 0.5)), engine.simplify(*tup(p), zeroprec=0.5))
    # exact cancellation removes the term
    z = workloads.Poly(np.arange(2, dtype=np.uint64), np.array([[1, 1], [1, 1], [0, 1]], np.uint8),
                       np.array([0.25, -0.25, 1.0]))
    s = host(pl.simplify(pl.to_device(z)))
    assert s[1].tolist() == [[0, 1]] and s[2].tolist() == [1.0]


def test_wide_keys_128bit(pl):
    """n=400, degree up to 12: more than 2^64 monomials, 128-bit keys."""
    rng = np.random.default_rng(5)
    ea = workloads.sparse_monomials(rng, 400, 300, 6, 4)
    eb = workloads.sparse_monomials(rng, 400, 300, 6, 4)
    a = workloads.Poly(np.arange(400, dtype=np.uint64), ea, rng.standard_normal(300))
    b = workloads.Poly(np.arange(400, dtype=np.uint64) + 200, eb, rng.standard_normal(300))
    compare(host(pl.mul(pl.to_device(a), pl.to_device(b))), engine.mul(tup(a), tup(b)))


def test_errors_and_edges(pl):
    one = workloads.Poly(np.array([1], np.uint64), np.array([[200]], np.uint8), np.array([1.0]))
    two = workloads.Poly(np.array([1], np.uint64), np.array([[100]], np.uint8), np.array([1.0]))
    with pytest.raises(pl.PolylabError) as ei:
        pl.mul(pl.to_device(one), pl.to_device(two))
    assert ei.value.status == 2
    ok = pl.mul(pl.to_device(workloads.Poly(np.array([1], np.uint64), np.array([[155]], np.uint8), np.ones(1))),
                pl.to_device(two))
    assert ok.exps.cpu().tolist() == [[255]]
    dup = workloads.Poly(np.array([4, 4], np.uint64), np.ones((1, 2), np.uint8), np.ones(1))
    with pytest.raises(pl.PolylabError) as ei:
        pl.simplify(pl.to_device(dup))
    assert ei.value.status == 3
    empty = workloads.Poly(np.array([1, 2], np.uint64), np.zeros((0, 2), np.uint8), np.zeros(0))
    r = pl.mul(pl.to_device(empty), pl.to_device(one))
    assert r.m == 0 and [int(v) for v in r.var_ids] == [1, 2]
    r = pl.simplify(pl.to_device(workloads.Poly(np.array([9], np.uint64), np.zeros((1, 1), np.uint8),
                                                np.array([0.0]))))
    assert r.m == 0
