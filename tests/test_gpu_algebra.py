"""Parity of the algebra entry points (polylab_sub, polylab_pow,
polylab_diff) against the oracle, with the engine's bar: exponent rows
bit-exact and in canonical order, coefficients within 1e-12 of the oracle's
sum of |contributions| (bit-exact for integer-coefficient powers)."""
import numpy as np
import pytest
import torch

from oracle import engine
from paper_2604_06575_b300 import workloads
from tests.test_gpu_engine import compare, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pl(cuda_ok):
    from paper_2604_06575_b300 import polylab
    return polylab


def rand_poly(rng, n, m, deg, act, ids=None):
    e = workloads.sparse_monomials(rng, n, m, deg, act)
    ids = np.arange(n, dtype=np.uint64) if ids is None else np.asarray(ids, np.uint64)
    return workloads.Poly(ids, e, rng.standard_normal(e.shape[0]))


def t(p):
    return (p.var_ids, p.exps, p.coef)


@pytest.mark.parametrize("seed", range(4))
def test_sub_random_mixed_ids(pl, seed):
    rng = np.random.default_rng(seed)
    a = rand_poly(rng, 6, 40, 4, 3, ids=[1, 3, 5, 7, 9, 11])
    b = rand_poly(rng, 5, 35, 4, 3, ids=[2, 3, 4, 9, 20])
    got = pl.sub(pl.to_device(a), pl.to_device(b))
    compare(host(got), engine.sub(t(a), t(b)))
    z = pl.sub(pl.to_device(a), pl.to_device(a))
    assert z.m == 0


@pytest.mark.parametrize("d,k", [(2, 3), (3, 3), (2, 5), (1, 7)])
def test_pow_dense_base_exact(pl, d, k):
    p = workloads.dense_power_base(d)
    got = pl.pow(pl.to_device(p), k)
    compare(host(got), engine.power(t(p), k), exact=True)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_pow_random(pl, k):
    rng = np.random.default_rng(40 + k)
    p = rand_poly(rng, 5, 12, 3, 3)
    got = pl.pow(pl.to_device(p), k)
    ref = engine.power(t(p), k)
    # binary exponentiation associates the sums differently: bound by the
    # oracle's sum of |contributions| of the left-to-right product
    compare(host(got), ref, rel=1e-11)


def test_pow_overflow(pl):
    p = workloads.Poly(np.array([3], np.uint64), np.array([[200]], np.uint8), np.ones(1))
    with pytest.raises(RuntimeError, match="EXP_OVERFLOW"):
        pl.pow(pl.to_device(p), 2)


@pytest.mark.parametrize("seed", range(3))
def test_diff_and_jacobian(pl, seed):
    rng = np.random.default_rng(70 + seed)
    p = rand_poly(rng, 8, 60, 5, 4, ids=[10, 20, 30, 40, 50, 60, 70, 80])
    dp = pl.to_device(p)
    jac = pl.jacobian(dp)
    assert len(jac) == 8
    for v, d in zip(p.var_ids, jac):
        compare(host(d), engine.diff(t(p), int(v)))
    assert pl.diff(dp, 999).m == 0


def test_paper_gradient_sec33(pl):
    p = workloads.Poly(np.array([1, 2, 3], np.uint64),
                       np.array([[3, 0, 0], [1, 1, 0], [0, 0, 1], [0, 0, 0]], np.uint8), np.array([1.0, 2.0, -1.0, 1.0]))
    dp = pl.to_device(p)
    for v in (1, 2, 3):
        compare(host(pl.diff(dp, v)), engine.diff(t(p), v), exact=True)
