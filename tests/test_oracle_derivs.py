"""Pins for the derivative oracle: the paper's worked gradient, closed forms on
single monomials, Euler identities for homogeneous polynomials, symmetry and
Richardson-extrapolated central differences."""
import numpy as np
import pytest

from oracle import derivs
from paper_2604_06575_b300 import workloads
from tests.golden_io import floats, read_kv


def test_paper_gradient_example_sec33():
    g = read_kv("engine_examples.txt")
    # p = x1^3 + 2 x1 x2 - x3 + 1
    exps = np.array([[3, 0, 0], [1, 1, 0], [0, 0, 1], [0, 0, 0]], np.uint8)
    coef = np.array([1.0, 2.0, -1.0, 1.0])
    X = floats(g["grad.point"])[None, :]
    F, G, H, *_ = derivs.eval_derivs(exps, coef, X)
    assert F[0] == float(g["grad.value"])
    assert np.array_equal(G[0], floats(g["grad.gradient"]))
    # Hessian by hand: [[6 x1, 2, 0], [2, 0, 0], [0, 0, 0]]
    assert np.array_equal(H[0], np.array([[6.0, 2, 0], [2, 0, 0], [0, 0, 0]]))


@pytest.mark.parametrize("a,b,d", [(3, 2, 1), (1, 0, 4), (4, 4, 0), (2, 1, 3)])
def test_single_monomial_closed_form(a, b, d):
    rng = np.random.default_rng(a * 100 + b * 10 + d)
    X = rng.uniform(-1.5, 1.5, size=(7, 3))
    c = -1.75
    F, G, H, *_ = derivs.eval_derivs(np.array([[a, b, d]], np.uint8), np.array([c]), X)
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    p = lambda base, k: base ** k if k >= 0 else 0.0 * base
    np.testing.assert_allclose(F, c * x ** a * y ** b * z ** d, rtol=1e-14)
    np.testing.assert_allclose(G[:, 0], c * a * p(x, a - 1) * y ** b * z ** d, rtol=1e-14, atol=1e-300)
    np.testing.assert_allclose(G[:, 1], c * b * x ** a * p(y, b - 1) * z ** d, rtol=1e-14, atol=1e-300)
    np.testing.assert_allclose(H[:, 0, 0], c * a * (a - 1) * p(x, a - 2) * y ** b * z ** d, rtol=1e-14, atol=1e-300)
    np.testing.assert_allclose(H[:, 0, 1], c * a * b * p(x, a - 1) * p(y, b - 1) * z ** d, rtol=1e-14, atol=1e-300)
    np.testing.assert_allclose(H[:, 2, 2], c * d * (d - 1) * x ** a * y ** b * p(z, d - 2), rtol=1e-14, atol=1e-300)
    T = derivs.third_tensor(np.array([[a, b, d]], np.uint8), np.array([c]), X[0])
    np.testing.assert_allclose(T[0, 0, 1], c * a * (a - 1) * b * p(X[0, 0], a - 2) * p(X[0, 1], b - 1) * X[0, 2] ** d,
                               rtol=1e-14, atol=1e-300)


def test_euler_identities_homogeneous():
    rng = np.random.default_rng(3)
    deg = 4
    exps = workloads.sparse_monomials(rng, 5, 30, deg, 4, degree=deg)
    coef = rng.standard_normal(exps.shape[0])
    X = rng.uniform(-1, 1, size=(5, 5))
    F, G, H, SF, SG, SH = derivs.eval_derivs(exps, coef, X)
    np.testing.assert_allclose(np.einsum("pi,pi->p", X, G), deg * F, atol=1e-13 * SF.max() * deg)
    np.testing.assert_allclose(np.einsum("pij,pj->pi", H, X), (deg - 1) * G, atol=1e-13 * SG.max() * deg)
    T = derivs.third_tensor(exps, coef, X[0])
    np.testing.assert_allclose(np.einsum("ijk,k->ij", T, X[0]), (deg - 2) * H[0], atol=1e-12 * SH.max() * deg)


def test_symmetry_and_finite_differences():
    rng = np.random.default_rng(7)
    exps = workloads.sparse_monomials(rng, 4, 25, 5, 3)
    coef = rng.standard_normal(exps.shape[0])
    x = rng.uniform(-1, 1, size=4)

    def fgh(y):
        F, G, H, *_ = derivs.eval_derivs(exps, coef, y[None, :])
        return F[0], G[0], H[0]

    def richardson(fun, i, h):
        e = np.zeros(4)
        e[i] = 1.0
        d = lambda hh: (fun(x + hh * e) - fun(x - hh * e)) / (2 * hh)
        return (4 * d(h / 2) - d(h)) / 3

    F, G, H = fgh(x)
    T = derivs.third_tensor(exps, coef, x)
    assert np.array_equal(H, H.T)
    for perm in [(1, 0, 2), (2, 1, 0), (0, 2, 1)]:
        assert np.allclose(T, T.transpose(perm), rtol=0, atol=1e-13)
    for i in range(4):
        np.testing.assert_allclose(richardson(lambda y: fgh(y)[0], i, 1e-3), G[i], rtol=1e-8, atol=1e-9)
        np.testing.assert_allclose(richardson(lambda y: fgh(y)[1], i, 1e-3), H[i], rtol=1e-8, atol=1e-9)
        np.testing.assert_allclose(richardson(lambda y: fgh(y)[2], i, 1e-3), T[i], rtol=1e-7, atol=1e-8)


def test_third_contract_matches_tensor():
    rng = np.random.default_rng(11)
    exps = workloads.sparse_monomials(rng, 5, 30, 5, 4)
    coef = rng.standard_normal(exps.shape[0])
    x = rng.uniform(-1, 1, size=5)
    T = derivs.third_tensor(exps, coef, x)
    W = rng.standard_normal((5, 5))
    W = W + W.T
    u, v = rng.standard_normal(5), rng.standard_normal(5)
    np.testing.assert_allclose(derivs.third_contract(exps, coef, x, W, np.eye(5)),
                               np.einsum("ljk,jk->l", T, W), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(derivs.third_contract(exps, coef, x, u[:, None], v[:, None]),
                               np.einsum("ljk,j,k->l", T, u, v), rtol=1e-12, atol=1e-12)


def test_abs_scales_bound_values():
    p, X = workloads.eval_batch(n=6, m=40, P=9)
    F, G, H, SF, SG, SH = derivs.eval_derivs(p.exps, p.coef, X)
    assert np.all(np.abs(F) <= SF) and np.all(np.abs(G) <= SG) and np.all(np.abs(H) <= SH)
