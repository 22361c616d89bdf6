"""Pins for the affine-normal oracle.

* the paper's printed worked example (Sec. 5), all shown digits;
* classical affine differential geometry: affine normals of a quadric pass
  through its centre; the affine normal of a plane curve y = phi(x) is
  parallel to (-phi'''/(3 phi''), phi'' - phi' phi'''/(3 phi'')) (derivative of
  the affine tangent with respect to affine arc length ds = phi''^(1/3) dx);
* equiaffine covariance: for g(y) = f(My + b), M nu_g(y) is a positive
  multiple of nu_f(My + b) -- this fixes the |g|/(n+1) weight of the trace term;
* frame independence; tensor and term-by-term contractions agree;
* the stochastic estimator equals the exact one when the probes are all 2^n
  sign vectors (their second moment is exactly the identity);
* PCG against a direct solve; flags.
"""
import itertools

import numpy as np
import pytest

from oracle import affine, derivs, engine
from paper_2604_06575_b300 import workloads
from tests.golden_io import floats, parse_terms, read_kv


def test_worked_example_sec5():
    g = read_kv("affine_worked_example.txt")
    exps, coef = parse_terms(g["terms"])
    x0 = floats(g["x0"])
    nu, unit, info = affine.affine_normal_ad(exps, coef, x0, r=float(g["regularization"]))
    d = floats(g["d"])
    # 7 significant digits are printed: half a unit in the last place
    assert np.all(np.abs(nu - d) <= 0.5e-6 * np.abs(d))
    assert abs(info["grad_norm"] - float(g["grad_norm"])) <= 0.5e-6 * float(g["grad_norm"])
    assert info["hv_evals"] == int(g["hv_evals"]) and info["third_evals"] == int(g["third_evals"])
    assert nu @ (unit / np.linalg.norm(unit)) > 0
    # the regularisation must enter the tau solve: without it the third entry is ~1e-16
    nu0, _, _ = affine.affine_normal_ad(exps, coef, x0, r=0.0)
    assert abs(nu0[2]) < 1e-14


def quadric(A, c):
    """(x-c)^T A (x-c) as explicit terms."""
    n = len(c)
    rows, coefs = [], []
    for i in range(n):
        for j in range(n):
            r = np.zeros(n, np.uint8)
            r[i] += 1
            r[j] += 1
            rows.append(r)
            coefs.append(A[i, j])
        r = np.zeros(n, np.uint8)
        r[i] = 1
        rows.append(r)
        coefs.append(-2.0 * (A[i] @ c))
    rows.append(np.zeros(n, np.uint8))
    coefs.append(c @ A @ c)
    return np.array(rows), np.array(coefs)


@pytest.mark.parametrize("n", [2, 3, 5])
def test_quadric_normals_pass_through_centre(n):
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    A = B @ B.T + n * np.eye(n)
    c = rng.standard_normal(n)
    exps, coef = quadric(A, c)
    for _ in range(3):
        x = c + rng.standard_normal(n)
        nu, unit, info = affine.affine_normal_ad(exps, coef, x, r=0.0)
        d = (c - x) / np.linalg.norm(c - x)
        assert unit @ d == pytest.approx(1.0, abs=1e-12)


def test_plane_curve_closed_form():
    # f(x1, x2) = phi(x1) - x2, phi(t) = t^3 + 2 t^2 + t/2
    exps = np.array([[3, 0], [2, 0], [1, 0], [0, 1]], np.uint8)
    coef = np.array([1.0, 2.0, 0.5, -1.0])
    for t in (0.3, -0.1, 1.2):
        d1, d2, d3 = 3 * t * t + 4 * t + 0.5, 6 * t + 4, 6.0
        N = np.array([-d3 / (3 * d2), d2 - d1 * d3 / (3 * d2)])
        nu, unit, _ = affine.affine_normal_ad(exps, coef, np.array([t, 0.7]), r=0.0)
        assert unit @ (N / np.linalg.norm(N)) == pytest.approx(1.0, abs=1e-13)


def substitute_affine(exps, coef, M, b):
    """Expand f(My + b) with the engine oracle (products and sums only)."""
    n = M.shape[0]
    ids = np.arange(n, dtype=np.uint64)
    lin = []
    for i in range(n):
        rows = np.vstack([np.eye(n, dtype=np.uint8), np.zeros((1, n), np.uint8)])
        lin.append((ids, rows, np.concatenate([M[i], [b[i]]])))
    acc = (ids, np.zeros((1, n), np.uint8), np.array([0.0]))
    for row, c in zip(exps, coef):
        term = (ids, np.zeros((1, n), np.uint8), np.array([c]))
        for i in range(n):
            for _ in range(int(row[i])):
                term = engine.mul(term, lin[i])[:3]
        acc = engine.add(acc, term)[:3]
    return acc[1], acc[2]


@pytest.mark.parametrize("seed", [0, 1])
def test_affine_covariance(seed):
    rng = np.random.default_rng(100 + seed)
    n = 3
    rnd = workloads.sparse_monomials(rng, n, 12, 4, 3)
    f = workloads.convexified(rng, n, rnd, 0.1)
    M = rng.standard_normal((n, n))
    if seed == 1:
        M[:, 0] *= -1.0  # orientation reversing
    b = rng.standard_normal(n) * 0.3
    ge, gc = substitute_affine(f.exps, f.coef, M, b)
    for _ in range(3):
        y = rng.standard_normal(n) * 0.5
        x = M @ y + b
        nu_f, uf, _ = affine.affine_normal_ad(f.exps, f.coef, x, r=0.0)
        nu_g, ug, _ = affine.affine_normal_ad(ge, gc, y, r=0.0)
        v = M @ nu_g
        assert (v / np.linalg.norm(v)) @ uf == pytest.approx(1.0, abs=1e-11)


def test_frame_independence():
    g = read_kv("affine_worked_example.txt")
    exps, coef = parse_terms(g["terms"])
    x0 = floats(g["x0"])
    rng = np.random.default_rng(5)

    def random_frame(e):
        n = e.shape[0]
        M = np.column_stack([e, rng.standard_normal((n, n - 1))])
        Q, _ = np.linalg.qr(M)
        return Q[:, 1:]

    def householder_frame(e):
        n = e.shape[0]
        s = 1.0 if e[-1] >= 0 else -1.0
        v = e.copy()
        v[-1] += s
        Pm = np.eye(n) - 2 * np.outer(v, v) / (v @ v)
        return Pm[:, : n - 1]

    ref, _, _ = affine.affine_normal_ad(exps, coef, x0, r=1e-8)
    for fr in (random_frame, random_frame, householder_frame):
        nu, _, _ = affine.affine_normal_ad(exps, coef, x0, r=1e-8, frame=fr)
        np.testing.assert_allclose(nu, ref, rtol=1e-12, atol=1e-12)


def test_tensor_and_contract_routes_agree():
    p, X = workloads.batched_uneven(n_polys=1, n_lo=6, n_hi=6, t_lo=40, t_hi=40, p_lo=4, p_hi=4)
    for x in X[0]:
        a, _, _ = affine.affine_normal_ad(p[0].exps, p[0].coef, x, r=1e-6, third="tensor")
        b, _, _ = affine.affine_normal_ad(p[0].exps, p[0].coef, x, r=1e-6, third="contract")
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-12)


def test_stochastic_with_all_sign_vectors_is_exact():
    g = read_kv("affine_worked_example.txt")
    exps, coef = parse_terms(g["terms"])
    x0 = floats(g["x0"])
    n = 4
    signs = np.array(list(itertools.product([1.0, -1.0], repeat=n)))
    ex, _, _ = affine.affine_normal_ad(exps, coef, x0, r=1e-3)
    st, _, info = affine.affine_normal_stochastic(exps, coef, x0, r=1e-3, q=len(signs), tol=1e-14, maxit=60,
                                                  seed=0, point_index=0, probes=signs)
    np.testing.assert_allclose(st, ex, rtol=1e-10, atol=1e-10)
    # with one random probe the estimate differs (the test above is not vacuous)
    one, _, _ = affine.affine_normal_stochastic(exps, coef, x0, r=1e-3, q=1, tol=1e-14, maxit=60,
                                                seed=3, point_index=0)
    assert np.abs(one - ex).max() > 1e-6


def test_stochastic_converges_with_probe_count():
    rng = np.random.default_rng(9)
    n = 6
    f = workloads.convexified(rng, n, workloads.sparse_monomials(rng, n, 17, 4, 4), 0.3)
    x = workloads.shell_points(rng, n, 1)[0]
    ex, ue, _ = affine.affine_normal_ad(f.exps, f.coef, x, r=1e-8)
    errs = []
    for q in (4, 64, 1024):
        ang = [affine.angle_deg(affine.affine_normal_stochastic(f.exps, f.coef, x, 1e-8, q, 1e-10, 80, s, 0)[0], ex)
               for s in range(4)]
        errs.append(np.mean(ang))
    assert errs[2] < errs[0] and errs[2] < 0.5 * errs[0]


def test_pcg_matches_direct_solve():
    rng = np.random.default_rng(4)
    for n in (1, 5, 30):
        B = rng.standard_normal((n, n))
        A = B @ B.T + 0.5 * np.eye(n)
        b = rng.standard_normal(n)
        d = 1.0 / np.diag(A)
        x, k, ok = affine.pcg(lambda v: A @ v, b, lambda v: d * v, 1e-12, 500)
        assert ok
        np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-10)
    x, k, ok = affine.pcg(lambda v: A @ v, b, lambda v: v, 1e-30, 3)
    assert k == 3 and not ok


def test_flags_and_degenerate_cases():
    # saddle x1^2 - x2^2 + x3: tangent Hessian indefinite
    exps = np.array([[2, 0, 0], [0, 2, 0], [0, 0, 1]], np.uint8)
    coef = np.array([1.0, -1.0, 1.0])
    nu, _, info = affine.affine_normal_ad(exps, coef, np.array([0.5, 0.3, 0.1]), r=1e-8)
    assert info["flags"] == affine.FLAG_NOT_PD and np.all(np.isnan(nu))
    # zero gradient at the origin
    nu, _, info = affine.affine_normal_ad(np.array([[2, 0], [0, 2]], np.uint8), np.ones(2), np.zeros(2))
    assert info["flags"] == affine.FLAG_ZERO_GRAD and np.all(np.isnan(nu))
    # n = 1: the tangent space is empty and nu = -e
    nu, _, info = affine.affine_normal_ad(np.array([[2], [1]], np.uint8), np.ones(2), np.array([1.0]))
    assert info["flags"] == 0 and nu[0] == -1.0
