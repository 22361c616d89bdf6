"""Parity of the 'ad' route on the GPU (POLYLAB_AD: the affine-normal direction
from the materialised third-derivative tensor, Sec. 5) against the oracle's
'ad' route with the full tensor (``third='tensor'``).

FP64 bar as for the exact method: |nu_gpu - nu_oracle| <= 1e-11 * kappa *
|nu_oracle| with kappa the condition number of H_T + r I; flags equal except
at points where H_T + r I is singular to 1e-10 of its norm.  Cases: the
worked example of Sec. 5, the n = 3 family at every point (more points than
CTAs, so the grid-stride loop runs), the flag stress family, the paper's
accuracy-table shape (n = 6, 17 monomials), terms with 7 and 8 active
variables, the largest n the route takes, n = 1, no points, and the argument
errors (n above the limit, a reduced precision).
"""
import numpy as np
import pytest
import torch

from oracle import affine
from paper_2604_06575_b300 import workloads
from tests.golden_io import floats, parse_terms, read_kv
from tests.test_gpu_affine_exact import compare, oracle_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pl(cuda_ok):
    from paper_2604_06575_b300 import polylab
    return polylab


def run(pl, poly, X, **kw):
    dp = pl.to_device(poly)
    D, Du, info = pl.affine_normal(dp, torch.as_tensor(X, device="cuda"), method="ad", **kw)
    return D.cpu().numpy(), Du.cpu().numpy(), pl.info_numpy(info)


def test_worked_example_sec5(pl):
    g = read_kv("affine_worked_example.txt")
    exps, coef = parse_terms(g["terms"])
    poly = workloads.Poly(np.arange(4, dtype=np.uint64), exps, coef)
    x0 = floats(g["x0"])[None, :]
    D, Du, info = run(pl, poly, x0, regularization=float(g["regularization"]), assume_nonzero_x=True)
    d = floats(g["d"])
    # half a unit in the 7th printed digit, plus FP64 rounding of the vector
    assert np.all(np.abs(D[0] - d) <= 0.5e-6 * np.abs(d) + 2e-15 * np.linalg.norm(d))
    assert abs(info["grad_norm"][0] - float(g["grad_norm"])) <= 0.5e-6 * float(g["grad_norm"])
    assert info["hv_evals"][0] == int(g["hv_evals"]) and info["third_evals"][0] == int(g["third_evals"])
    np.testing.assert_allclose(np.linalg.norm(Du[0]), 1.0, rtol=1e-15)


def test_affine_small_all_points(pl):
    poly, X = workloads.affine_small(P=6000)  # more points than resident CTAs
    D, Du, info = run(pl, poly, X, regularization=1e-8)
    ref = oracle_all(poly, X[:600], 1e-8)
    assert compare(poly, X[:600], D[:600], info[:600], ref, 1e-8) == 0
    tail = np.arange(5400, 6000)
    ref = oracle_all(poly, X[tail], 1e-8)
    assert compare(poly, X[tail], D[tail], info[tail], ref, 1e-8) == 0


def test_flags_stress(pl):
    poly, X = workloads.affine_small_stress(P=256)
    D, Du, info = run(pl, poly, X, regularization=1e-8)
    ref = oracle_all(poly, X, 1e-8)
    flags = np.array([o["flags"] for _, o in ref])
    assert (flags == affine.FLAG_NOT_PD).sum() > 10
    assert compare(poly, X, D, info, ref, 1e-8) < 8
    zp = workloads.Poly(np.arange(2, dtype=np.uint64), np.array([[2, 0], [0, 2]], np.uint8), np.ones(2))
    D, Du, info = run(pl, zp, np.zeros((2, 2)))
    assert np.all(info["flags"] == affine.FLAG_ZERO_GRAD) and np.all(np.isnan(D)) and np.all(np.isnan(Du))


def test_accuracy_table_shape_and_agreement_with_exact(pl):
    """n = 6, 17 random quartic monomials plus the convexifying x_i^4 + x_i^2
    (the shape of the accuracy table's sparse quartic); the GPU
    'ad' and MF-logDet-Exact directions agree to rounding."""
    poly, X = workloads.sparse_quartic(6, 17, 3, P=512)
    D, Du, info = run(pl, poly, X, regularization=1e-6)
    ref = oracle_all(poly, X[:128], 1e-6)
    assert compare(poly, X[:128], D[:128], info[:128], ref, 1e-6) == 0
    dp = pl.to_device(poly)
    De, _, ie = pl.affine_normal(dp, torch.as_tensor(X, device="cuda"), regularization=1e-6)
    De = De.cpu().numpy()
    ok = info["flags"] == 0
    assert np.array_equal(info["flags"], pl.info_numpy(ie)["flags"])
    err = np.linalg.norm(D[ok] - De[ok], axis=1) / np.linalg.norm(De[ok], axis=1)
    assert err.max() <= 1e-9, err.max()


@pytest.mark.parametrize("n,m,deg,act", [(12, 300, 8, 8), (24, 400, 6, 6)])
def test_wide_terms_and_largest_n(pl, n, m, deg, act):
    rng = np.random.default_rng(100 + n)
    e = workloads.sparse_monomials(rng, n, m, deg, act)
    assert (e > 0).sum(axis=1).max() == act  # the widest support the plan takes occurs
    poly = workloads.convexified(rng, n, e, 0.1)
    X = workloads.shell_points(rng, n, 300)
    D, Du, info = run(pl, poly, X, regularization=1e-6)
    pick = np.r_[0:6, 294:300]
    ref = oracle_all(poly, X[pick], 1e-6)
    compare(poly, X[pick], D[pick], info[pick], ref, 1e-6)


def test_degenerate_n1_and_empty(pl):
    poly = workloads.Poly(np.array([3], np.uint64), np.array([[2], [1], [3]], np.uint8), np.array([1.0, 1.0, 0.1]))
    D, Du, info = run(pl, poly, np.array([[1.0], [-2.0]]))
    np.testing.assert_array_equal(D[:, 0], [-1.0, 1.0])
    assert np.all(info["logdet"] == 0.0)
    D, Du, info = run(pl, poly, np.zeros((0, 1)))
    assert D.shape == (0, 1)


def test_argument_errors(pl):
    rng = np.random.default_rng(5)
    n = pl.AD_MAX_N + 1
    poly = workloads.convexified(rng, n, workloads.sparse_monomials(rng, n, 50, 4, 4), 0.1)
    with pytest.raises(pl.PolylabError) as ei:
        run(pl, poly, workloads.shell_points(rng, n, 4))
    assert ei.value.status == 7  # UNSUPPORTED
    poly, X = workloads.affine_small(P=4)
    with pytest.raises(pl.PolylabError) as ei:
        run(pl, poly, X, prec="fp32")
    assert ei.value.status == 1  # INVALID_ARG
