"""MF-logDet-Stochastic (C ABI) against the stochastic oracle with the same
probes (SplitMix64, ambient Rademacher projected to e-perp).

Bars: FP64 form with krylov_tol 1e-10 -- directions within 1e-7 relative of
the oracle's and the same Krylov iteration counts up to one per solve
(rounding can move a residual across the threshold); FP32 form with the
paper's default tol 1e-4 -- angle to the oracle's direction at most 2e-3 rad."""
import numpy as np
import pytest
import torch

from oracle import affine
from paper_2604_06575_b300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pl(cuda_ok):
    from paper_2604_06575_b300 import polylab
    return polylab


def quartic6():
    """Six variables, 17 monomials (the shape of the paper's accuracy case)."""
    rng = np.random.default_rng(606)
    e = workloads.sparse_monomials(rng, 6, 11, 4, 4, degree=4)
    poly = workloads.convexified(rng, 6, e, 0.3)  # 12 + 11 = 23 terms, 17 distinct monomials up to merging
    X = workloads.shell_points(rng, 6, 6)
    return poly, X


def run(pl, poly, X, **kw):
    dp = pl.to_device(poly)
    D, Du, info = pl.affine_normal(dp, torch.as_tensor(X, device="cuda"), method="mf-stochastic", **kw)
    return D.cpu().numpy(), pl.info_numpy(info)


@pytest.mark.parametrize("precond", ["jacobi", "none"])
def test_fp64_matches_stochastic_oracle(pl, precond):
    poly, X = quartic6()
    kw = dict(regularization=1e-6, num_probes=8, krylov_tol=1e-10, krylov_maxit=80, seed=99, precond=precond)
    D, info = run(pl, poly, X, prec="fp64", **kw)
    for j in range(X.shape[0]):
        nu, _, oi = affine.affine_normal_stochastic(poly.exps, poly.coef, X[j], r=1e-6, q=8, tol=1e-10, maxit=80,
                                                    seed=99, point_index=j, precond=precond)
        assert np.linalg.norm(D[j] - nu) <= 1e-7 * np.linalg.norm(nu), j
        assert abs(int(info["krylov_iters"][j]) - oi["krylov_iters"]) <= 9, (info["krylov_iters"][j], oi)
        assert info["third_evals"][j] == 8 and info["flags"][j] == oi["flags"]


def test_fp32_default_tolerance(pl):
    poly, X = quartic6()
    D, info = run(pl, poly, X, prec="fp32", regularization=1e-6, num_probes=16, krylov_tol=1e-4,
                  krylov_maxit=40, seed=5)
    for j in range(X.shape[0]):
        nu, _, _ = affine.affine_normal_stochastic(poly.exps, poly.coef, X[j], r=1e-6, q=16, tol=1e-4, maxit=40,
                                                   seed=5, point_index=j)
        assert np.radians(affine.angle_deg(D[j], nu)) <= 2e-3, j


def test_more_probes_approach_exact(pl):
    poly, X = quartic6()
    dp = pl.to_device(poly)
    Xd = torch.as_tensor(X, device="cuda")
    ex, _, _ = pl.affine_normal(dp, Xd, regularization=1e-6)
    errs = {}
    for q in (2, 512):  # FP32 CG can resolve a relative residual of 1e-5, not much less
        D, _, _ = pl.affine_normal(dp, Xd, method="mf-stochastic", regularization=1e-6, num_probes=q,
                                   krylov_tol=1e-5, krylov_maxit=80, prec="fp32", seed=17)
        c = (torch.nn.functional.normalize(D, dim=1) * torch.nn.functional.normalize(ex, dim=1)).sum(1)
        errs[q] = float(torch.arccos(c.clamp(-1, 1)).mean())
    assert errs[512] < 0.3 * errs[2], errs


def test_flags(pl):
    poly, X = quartic6()
    D, info = run(pl, poly, X[:2], prec="fp64", num_probes=4, krylov_tol=1e-14, krylov_maxit=1, seed=1)
    assert np.all(info["flags"] & pl.FLAG_KRYLOV_MAXIT)
    zp = workloads.Poly(np.arange(2, dtype=np.uint64), np.array([[2, 0], [0, 2]], np.uint8), np.ones(2))
    D, info = run(pl, zp, np.zeros((1, 2)), prec="fp32")
    assert info["flags"][0] == pl.FLAG_ZERO_GRAD and np.all(np.isnan(D))


def test_large_n_point(pl):
    """n=500 with 20n random terms (the large sparse family), 2 probes, 2 points."""
    poly, X = workloads.large_sparse(500, P=2)
    kw = dict(regularization=1e-6, num_probes=2, krylov_tol=1e-10, krylov_maxit=200, seed=3)
    D, info = run(pl, poly, X, prec="fp64", **kw)
    for j in range(2):
        nu, _, oi = affine.affine_normal_stochastic(poly.exps, poly.coef, X[j], r=1e-6, q=2, tol=1e-10, maxit=200,
                                                    seed=3, point_index=j)
        assert np.linalg.norm(D[j] - nu) <= 1e-6 * np.linalg.norm(nu), j
