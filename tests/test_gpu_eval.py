"""Parity of the batched derivative evaluation (C ABI) against the oracle.

FP64 bar: every output within 1e-12 of the oracle's sum of |term
contributions| for that output (plus 1e-300 for outputs with no terms).
FP32 direct form: 2e-6 of that scale (24-bit products and sums over <= a few
thousand terms).
"""
import numpy as np
import pytest
import torch

from oracle import derivs
from paper_2604_06575_b300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pl(cuda_ok):
    from paper_2604_06575_b300 import polylab
    return polylab


def check(poly, X, F, G, H, idx, rel, order=2):
    Fo, Go, Ho, SF, SG, SH = derivs.eval_derivs(poly.exps, poly.coef, X[idx], order=order)
    F = F.cpu().numpy()[idx]
    assert np.all(np.abs(F - Fo) <= rel * SF + 1e-300), np.max(np.abs(F - Fo) / (SF + 1e-300))
    if order >= 1:
        G = G.cpu().numpy()[idx]
        assert np.all(np.abs(G - Go) <= rel * SG + 1e-300), np.max(np.abs(G - Go) / (SG + 1e-300))
    if order >= 2:
        H = H.cpu().numpy()[idx]
        assert np.all(np.abs(H - Ho) <= rel * SH + 1e-300), np.max(np.abs(H - Ho) / (SH + 1e-300))


@pytest.mark.parametrize("prec,rel", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_affine_small_all_points(pl, prec, rel):
    poly, X = workloads.affine_small(P=1024)
    dp = pl.to_device(poly)
    F, G, H = pl.eval_derivs(dp, torch.as_tensor(X, device="cuda"), prec=prec)
    check(poly, X, F, G, H, np.arange(1024), rel)


@pytest.mark.parametrize("order", [0, 1, 2])
def test_orders_and_ragged_tail(pl, order):
    poly, X = workloads.eval_batch(n=12, m=300, P=77)  # 77: several CTAs plus a ragged tail
    dp = pl.to_device(poly)
    F, G, H = pl.eval_derivs(dp, torch.as_tensor(X, device="cuda"), order=order)
    check(poly, X, F, G, H, np.arange(77), 1e-12, order)


def test_eval_batch_full_size_sampled(pl):
    """n=30, 5,000 terms, 65,536 points: the full-size batch, sampled outputs."""
    poly, X = workloads.eval_batch()
    dp = pl.to_device(poly)
    Xd = torch.as_tensor(X, device="cuda")
    with pl.Plan(dp) as plan:
        F, G, H = pl.eval_derivs(dp, Xd, plan=plan)
    idx = np.random.default_rng(0).choice(X.shape[0], 12, replace=False)
    idx = np.concatenate([idx, [0, X.shape[0] - 1]])
    check(poly, X, F, G, H, idx, 1e-12)
    # symmetry holds everywhere
    assert torch.equal(H, H.transpose(1, 2))


def test_large_n_global_accumulation(pl):
    """n=400: one point's accumulators do not fit in shared memory."""
    rng = np.random.default_rng(1)
    e = workloads.sparse_monomials(rng, 400, 600, 4, 4)
    poly = workloads.Poly(np.arange(400, dtype=np.uint64), e, rng.standard_normal(e.shape[0]))
    X = workloads.box_points(rng, 400, 5)
    dp = pl.to_device(poly)
    F, G, H = pl.eval_derivs(dp, torch.as_tensor(X, device="cuda"))
    check(poly, X, F, G, H, np.arange(5), 1e-12)


def test_edge_cases(pl):
    # empty point set
    poly, X = workloads.affine_small(P=4)
    dp = pl.to_device(poly)
    Xe = torch.zeros(0, 3, dtype=torch.float64, device="cuda")
    F, G, H = pl.eval_derivs(dp, Xe)
    assert F.shape == (0,)
    # polynomial with no terms: all zeros
    zero = workloads.Poly(np.arange(3, dtype=np.uint64), np.zeros((0, 3), np.uint8), np.zeros(0))
    F, G, H = pl.eval_derivs(pl.to_device(zero), torch.as_tensor(X, device="cuda"))
    assert float(F.abs().sum() + G.abs().sum() + H.abs().sum()) == 0.0
    # one variable, high exponents
    one = workloads.Poly(np.array([7], np.uint64), np.array([[0], [1], [9], [12]], np.uint8),
                         np.array([1.0, -2.0, 0.5, 0.25]))
    x1 = np.array([[0.7], [-1.1], [0.0]])
    F, G, H = pl.eval_derivs(pl.to_device(one), torch.as_tensor(x1, device="cuda"))
    check(one, x1, F, G, H, np.arange(3), 1e-12)
    # a term with more than 8 active variables is outside the term-list limit
    wide = workloads.Poly(np.arange(9, dtype=np.uint64), np.ones((1, 9), np.uint8), np.ones(1))
    with pytest.raises(pl.PolylabError) as ei:
        pl.eval_derivs(pl.to_device(wide), torch.zeros(1, 9, dtype=torch.float64, device="cuda"))
    assert ei.value.status == 7
    # duplicate variable ids
    dup = workloads.Poly(np.array([1, 1], np.uint64), np.ones((1, 2), np.uint8), np.ones(1))
    with pytest.raises(pl.PolylabError) as ei:
        pl.eval_derivs(pl.to_device(dup), torch.zeros(1, 2, dtype=torch.float64, device="cuda"))
    assert ei.value.status == 3
