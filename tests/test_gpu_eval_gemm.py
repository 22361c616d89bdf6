"""Tensor-core forms of the derivative evaluation (monomial x derived-
coefficient contraction on tcgen05) against the oracle.

Stated bounds, relative to the oracle's sum of |term contributions| of each
output: BF16 operands with per-column scaling, FP32 accumulation: 1.5e-2
(8-bit significands on both operands); 3xTF32 with FP32 accumulation: 2e-5
(about 21 significand bits per operand pair, FP32 sums over the closure)."""
import numpy as np
import pytest
import torch

from oracle import derivs
from paper_2604_06575_b300 import workloads

pytestmark = pytest.mark.gpu
BOUND = {"bf16": 1.5e-2, "tf32x3": 2e-5}


@pytest.fixture(scope="module")
def pl(cuda_ok):
    from paper_2604_06575_b300 import polylab
    return polylab


def closure_count(exps):
    """|{alpha, alpha - e_i, alpha - e_i - e_j}| by brute force over the terms."""
    seen = set()
    for row in exps:
        a = [int(v) for v in row]
        seen.add(tuple(a))
        for i in range(len(a)):
            if a[i] >= 1:
                a[i] -= 1
                seen.add(tuple(a))
                for j in range(i, len(a)):
                    if a[j] >= 1:
                        a[j] -= 1
                        seen.add(tuple(a))
                        a[j] += 1
                a[i] += 1
    return len(seen)


def check(poly, X, out, idx, rel, order=2):
    F, G, H = out
    Fo, Go, Ho, SF, SG, SH = derivs.eval_derivs(poly.exps, poly.coef, X[idx], order=order)
    F = F.cpu().numpy()[idx]
    assert np.all(np.abs(F - Fo) <= rel * SF + 1e-300), np.max(np.abs(F - Fo) / (SF + 1e-300))
    if order >= 1:
        G = G.cpu().numpy()[idx]
        assert np.all(np.abs(G - Go) <= rel * SG + 1e-300), np.max(np.abs(G - Go) / (SG + 1e-300))
    if order >= 2:
        H = H.cpu().numpy()[idx]
        assert np.all(np.abs(H - Ho) <= rel * SH + 1e-300), np.max(np.abs(H - Ho) / (SH + 1e-300))


@pytest.mark.parametrize("prec", ["bf16", "tf32x3"])
def test_small_ragged(pl, prec):
    poly, X = workloads.eval_batch(n=12, m=300, P=300)  # 3 point tiles, ragged tail
    dp = pl.to_device(poly)
    with pl.Plan(dp, gemm=True) as plan:
        assert plan.closure_size == closure_count(poly.exps)
        out = pl.eval_derivs(dp, torch.as_tensor(X, device="cuda"), plan=plan, prec=prec)
        pl.eval_check()  # synchronises; no bounded wait expired
    check(poly, X, out, np.arange(300), BOUND[prec])


@pytest.mark.parametrize("prec", ["bf16", "tf32x3"])
def test_eval_batch_full_size_sampled(pl, prec):
    poly, X = workloads.eval_batch()
    dp = pl.to_device(poly)
    with pl.Plan(dp, gemm=True) as plan:
        out = pl.eval_derivs(dp, torch.as_tensor(X, device="cuda"), plan=plan, prec=prec)
        pl.eval_check()
    idx = np.concatenate([np.random.default_rng(1).choice(X.shape[0], 254, replace=False), [0, X.shape[0] - 1]])
    check(poly, X, out, idx, BOUND[prec])
    assert torch.equal(out[2], out[2].transpose(1, 2))


@pytest.mark.parametrize("order", [0, 1])
def test_orders_and_tiny(pl, order):
    poly, X = workloads.affine_small(P=5)  # fewer points than one tile; repeated monomials
    dp = pl.to_device(poly)
    out = pl.eval_derivs(dp, torch.as_tensor(X, device="cuda"), prec="tf32x3", order=order)
    pl.eval_check()
    check(poly, X, out, np.arange(5), BOUND["tf32x3"], order)


def test_large_n_several_chunks(pl):
    """n=40: 861 output columns, two BF16 column chunks / four TF32 chunks."""
    rng = np.random.default_rng(4)
    e = workloads.sparse_monomials(rng, 40, 400, 4, 4)
    poly = workloads.Poly(np.arange(40, dtype=np.uint64), e, rng.standard_normal(e.shape[0]))
    X = workloads.box_points(rng, 40, 130)
    dp = pl.to_device(poly)
    with pl.Plan(dp, gemm=True) as plan:
        for prec in ("bf16", "tf32x3"):
            out = pl.eval_derivs(dp, torch.as_tensor(X, device="cuda"), plan=plan, prec=prec)
            pl.eval_check()
            check(poly, X, out, np.arange(0, 130, 13), BOUND[prec])
