"""Parity at the bench's full sizes and launch configurations, on sampled
outputs the oracle computes one by one, plus properties checked on every
output:

* the 256-polynomial uneven batch (290,592 points) through the batch API in
  the three forms, at the default and the autotuned configuration: every
  point's flags agree between the forms, the double-word form is within 1e-9
  relative of the FP64 form and the FP32-sum form within its stated 1e-3 rad;
  sampled points (the polynomials with the most terms, the largest n and the
  smallest n) match the oracle;
* the stochastic form on the large sparse family at n = 500 and n = 2000 with
  4,096 points and the bench's settings (FP32, q = 16, tol 1e-4, Jacobi):
  a sampled point matches the stochastic oracle run with the same probes."""
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


def angle(a, b):
    a = np.asarray(a) / np.linalg.norm(a)
    b = np.asarray(b) / np.linalg.norm(b)
    return float(np.arccos(np.clip(a @ b, -1.0, 1.0)))


@pytest.fixture(scope="module")
def bench_batch():
    return workloads.batched_uneven()


def test_bench_batch_full_size_sampled(pl, bench_batch):
    polys, Xs = bench_batch
    dps = [pl.to_device(p) for p in polys]
    plans = [pl.Plan(d) for d in dps]
    Xd = [torch.as_tensor(X, device="cuda") for X in Xs]
    out = {}
    for form in ("fp64", "f32x2", "fp32"):
        b = pl.Batch(dps, plans, Xd, pl.an_opts(prec=form, regularization=1e-6))
        b.run()
        b.check()
        if form != "fp64":
            first = [d.clone() for d in b.Du]
            b.autotune(reps=1)  # the bench's launch configuration
            b.run()
            b.check()
            for d0, d1 in zip(first, b.Du):  # configurations differ only in summation order
                ok = torch.isfinite(d0).all(dim=1)
                cos = (d0[ok] * d1[ok]).sum(dim=1).clamp(-1, 1)
                assert float(torch.arccos(cos).max()) <= 1e-4
        out[form] = ([d.cpu().numpy() for d in b.D], [pl.info_numpy(i)["flags"] for i in b.info])
        b.close()
    worst, worst_dw = 0.0, 0.0
    for i in range(len(polys)):
        f64, f32, fdw = out["fp64"][1][i], out["fp32"][1][i], out["f32x2"][1][i]
        assert np.array_equal(f64, f32) and np.array_equal(f64, fdw), i
        ok = f64 == 0
        a, c, w = out["fp64"][0][i][ok], out["fp32"][0][i][ok], out["f32x2"][0][i][ok]
        cos = np.sum(a * c, axis=1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(c, axis=1))
        worst = max(worst, float(np.arccos(np.clip(cos, -1, 1)).max()))
        if ok.any():
            worst_dw = max(worst_dw, float((np.linalg.norm(w - a, axis=1) / np.linalg.norm(a, axis=1)).max()))
    assert worst <= 1e-3, worst
    assert worst_dw <= 1e-9, worst_dw
    # sampled points against the oracle: most terms, largest n, smallest n
    sizes = [(p.m, p.n, i) for i, p in enumerate(polys)]
    picks = {max(sizes)[2], max(sizes, key=lambda s: s[1])[2], min(sizes, key=lambda s: s[1])[2]}
    for i in picks:
        for j in (0, Xs[i].shape[0] - 1):
            nu, _, oi = affine.affine_normal_ad(polys[i].exps, polys[i].coef, Xs[i][j], r=1e-6, third="contract")
            assert out["fp64"][1][i][j] == oi["flags"], (i, j)
            if oi["flags"]:
                continue
            d64, d32, ddw = out["fp64"][0][i][j], out["fp32"][0][i][j], out["f32x2"][0][i][j]
            assert np.linalg.norm(d64 - nu) <= 1e-9 * np.linalg.norm(nu), (i, j)
            assert np.linalg.norm(ddw - nu) <= 1e-9 * np.linalg.norm(nu), (i, j)
            assert angle(d32, nu) <= 1e-3, (i, j)


@pytest.mark.parametrize("n", [500, 2000])
def test_stochastic_full_size_sampled(pl, n):
    poly, X = workloads.large_sparse(n, P=4096)
    dp = pl.to_device(poly)
    Xd = torch.as_tensor(X, device="cuda")
    r = 1e-4
    with pl.Plan(dp) as plan:
        D, _, info = pl.affine_normal(dp, Xd, method="mf-stochastic", regularization=r, num_probes=16,
                                      krylov_tol=1e-4, krylov_maxit=80, prec="fp32", plan=plan, seed=7,
                                      precond="jacobi")
    D = D.cpu().numpy()
    flags = pl.info_numpy(info)["flags"]
    assert np.all(np.isfinite(D[flags == 0]))
    j = 4095 if n == 500 else 1234
    nu, _, oi = affine.affine_normal_stochastic(poly.exps, poly.coef, X[j], r=r, q=16, tol=1e-4, maxit=80, seed=7,
                                               point_index=j)
    assert (flags[j] & pl.FLAG_ZERO_GRAD) == (oi["flags"] & pl.FLAG_ZERO_GRAD)
    assert angle(D[j], nu) <= 2e-3, angle(D[j], nu)
