"""Learned preconditioner: the data kernel and the hand-written backward pass
against the FP64 oracle, and a trained network used inside the stochastic
solver (gain over the method without it; the exact variant is the reference for the error).

Bars: features, diagonal, e and y within 1e-4 relative (FP32); loss within
1e-4 and gradient within 2e-3 (relative, norm-wise) of the oracle's on the same
FP32 data."""
import numpy as np
import pytest
import torch

from oracle import derivs, mlp
from oracle.rng import rademacher
from paper_2604_06575_b300 import workloads

pytestmark = pytest.mark.gpu
R = 1e-4


@pytest.fixture(scope="module")
def pl(cuda_ok):
    from paper_2604_06575_b300 import polylab
    return polylab


def oracle_point(poly, x, p, seed):
    n = x.shape[0]
    F, G, H, SF, SG, SH = derivs.eval_derivs(poly.exps, poly.coef, x[None, :])
    g, H, SH = G[0], H[0], SH[0]
    e = g / np.linalg.norm(g)
    Pi = np.eye(n) - np.outer(e, e)
    Z = np.column_stack([Pi @ rademacher(seed, p, k, 4, n) for k in range(4)])
    Y = Pi @ (H + R * np.eye(n)) @ Z
    return mlp.features(H, SH, g, x, R), np.diag(H), e, Z, Y


def test_data_kernel_matches_oracle(pl):
    poly, X = workloads.large_sparse(60, P=5, shell=True)
    f, hd, e, Z, Y = (t.cpu().numpy() for t in pl.mlp_data(pl.to_device(poly), torch.as_tensor(X, device="cuda"),
                                                             R, seed=11))
    for p in range(5):
        of, ohd, oe, oZ, oY = oracle_point(poly, X[p], p, 11)
        np.testing.assert_allclose(f[p], of, rtol=1e-4, atol=1e-4)
        np.testing.assert_allclose(hd[p], ohd, rtol=1e-4, atol=1e-5)
        np.testing.assert_allclose(e[p], oe, rtol=1e-4, atol=1e-6)
        np.testing.assert_allclose(Z[p], oZ, rtol=1e-5, atol=1e-5)
        np.testing.assert_allclose(Y[p], oY, rtol=1e-4, atol=1e-4 * np.abs(oY).max())


def test_gradient_matches_oracle(pl):
    poly, X = workloads.large_sparse(40, P=6, shell=True)
    data = [oracle_point(poly, X[p], p, 3) for p in range(6)]
    theta = np.random.default_rng(0).normal(0.0, 0.3, mlp.N_PARAMS).astype(np.float32)
    L, G = 0.0, np.zeros(mlp.N_PARAMS)
    for f, hd, e, Z, Y in data:
        f32 = [a.astype(np.float32).astype(np.float64) for a in (f, hd, e, Z, Y)]
        l, gr = mlp.point_loss_grad(theta.astype(np.float64), *f32[:2], R, *f32[2:])
        L += l
        G += gr
    L /= 6 * 4
    G /= 6 * 4
    dev = lambda a: torch.as_tensor(np.stack(a).astype(np.float32), device="cuda")
    gdata = tuple(dev([d[i] for d in data]) for i in range(5))
    loss, grad = pl.mlp_loss_grad(torch.as_tensor(theta, device="cuda"), gdata, R)
    assert abs(float(loss) - L) <= 1e-4 * abs(L)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - G) <= 2e-3 * np.linalg.norm(G), np.linalg.norm(g - G) / np.linalg.norm(G)


def test_trained_network_gain(pl):
    """Train on 48 points of the n=500 large sparse family, then solve at 16
    held-out points with Jacobi, no preconditioner and the network."""
    poly, X = workloads.large_sparse(500, P=64)
    dp = pl.to_device(poly)
    Xd = torch.as_tensor(X, device="cuda")
    with pl.Plan(dp) as plan:
        data = pl.mlp_data(dp, Xd[:48], R, seed=21, plan=plan)
        params, packed, hist = pl.train_preconditioner(data, R, steps=150, lr=3e-3)
        assert hist[-1] < hist[0]  # training reduces the loss from the Jacobi starting point
        test = Xd[48:]
        ex, _, _ = pl.affine_normal(dp, test, plan=plan, regularization=R)
        res = {}
        for pre in ("none", "jacobi", "mlp"):
            D, Du, info = pl.affine_normal(dp, test, plan=plan, method="mf-stochastic", regularization=R,
                                           num_probes=8, krylov_tol=1e-4, krylov_maxit=80, prec="fp32",
                                           precond=pre, mlp_weights=packed if pre == "mlp" else None, seed=5)
            it = pl.info_numpy(info)["krylov_iters"].mean()
            c = (torch.nn.functional.normalize(D, dim=1) * torch.nn.functional.normalize(ex, dim=1)).sum(1)
            res[pre] = (it, float(torch.arccos(c.clamp(-1, 1)).mean()))
    print("iterations / angle to exact:", res, "loss", hist[0], hist[-1])
    assert res["mlp"][0] < res["none"][0]
    # same probes and tolerance: the preconditioner must not change the answer beyond CG tolerance effects
    assert res["mlp"][1] <= 1.5 * res["jacobi"][1] + 1e-3
