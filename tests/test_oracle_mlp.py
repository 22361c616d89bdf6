"""Pins for the preconditioner-network oracle: hand-written backpropagation
against central finite differences of the loss, the zero-weight network is
exactly Jacobi, and a perfect preconditioner has zero loss."""
import numpy as np

from oracle import affine, derivs, mlp
from oracle.rng import rademacher
from paper_2604_06575_b300 import workloads


def point_data(seed=0, n=7, nz=3, r=1e-3):
    rng = np.random.default_rng(seed)
    poly = workloads.convexified(rng, n, workloads.sparse_monomials(rng, n, 20, 4, 3), 0.3)
    x = workloads.shell_points(rng, n, 1)[0]
    F, G, H, SF, SG, SH = derivs.eval_derivs(poly.exps, poly.coef, x[None, :])
    g, H, SH = G[0], H[0], SH[0]
    e = g / np.linalg.norm(g)
    Pi = np.eye(n) - np.outer(e, e)
    Z = np.column_stack([Pi @ rademacher(seed, 0, s, nz, n) for s in range(nz)])
    Y = Pi @ (H + r * np.eye(n)) @ Z
    return mlp.features(H, SH, g, x, r), np.diag(H), r, e, Z, Y, H


def test_gradient_matches_finite_differences():
    f, hd, r, e, Z, Y, _ = point_data()
    theta = np.random.default_rng(1).normal(0.0, 0.3, mlp.N_PARAMS)
    L, grad = mlp.point_loss_grad(theta, f, hd, r, e, Z, Y)
    assert abs(L - mlp.point_loss(theta, f, hd, r, e, Z, Y)) <= 1e-12 * abs(L)
    h = 1e-6
    for i in np.random.default_rng(2).choice(mlp.N_PARAMS, 40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.point_loss(tp, f, hd, r, e, Z, Y) - mlp.point_loss(tm, f, hd, r, e, Z, Y)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_zero_output_weights_are_jacobi():
    f, hd, r, e, Z, Y, H = point_data(seed=3)
    theta = np.random.default_rng(4).normal(0.0, 0.5, mlp.N_PARAMS)
    W1, b1, W2, b2 = mlp.unpack(theta)
    theta[mlp.F * mlp.HD + mlp.HD:] = 0.0  # W2 = 0, b2 = 0
    D, U = mlp.precond_factors(theta, f, hd, r)
    np.testing.assert_allclose(D, 1.0 / (np.abs(hd) + r), rtol=1e-15)
    assert np.all(U == 0.0)


def test_exact_inverse_has_zero_loss():
    f, hd, r, e, Z, Y, H = point_data(seed=6)
    n = H.shape[0]
    Pi = np.eye(n) - np.outer(e, e)
    A = Pi @ (H + r * np.eye(n)) @ Pi
    Ainv = np.linalg.pinv(A)
    for k in range(Z.shape[1]):
        np.testing.assert_allclose(Pi @ (Ainv @ Y[:, k]), Z[:, k], atol=1e-10)


def test_lowrank_preconditioned_pcg_matches_stochastic_oracle_option():
    """The 'lowrank' preconditioner of the stochastic oracle is M = Pi (D + UU^T) Pi."""
    f, hd, r, e, Z, Y, H = point_data(seed=7)
    theta = np.random.default_rng(8).normal(0.0, 0.2, mlp.N_PARAMS)
    D, U = mlp.precond_factors(theta, f, hd, r)
    n = H.shape[0]
    QT = affine.qr_frame(e)
    M = QT.T @ (np.diag(D) + U @ U.T) @ QT
    v = np.random.default_rng(9).normal(size=n - 1)
    np.testing.assert_allclose(QT @ (M @ v), (np.eye(n) - np.outer(e, e)) @ ((D * (QT @ v)) + U @ (U.T @ (QT @ v))),
                               atol=1e-12)


def test_signed_coupling_features_closed_form():
    """f = sum_i d_i x_i^2 / 2 - (c/2) (sum_i x_i)^2 has H = diag(d) - c 1 1^T at
    every x, so the two signed coupling features are known in closed form:
    sum_{j != i} H_ij / a_i = -(n - 1) c / a_i and sum_{j != i} H_ij / a_j =
    -c sum_{j != i} 1 / a_j, with a_i = |d_i - c| + r."""
    n, c, r = 5, 0.5, 1e-3
    d = np.array([3.0, 4.0, 5.0, 6.0, 7.0])
    rows, coef = [], []
    for i in range(n):
        e = np.zeros(n, np.uint8)
        e[i] = 2
        rows.append(e)
        coef.append((d[i] - c) / 2)
        for j in range(i + 1, n):
            e = np.zeros(n, np.uint8)
            e[i] = e[j] = 1
            rows.append(e)
            coef.append(-c)
    x = np.array([0.3, -0.2, 0.5, 0.1, -0.4])
    F, G, H, SF, SG, SH = derivs.eval_derivs(np.array(rows), np.array(coef), x[None, :])
    np.testing.assert_allclose(H[0], np.diag(d) - c, rtol=1e-14)
    f = mlp.features(H[0], SH[0], G[0], x, r)
    a = np.abs(d - c) + r
    np.testing.assert_allclose(f[:, 5], -(n - 1) * c / a, rtol=1e-14)
    np.testing.assert_allclose(f[:, 6], [-c * (np.sum(1 / a) - 1 / a[i]) for i in range(n)], rtol=1e-14)
