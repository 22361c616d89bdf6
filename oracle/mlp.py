"""Oracle: the learned diagonal-plus-low-rank preconditioner (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper is silent on learned preconditioners; this network is the
project's own design, and this module is its plain definition:

* per-coordinate features of a point x (H = Hessian, g = gradient,
  e = g/|g|, r = regularisation, S_ij = sum over terms of |term's d_i d_j|,
  a_i = |H_ii| + r):
      f_i = [log(a_i), log(sum_{j != i} S_ij + r), x_i, n e_i^2,
             log(|g_i| + 1e-30), sum_{j != i} H_ij / a_i,
             sum_{j != i} H_ij / a_j]
  (the last two are signed: couplings of one sign that many coordinates
  share -- a collective mode of the Hessian -- show there, while couplings of
  random sign cancel);
* one MLP shared by all coordinates: h = tanh(W1^T f + b1) (32 units),
  o = W2^T h + b2 (3 outputs);
* preconditioner M = Pi (D + U U^T) Pi, Pi = I - e e^T, with
      D_i = exp(clip(o_0, -5, 5)) / (|H_ii| + r),
      U_ik = 0.1 o_k / sqrt(|H_ii| + r),  k = 1, 2,
  so zero output weights give exactly the Jacobi preconditioner;
* training loss for probes z in e-perp and y = Pi (H + r I) z:
      L = mean over (point, probe) of |Pi (D y + U U^T y) - z|^2 / |z|^2.

Parameters are one flat vector in the order W1 (F x Hd, row-major), b1,
W2 (Hd x 3, row-major), b2.
"""
from __future__ import annotations

import numpy as np

F = 7
HD = 32
NO = 3
RANK = NO - 1
N_PARAMS = F * HD + HD + HD * NO + NO


def unpack(theta: np.ndarray):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = theta[o:o + F * HD].reshape(F, HD)
    o += F * HD
    b1 = theta[o:o + HD]
    o += HD
    W2 = theta[o:o + HD * NO].reshape(HD, NO)
    o += HD * NO
    b2 = theta[o:o + NO]
    return W1, b1, W2, b2


def features(H: np.ndarray, SH: np.ndarray, g: np.ndarray, x: np.ndarray, r: float) -> np.ndarray:
    """SH: per-entry sums of |term contributions| to H (``derivs.eval_derivs``)."""
    n = x.shape[0]
    a = np.abs(np.diag(H)) + r
    off = SH.sum(axis=1) - np.diag(SH)
    e = g / np.linalg.norm(g)
    Hoff = H - np.diag(np.diag(H))
    return np.column_stack([np.log(a), np.log(off + r), x, n * e * e, np.log(np.abs(g) + 1e-30),
                            Hoff.sum(axis=1) / a, Hoff @ (1.0 / a)])


def forward(theta, f):
    W1, b1, W2, b2 = unpack(theta)
    a = f @ W1 + b1
    h = np.tanh(a)
    o = h @ W2 + b2
    return a, h, o


def precond_factors(theta, f, hdiag, r):
    _, _, o = forward(theta, f)
    s = np.abs(hdiag) + r
    D = np.exp(np.clip(o[:, 0], -5.0, 5.0)) / s
    U = 0.1 * o[:, 1:] / np.sqrt(s)[:, None]
    return D, U


def point_loss(theta, f, hdiag, r, e, Z, Y):
    """Loss summed over the probe columns of one point (divided by |z|^2 each)."""
    D, U = precond_factors(theta, f, hdiag, r)
    tot = 0.0
    for k in range(Z.shape[1]):
        z, y = Z[:, k], Y[:, k]
        w = D * y + U @ (U.T @ y)
        m = w - e * (e @ w)
        res = m - z
        tot += float(res @ res) / float(z @ z)
    return tot


def point_loss_grad(theta, f, hdiag, r, e, Z, Y):
    """(loss, dloss/dtheta) for one point, by hand-written backpropagation."""
    W1, b1, W2, b2 = unpack(theta)
    a, h, o = forward(theta, f)
    s = np.abs(hdiag) + r
    oc = np.clip(o[:, 0], -5.0, 5.0)
    D = np.exp(oc) / s
    U = 0.1 * o[:, 1:] / np.sqrt(s)[:, None]
    gD = np.zeros_like(D)
    gU = np.zeros_like(U)
    tot = 0.0
    for k in range(Z.shape[1]):
        z, y = Z[:, k], Y[:, k]
        uy = U.T @ y
        w = D * y + U @ uy
        m = w - e * (e @ w)
        res = m - z
        zz = float(z @ z)
        tot += float(res @ res) / zz
        gw = 2.0 * (res - e * (e @ res)) / zz     # d/dw of |Pi w - z|^2 / |z|^2
        gD += gw * y
        gU += np.outer(gw, uy) + np.outer(y, U.T @ gw)
    go = np.zeros_like(o)
    inside = (o[:, 0] > -5.0) & (o[:, 0] < 5.0)
    go[:, 0] = gD * D * inside
    go[:, 1:] = gU * 0.1 / np.sqrt(s)[:, None]
    gW2 = h.T @ go
    gb2 = go.sum(axis=0)
    gh = go @ W2.T
    ga = gh * (1.0 - h * h)
    gW1 = f.T @ ga
    gb1 = ga.sum(axis=0)
    return tot, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2])
