"""Parity of the exact affine-normal direction (C ABI) against the 'ad' oracle.

FP64 bar: |nu_gpu - nu_oracle| <= 1e-11 * kappa * |nu_oracle| with kappa the
2-norm condition number of H_T + r I (errors of ~1e-16 relative in g and H
are amplified by the tangent solves).  Flags must match except where the
oracle's eigenvalue of H_T + r I closest to zero is within 1e-10 |H_T|_F of it
(ambiguous points, counted and excluded).  The double-word form (POLYLAB_F32X2:
FP32-pair term sums, inverse and W; FP64 Cholesky) is held to the same FP64
bar.  FP32 form: the angle between the directions stays below the
kappa-scaled bound stated in the test.
"""
import numpy as np
import pytest
import torch

from oracle import affine, derivs
from paper_2604_06575_b300 import workloads
from tests.golden_io import floats, parse_terms, read_kv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pl(cuda_ok):
    from paper_2604_06575_b300 import polylab
    return polylab


def oracle_all(poly, X, r, **kw):
    out = []
    for x in X:
        nu, unit, info = affine.affine_normal_ad(poly.exps, poly.coef, x, r=r, **kw)
        out.append((nu, info))
    return out


def kappa_and_ambiguity(poly, x, r):
    F, G, H, *_ = derivs.eval_derivs(poly.exps, poly.coef, x[None, :])
    g, Hm = G[0], H[0]
    gn = np.linalg.norm(g)
    if gn == 0:
        return np.inf, False
    QT = affine.qr_frame(g / gn)
    HT = QT.T @ Hm @ QT + r * np.eye(len(x) - 1)
    ev = np.linalg.eigvalsh(HT) if len(x) > 1 else np.array([1.0])
    amb = np.abs(ev).min() <= 1e-10 * np.linalg.norm(HT)
    return (abs(ev).max() / max(abs(ev).min(), 1e-300)), amb


def run(pl, poly, X, **kw):
    dp = pl.to_device(poly)
    D, Du, info = pl.affine_normal(dp, torch.as_tensor(X, device="cuda"), **kw)
    return D.cpu().numpy(), Du.cpu().numpy(), pl.info_numpy(info)


def compare(poly, X, D, info, ref, r, rel=1e-11):
    ambiguous = 0
    for i, (nu, oi) in enumerate(ref):
        kap, amb = kappa_and_ambiguity(poly, X[i], r)
        if amb:
            ambiguous += 1
            continue
        assert info["flags"][i] == oi["flags"], (i, info["flags"][i], oi["flags"])
        if oi["flags"]:
            assert np.all(np.isnan(D[i]))
            continue
        err = np.linalg.norm(D[i] - nu) / np.linalg.norm(nu)
        assert err <= rel * max(kap, 1.0), (i, err, kap)
        assert info["grad_norm"][i] == pytest.approx(oi["grad_norm"], rel=1e-13)
        assert info["logdet"][i] == pytest.approx(oi["logdet"], rel=1e-9, abs=1e-9)
        assert info["hv_evals"][i] == oi["hv_evals"] and info["third_evals"][i] == oi["third_evals"]
    return ambiguous


@pytest.mark.parametrize("prec", ["fp64", "f32x2"])
def test_worked_example_sec5(pl, prec):
    g = read_kv("affine_worked_example.txt")
    exps, coef = parse_terms(g["terms"])
    poly = workloads.Poly(np.arange(4, dtype=np.uint64), exps, coef)
    x0 = floats(g["x0"])[None, :]
    D, Du, info = run(pl, poly, x0, regularization=float(g["regularization"]), assume_nonzero_x=True, prec=prec)
    d = floats(g["d"])
    # half a unit in the 7th printed digit; the third entry (~1e-9) sits at the
    # FP64 rounding level of the whole vector (|d| ~ 4.5, ulp ~ 1e-15), so it
    # also gets 2e-15 |d| of absolute slack
    assert np.all(np.abs(D[0] - d) <= 0.5e-6 * np.abs(d) + 2e-15 * np.linalg.norm(d))
    assert abs(info["grad_norm"][0] - float(g["grad_norm"])) <= 0.5e-6 * float(g["grad_norm"])
    assert info["hv_evals"][0] == int(g["hv_evals"]) and info["third_evals"][0] == int(g["third_evals"])
    np.testing.assert_allclose(np.linalg.norm(Du[0]), 1.0, rtol=1e-15)


@pytest.mark.parametrize("r,prec", [(1e-8, "fp64"), (1e-6, "fp64"), (1e-8, "f32x2"), (1e-6, "f32x2")])
def test_affine_small_all_points(pl, r, prec):
    poly, X = workloads.affine_small(P=1024)
    D, Du, info = run(pl, poly, X, regularization=r, prec=prec)
    ref = oracle_all(poly, X, r)
    amb = compare(poly, X, D, info, ref, r)
    assert amb == 0


@pytest.mark.parametrize("prec", ["fp64", "f32x2"])
def test_flags_stress(pl, prec):
    poly, X = workloads.affine_small_stress(P=256)
    X[0] = 0.0  # the gradient of this polynomial at the origin is (0, 0, 1): not zero
    D, Du, info = run(pl, poly, X, regularization=1e-8, prec=prec)
    ref = oracle_all(poly, X, 1e-8)
    flags = np.array([o["flags"] for _, o in ref])
    assert (flags == affine.FLAG_NOT_PD).sum() > 10  # the stress case really flags points
    amb = compare(poly, X, D, info, ref, 1e-8)
    assert amb < 8
    # exact zero gradient: x1^2 + x2^2 at the origin
    zp = workloads.Poly(np.arange(2, dtype=np.uint64), np.array([[2, 0], [0, 2]], np.uint8), np.ones(2))
    D, Du, info = run(pl, zp, np.zeros((2, 2)), prec=prec)
    assert np.all(info["flags"] == affine.FLAG_ZERO_GRAD) and np.all(np.isnan(D))


@pytest.mark.parametrize("prec", ["fp64", "f32x2"])
def test_medium_and_large_n(pl, prec):
    for n, m, P in [(20, 200, 9), (45, 600, 5), (70, 400, 3), (130, 300, 2)]:
        rng = np.random.default_rng(n)
        poly = workloads.convexified(rng, n, workloads.sparse_monomials(rng, n, m, 6, 6), 0.1)
        X = workloads.shell_points(rng, n, P)
        D, Du, info = run(pl, poly, X, regularization=1e-6, prec=prec)
        ref = oracle_all(poly, X, 1e-6, third="contract")
        compare(poly, X, D, info, ref, 1e-6)


def test_degenerate_n1_and_empty(pl):
    poly = workloads.Poly(np.array([3], np.uint64), np.array([[2], [1]], np.uint8), np.ones(2))
    D, Du, info = run(pl, poly, np.array([[1.0], [-2.0]]))
    np.testing.assert_array_equal(D[:, 0], [-1.0, 1.0])
    D, Du, info = run(pl, poly, np.zeros((0, 1)))
    assert D.shape == (0, 1)


def test_fp32_form_error_bound(pl):
    """Mixed form: FP32 term sums, FP64 Cholesky/tau/normalisation.  Stated
    bound: angle <= 2e-5 rad * max(kappa, 1) on the n=3 family."""
    poly, X = workloads.affine_small(P=512)
    D, Du, info = run(pl, poly, X, regularization=1e-6, prec="fp32")
    ref = oracle_all(poly, X, 1e-6)
    worst = 0.0
    for i, (nu, oi) in enumerate(ref):
        kap, amb = kappa_and_ambiguity(poly, X[i], 1e-6)
        assert info["flags"][i] == oi["flags"]
        ang = np.radians(affine.angle_deg(D[i], nu))
        worst = max(worst, ang / max(kap, 1.0))
        assert ang <= 2e-5 * max(kap, 1.0), (i, ang, kap)


@pytest.mark.parametrize("prec", ["fp64", "f32x2", "fp32"])
def test_gather_and_term_by_term_sweeps_agree(pl, prec):
    """Points with a zero or tiny coordinate take the term-by-term sweeps (no
    division by x); the others take the gather forms of both term sweeps.
    Both kinds, in one call, against the oracle."""
    rng = np.random.default_rng(77)
    n = 20
    poly = workloads.convexified(rng, n, workloads.sparse_monomials(rng, n, 600, 6, 5), 0.1)
    X = workloads.shell_points(rng, n, 24)
    X[0:6, 3] = 0.0
    X[6:12, 7] = 1e-7
    D, Du, info = run(pl, poly, X, regularization=1e-6, prec=prec)
    ref = oracle_all(poly, X, 1e-6, third="contract")
    if prec != "fp32":
        assert compare(poly, X, D, info, ref, 1e-6) == 0
    else:
        for i, (nu, oi) in enumerate(ref):
            kap, amb = kappa_and_ambiguity(poly, X[i], 1e-6)
            assert info["flags"][i] == oi["flags"]
            if oi["flags"] == 0:
                assert np.radians(affine.angle_deg(D[i], nu)) <= 2e-5 * max(kap, 1.0), i


@pytest.mark.parametrize("prec", ["fp64", "f32x2"])
def test_gather_and_term_by_term_sweeps_agree_large_n(pl, prec):
    """The same at n = 50 (the class of n > 40, whose gather launch takes one
    point per pass in double words): the passes with a zero or tiny coordinate
    go through the list to the term-by-term launch; all points against the
    oracle."""
    rng = np.random.default_rng(78)
    n = 50
    poly = workloads.convexified(rng, n, workloads.sparse_monomials(rng, n, 400, 6, 5), 0.1)
    X = workloads.shell_points(rng, n, 20)
    X[0:4, 3] = 0.0
    X[7:11, 41] = 1e-7
    D, Du, info = run(pl, poly, X, regularization=1e-6, prec=prec)
    ref = oracle_all(poly, X, 1e-6, third="contract")
    assert compare(poly, X, D, info, ref, 1e-6) == 0


@pytest.mark.parametrize("n,prec", [(131, "fp64"), (132, "fp64"), (131, "f32x2"), (132, "f32x2"), (171, "fp32")])
def test_global_memory_frame_both_parities(pl, n, prec):
    """Matrices too large for shared memory take the frame stage's global-memory
    path (the LDL^T in panels of two columns): even and odd m = n - 1, both forms."""
    rng = np.random.default_rng(n)
    poly = workloads.convexified(rng, n, workloads.sparse_monomials(rng, n, 300, 4, 4), 0.1)
    X = workloads.shell_points(rng, n, 3)
    D, Du, info = run(pl, poly, X, regularization=1e-6, prec=prec)
    ref = oracle_all(poly, X, 1e-6, third="contract")
    if prec != "fp32":
        compare(poly, X, D, info, ref, 1e-6)
    else:
        for i, (nu, oi) in enumerate(ref):
            kap, amb = kappa_and_ambiguity(poly, X[i], 1e-6)
            assert info["flags"][i] == oi["flags"]
            if oi["flags"] == 0:
                assert np.radians(affine.angle_deg(D[i], nu)) <= 2e-5 * max(kap, 1.0), i
