"""Single-precision storage (the ``*_f32`` calls; the paper's precision
control of Sec. 3.5 and its single/double table of Sec. 6) against the FP64
oracle run on the same FP32-rounded inputs.

Bars.  Engine: exponent rows bit-exact and in canonical order; a merged
coefficient of k contributions (each an FP32 product for mul, one rounding)
summed in FP32 in any order is within 1.01 (k + 1) 2^-24 S of the exact sum,
S the oracle's sum of |contributions|, k the oracle's count of contributions
(the same oracle call on all-one coefficients); terms within that bound of
zero may be present on one side only.  Integer-coefficient powers below
2^24 are bit-exact.  A derivative coefficient a_v c is one FP32 product:
within 2^-24 of it.  Evaluation and directions: the FP32-storage calls run
the FP32 arithmetic of the POLYLAB_FP32 form of the FP64 calls on the
widened inputs, and are held to that form's bars: f, g, H within 2e-6 of the
oracle's sums of |term contributions| (and within twice that of the FP32
form: both accumulate with shared-memory atomics, so equal arithmetic does
not mean equal bits); exact directions within 2e-5 rad * max(kappa, 1) of
the oracle with equal flags; stochastic directions within 2e-3 rad of the
stochastic oracle run with the same probes.
"""
import numpy as np
import pytest
import torch

from oracle import affine, derivs, engine
from paper_2604_06575_b300 import workloads
from tests.test_gpu_affine_exact import kappa_and_ambiguity
from tests.test_gpu_affine_stochastic import quartic6

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def pl(cuda_ok):
    from paper_2604_06575_b300 import polylab
    return polylab


def rounded(p):
    """The polynomial with coefficients rounded to FP32 (held as float64)."""
    return workloads.Poly(p.var_ids, p.exps, p.coef.astype(np.float32).astype(np.float64))


def ones(p):
    return (p.var_ids, p.exps, np.ones(p.m))


def t(p):
    return (p.var_ids, p.exps, p.coef)


def host(dp):
    return np.asarray(dp.var_ids), dp.exps.cpu().numpy(), dp.coef.cpu().numpy().astype(np.float64)


def compare_f32(got, ref, counts, extra_rounding=1):
    gid, ge, gc = got
    rid, re_, rc, rs = ref
    _, ce, cc, _ = counts
    assert [int(v) for v in gid] == [int(v) for v in rid]
    kmap = {r.tobytes(): k for r, k in zip(ce, cc)}
    g_map = {r.tobytes(): c for r, c in zip(ge, gc)}
    for r, c, s in zip(re_, rc, rs):
        key = r.tobytes()
        bound = 1.01 * (kmap[key] + extra_rounding) * U32 * s
        if key in g_map:
            assert abs(g_map[key] - c) <= bound, (g_map[key], c, bound)
        else:
            assert abs(c) <= bound, "missing term"
    r_set = {r.tobytes() for r in re_}
    for key, c in g_map.items():
        if key not in r_set:  # exact zero in FP64, rounding residue in FP32
            assert abs(c) <= 1.01 * (kmap.get(key, 0) + extra_rounding) * U32 * max(rs.max(initial=0.0), 1.0)
    assert np.array_equal(ge, ge[engine.canonical_order(ge)])


def rand_poly(rng, n, m, deg, act, ids=None, dup=0):
    e = workloads.sparse_monomials(rng, n, m, deg, act)
    if dup:
        e = np.concatenate([e, e[rng.integers(0, e.shape[0], dup)]])
    ids = np.arange(n, dtype=np.uint64) if ids is None else np.asarray(ids, np.uint64)
    return workloads.Poly(ids, e, rng.standard_normal(e.shape[0]))


@pytest.mark.parametrize("seed", range(3))
def test_simplify_with_duplicates(pl, seed):
    rng = np.random.default_rng(seed)
    p = rounded(rand_poly(rng, 12, 3000, 5, 4, dup=4000))
    got = pl.simplify(pl.to_device(p, dtype=torch.float32))
    assert got.coef.dtype == torch.float32
    compare_f32(host(got), engine.simplify(*t(p)), engine.simplify(*ones(p)), extra_rounding=0)
    g64 = pl.simplify(pl.to_device(p))  # same merged rows, same order
    assert np.array_equal(got.exps.cpu().numpy(), g64.exps.cpu().numpy())


def test_mul_mixed_ids_several_tiles(pl):
    A, B = workloads.product_pair(n=10, m=300, overlap=4, max_deg=4)
    A, B = rounded(A), rounded(B)
    got = pl.mul(pl.to_device(A, dtype=torch.float32), pl.to_device(B, dtype=torch.float32))
    compare_f32(host(got), engine.mul(t(A), t(B)), engine.mul(ones(A), ones(B)), extra_rounding=1)


def test_add_sub(pl):
    rng = np.random.default_rng(9)
    a = rounded(rand_poly(rng, 6, 50, 4, 3, ids=[1, 3, 5, 7, 9, 11]))
    b = rounded(rand_poly(rng, 5, 40, 4, 3, ids=[2, 3, 4, 9, 20]))
    da, db = pl.to_device(a, dtype=torch.float32), pl.to_device(b, dtype=torch.float32)
    compare_f32(host(pl.add(da, db)), engine.add(t(a), t(b)), engine.add(ones(a), ones(b)), extra_rounding=0)
    compare_f32(host(pl.sub(da, db)), engine.sub(t(a), t(b)), engine.add(ones(a), ones(b)), extra_rounding=0)
    assert pl.sub(da, da).m == 0  # c - c is exactly zero in FP32 too
    with pytest.raises(ValueError):
        pl.mul(da, pl.to_device(b))


@pytest.mark.parametrize("d,k", [(2, 3), (3, 3), (4, 3)])
def test_pow_dense_base_exact(pl, d, k):
    p = workloads.dense_power_base(d)
    got = pl.pow(pl.to_device(p, dtype=torch.float32), k)
    _, re_, rc, _ = engine.power(t(p), k)
    assert rc.max() < 2 ** 24
    _, ge, gc = host(got)
    assert np.array_equal(ge, re_) and np.array_equal(gc, rc)


def test_diff_and_jacobian(pl):
    rng = np.random.default_rng(3)
    p = rounded(rand_poly(rng, 7, 400, 6, 4))
    dp = pl.to_device(p, dtype=torch.float32)
    for v, d in zip(p.var_ids, pl.jacobian(dp)):
        _, re_, rc, rs = engine.diff(t(p), int(v))
        _, ge, gc = host(d)
        assert np.array_equal(ge, re_)
        assert np.all(np.abs(gc - rc) <= U32 * np.abs(rc))


def test_eval_matches_fp32_form_and_oracle(pl):
    poly, X = workloads.eval_batch(n=12, m=300, P=1000)
    poly = rounded(poly)
    X32 = X.astype(np.float32)
    dp32 = pl.to_device(poly, dtype=torch.float32)
    F, G, H = pl.eval_derivs(dp32, torch.as_tensor(X32, device="cuda"))
    assert F.dtype == torch.float32
    F64, G64, H64 = pl.eval_derivs(pl.to_device(poly), torch.as_tensor(X32.astype(np.float64), device="cuda"),
                                   prec="fp32")
    Fo, Go, Ho, SF, SG, SH = derivs.eval_derivs(poly.exps, poly.coef, X32.astype(np.float64), order=2)
    for a, b, o, sc in ((F, F64, Fo, SF), (G, G64, Go, SG), (H, H64, Ho, SH)):
        a = a.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(a - o) <= 2e-6 * sc + 1e-30)
        assert np.all(np.abs(a - b.cpu().numpy()) <= 4e-6 * sc + 1e-30)


def test_affine_exact(pl):
    poly, X = workloads.affine_small(P=512)
    poly = rounded(poly)
    X32 = X.astype(np.float32)
    D, Du, info = pl.affine_normal(pl.to_device(poly, dtype=torch.float32), torch.as_tensor(X32, device="cuda"),
                                   regularization=1e-6)
    assert D.dtype == torch.float32 and Du.dtype == torch.float32
    fl = pl.info_numpy(info)["flags"]
    D = D.cpu().numpy().astype(np.float64)
    for i in range(0, 512, 4):
        x = X32[i].astype(np.float64)
        nu, _, oi = affine.affine_normal_ad(poly.exps, poly.coef, x, r=1e-6)
        kap, amb = kappa_and_ambiguity(poly, x, 1e-6)
        if amb:
            continue
        assert fl[i] == oi["flags"]
        if oi["flags"] == 0:
            assert np.radians(affine.angle_deg(D[i], nu)) <= 2e-5 * max(kap, 1.0)


def test_affine_stochastic(pl):
    """The FP32 form's bar of the stochastic tests: within 2e-3 rad of the
    stochastic oracle with the same probes (q = 16, tol 1e-4)."""
    poly, X = quartic6()
    poly = rounded(poly)
    X32 = X.astype(np.float32)
    D, Du, info = pl.affine_normal(pl.to_device(poly, dtype=torch.float32), torch.as_tensor(X32, device="cuda"),
                                   method="mf-stochastic", regularization=1e-6, num_probes=16, krylov_tol=1e-4,
                                   krylov_maxit=40, seed=5)
    D = D.cpu().numpy().astype(np.float64)
    for j in range(X.shape[0]):
        nu, _, _ = affine.affine_normal_stochastic(poly.exps, poly.coef, X32[j].astype(np.float64), r=1e-6, q=16,
                                                   tol=1e-4, maxit=40, seed=5, point_index=j)
        assert np.radians(affine.angle_deg(D[j], nu)) <= 2e-3, j


def test_argument_errors(pl):
    poly, X = workloads.affine_small(P=4)
    dp = pl.to_device(poly, dtype=torch.float32)
    Xd = torch.as_tensor(X.astype(np.float32), device="cuda")
    with pytest.raises(pl.PolylabError) as ei:
        pl.affine_normal(dp, Xd, method="ad")
    assert ei.value.status == 1
    with pytest.raises(pl.PolylabError) as ei:
        pl.affine_normal(dp, Xd, prec="fp64")
    assert ei.value.status == 1
    with pytest.raises(ValueError):
        pl.eval_derivs(dp, Xd, prec="bf16")
