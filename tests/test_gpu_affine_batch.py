"""The batched exact affine normal (one persistent launch over many uneven
polynomials) against the single-polynomial call and the oracle; every
launch configuration of the autotuner gives the same directions up to the
order of the shared-memory sums; a CUDA-graph replay of the batch as well."""
import numpy as np
import pytest
import torch

from oracle import affine
from paper_2604_06575_b300 import workloads

pytestmark = pytest.mark.gpu

# the order of the shared-memory atomic sums depends on the CTA size, so runs
# agree to rounding: relative 1e-10 (FP64 and double-word forms), 2e-4 (FP32 form)
TOL = {"fp64": 1e-10, "f32x2": 1e-10, "fp32": 2e-4}


def close(a, b, tol):
    fa, fb = torch.isfinite(a).all(dim=1), torch.isfinite(b).all(dim=1)
    assert torch.equal(fa, fb)
    if fa.any():
        err = (a[fa] - b[fa]).norm(dim=1) / b[fa].norm(dim=1)
        assert float(err.max()) <= tol, float(err.max())


@pytest.fixture(scope="module")
def pl(cuda_ok):
    from paper_2604_06575_b300 import polylab
    return polylab


@pytest.fixture(scope="module")
def batch_inputs():
    polys, Xs = workloads.batched_uneven(seed_off=7, n_polys=14, t_hi=3000, p_lo=3, p_hi=40)
    # plus two hand-made members: n = 1 and a flagged point
    polys.append(workloads.Poly(np.array([5], np.uint64), np.array([[2], [1]], np.uint8), np.ones(2)))
    Xs.append(np.array([[1.0], [-2.0], [0.25]]))
    polys.append(workloads.Poly(np.arange(2, dtype=np.uint64), np.array([[2, 0], [0, 2]], np.uint8), np.ones(2)))
    Xs.append(np.array([[0.0, 0.0], [0.3, 0.4]]))
    return polys, Xs


@pytest.mark.parametrize("prec", ["fp64", "f32x2", "fp32"])
def test_batch_matches_single_calls_and_oracle(pl, batch_inputs, prec):
    polys, Xs = batch_inputs
    dps = [pl.to_device(p) for p in polys]
    Xd = [torch.as_tensor(X, device="cuda") for X in Xs]
    opts = pl.an_opts(prec=prec, regularization=1e-6)
    plans = [pl.Plan(d) if i % 2 == 0 else None for i, d in enumerate(dps)]  # mix of given and built plans
    b = pl.Batch(dps, plans, Xd, opts)
    b.run()
    b.check()  # no bounded wait expired
    for i, (dp, X) in enumerate(zip(dps, Xd)):
        D1, Du1, in1 = pl.affine_normal(dp, X, opts)
        close(b.D[i], D1, TOL[prec])
        fl_b, fl_1 = pl.info_numpy(b.info[i])["flags"], pl.info_numpy(in1)["flags"]
        assert np.array_equal(fl_b, fl_1)
    if prec != "fp32":
        for i in range(len(polys)):
            for j in range(min(2, Xs[i].shape[0])):
                nu, _, oi = affine.affine_normal_ad(polys[i].exps, polys[i].coef, Xs[i][j], r=1e-6,
                                                    third="contract")
                d = b.D[i][j].cpu().numpy()
                if oi["flags"]:
                    assert np.all(np.isnan(d))
                else:
                    assert np.linalg.norm(d - nu) <= 1e-9 * np.linalg.norm(nu)


def test_autotune_configs_agree_and_graph_replay(pl, batch_inputs):
    polys, Xs = batch_inputs
    dps = [pl.to_device(p) for p in polys]
    Xd = [torch.as_tensor(X, device="cuda") for X in Xs]
    b = pl.Batch(dps, [None] * len(dps), Xd, pl.an_opts(prec="fp64"))
    b.run()
    torch.cuda.synchronize()
    ref = [d.clone() for d in b.D]
    for threads in (64, 128, 256):
        for cap, order, split, t3 in ((0, 1, 1, 128), (2, 0, 0, 64), (0, 1, 0, 256)):
            # frame stage split by n or one launch; CTA size of the third sweep
            b.set_config(threads, cap, order, frame_split=split, third_threads=t3)
            b.run()
            b.check()
            for d, r in zip(b.D, ref):
                close(d, r, TOL["fp64"])
    with pytest.raises(pl.PolylabError):
        b.set_config(128, 0, 1, third_threads=96)  # not a supported CTA size
    b.set_config(128, 0, 1, term_threads=128, terms_ctas=2, third_ctas=3, frame_split=1, third_threads=128)
    b.run()
    b.check()
    for d, r in zip(b.D, ref):
        close(d, r, TOL["fp64"])
    b.set_config(128, 0, 1, term_threads=128, terms_ctas=0, third_ctas=0, frame_split=1, third_threads=128)
    cfg, ms = b.autotune(reps=1)
    assert cfg["threads"] in (64, 128, 256) and ms > 0
    assert b.config() == cfg
    # capture one run (the tuned configuration) in a CUDA graph and replay it twice
    for d in b.D:
        d.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run()  # warm the launch path on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for d in b.D:
        d.zero_()
    with torch.cuda.graph(g):
        b.run()
    g.replay()
    g.replay()
    b.check()
    for d, r in zip(b.D, ref):
        close(d, r, TOL["fp64"])


def test_double_word_third_stage_ranges_agree(pl, batch_inputs):
    """The double-word third stage in one to four launches over ranges of
    support sizes (a kernel per range, one launch per class of n, the classes
    of smaller n at more resident CTAs) gives the FP64 form's directions within
    the double-word form's bar (relative 1e-9 on nu); a batch whose terms reach
    support 8 takes the kernels that keep support sizes 7 and 8."""
    rng = np.random.default_rng(23)
    wide = workloads.convexified(rng, 12, workloads.sparse_monomials(rng, 12, 300, 8, 8), 0.1)
    assert int((wide.exps > 0).sum(axis=1).max()) >= 7
    cases = [batch_inputs, ([wide], [workloads.shell_points(rng, 12, 96)])]
    for polys, Xs in cases:
        dps = [pl.to_device(p) for p in polys]
        Xd = [torch.as_tensor(X, device="cuda") for X in Xs]
        ref = pl.Batch(dps, [None] * len(dps), Xd, pl.an_opts(prec="fp64", regularization=1e-6))
        ref.run()
        ref.check()
        b = pl.Batch(dps, [None] * len(dps), Xd, pl.an_opts(prec="f32x2", regularization=1e-6))
        for split in (1, 2, 3, 4):
            b.set_config(128, 0, 1, term_threads=256, frame_split=1, third_threads=128, third_split=split)
            b.run()
            b.check()
            for d, r in zip(b.D, ref.D):
                close(d, r, 1e-9)
