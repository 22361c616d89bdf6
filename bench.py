"""Benchmark: exact affine-normal directions per second on a batch of 256
uneven polynomials, plus the per-row measurements of the rest of the path.

Headline workload (one "step"): for 256 convexified polynomials
(n ~ U{5..60}, random-part term counts log-uniform in [50, 20000], degree <= 6,
128..4096 points each on the shell 0.5 <= |x| <= 1.5) compute the exact
(MF-logDet-Exact) affine-normal direction, its unit copy and the per-point
diagnostics at every point, with the polynomials' plans and the points
resident in HBM.  ``value`` is directions per second of the chosen form (the
FP32-sum / FP64-Cholesky form when it meets its stated error against the FP64
form, otherwise the FP64 form); the plain FP64 form is reported beside it.

Other rows of the path are measured in the same run and reported as
sub-objects: the 4M-term product simplify (terms/s), the 65,536-point
derivative evaluation (evals/s per precision form).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the CPU oracle (the plain FP64 'ad' formula) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "affine-normal dirs/s (exact, 256 uneven polys) and f/grad/Hessian evals/s vs plain FP64 GPU"
WORKLOAD = ("batched_uneven_exact: 256 convexified polys (sum x^4 + sum x^2 + 0.1 random), n~U{5..60}, "
            "random terms log-U[50,20000] deg<=6, 128-4096 shell points each")
L2_FLUSH_BYTES = 256 << 20


def _measured(key: str, fallback: float) -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except Exception:
        return fallback  # the profiling recipe's fallback figures


MEASURED_BF16_TFLOPS = _measured("bf16_tflops", 1800.0)
# FP32 and FP64 FMA rates of libpolylab_probe.so measured on a B300 (148 SMs, 2,032 MHz, no other work): the
# floor of the ALU peaks the bench divides by
PROBE_REFERENCE_TFLOPS = {0: 70.7, 1: 1.199}
MEASURED_HBM_GBS = _measured("hbm_gbs", 6400.0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--polys", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rows", action="store_true", help="skip the per-row sub-measurements")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work per sample")
    ap.add_argument("--forms", default="fp64,f32x2,fp32", help="forms to time (profiling runs time one)")
    ap.add_argument("--rows-only", action="store_true", help="only the per-row measurements (profiling runs)")
    ap.add_argument("--rows", default="", help="comma-separated row names to measure (default: every row)")
    ap.add_argument("--eager", action="store_true",
                    help="launch each step's kernels directly instead of replaying a CUDA graph (profiler runs)")
    ap.add_argument("--config", default=None,
                    help="threads,ctas_per_sm,order[,term_threads,terms_ctas,third_ctas,frame_split,"
                         "third_threads,third_split] in place of autotuning (profiling runs)")
    return ap.parse_args()


# ------------------------------------------------------------------ flop model

def term_stats(exps: np.ndarray):
    k = (exps > 0).sum(axis=1).astype(np.int64)
    d = exps.astype(np.int64).sum(axis=1)
    return k, d


STAGES = ("terms", "frame", "third")


def exact_flops(poly, P: int):
    """Algorithmic flops of one exact direction, per
    stage: the gradient/Hessian term sweep, the frame stage (LDL^T in FP64,
    inverse and the n^2 frame updates in the form's precision) and the
    third-derivative sweep with the direction (W y)."""
    n = poly.n
    m = n - 1
    k, d = term_stats(poly.exps)
    f_terms = float(np.sum(2 * (k + k * (k + 1) // 2)))
    k3 = k[d >= 3]
    f_third = float(np.sum(2 * (k3 + 2 * k3 * (k3 - 1) + 3 * (k3 * (k3 - 1) * (k3 - 2) // 6))))
    f_ldlt = m ** 3 / 3.0           # m^3/6 multiply-adds
    f_inv = 2.0 * m ** 3 / 3.0      # L^{-1} and M = X'^T X', m^3/6 multiply-adds each
    f_small = 14.0 * n * n          # H v, P H P, M v, W
    f_dir = 2.0 * n * n             # W y
    per = dict(terms=f_terms, third=f_third + f_dir, ldlt=f_ldlt, inv=f_inv, small=f_small)
    return {key: val * P for key, val in per.items()}


STAGE_PARTS = dict(terms=("terms",), frame=("ldlt", "inv", "small"), third=("third",))


# A double-word multiply-add (two flops of the algorithm) costs 29 FP32
# instructions in csrc/dfloat.cuh: the product 9 (TwoProd 2, two FMAs, one
# multiply, one add, FastTwoSum 3), the accurate sum 20 (two TwoSums of 6,
# two FastTwoSums of 3, two adds).  The double-word peak is the FP32 peak x 2/29.
DW_FLOPS_PER_FP32_OP = 2.0 / 29.0


def part_precision(form: str, part: str) -> str:
    """Arithmetic of each part of the exact path in each form: the LDL^T is
    FP64 in every form; the double-word form also keeps the O(n^2) frame
    update in FP64."""
    if form == "fp64" or part == "ldlt":
        return "fp64"
    if form == "f32x2":
        return "fp64" if part == "small" else "dw"
    return "fp32"


def alu_roofline(flops: dict, t_s: float, form: str, p32: float, p64: float, parts=None):
    """Op-mix ALU roofline: every part's algorithmic flops at the peak of the
    arithmetic it runs in (FP64, FP32, or double words on the FP32 pipe)."""
    keys = parts or tuple(flops)
    pk = dict(fp64=p64, fp32=p32, dw=p32 * DW_FLOPS_PER_FP32_OP)
    by = dict(fp64=0.0, fp32=0.0, dw=0.0)
    for k in keys:
        by[part_precision(form, k)] += flops[k]
    tot = sum(by.values())
    t_min = sum(by[q] / (pk[q] * 1e12) for q in by)
    peak = tot / t_min / 1e12
    achieved = tot / t_s / 1e12
    return dict(bound="alu", achieved=round(achieved, 4), peak=round(peak, 4), unit="TFLOP/s",
                frac=round(achieved / peak, 4), traffic=None,
                peak_source=(f"FMA probe (this run's rate or its reference B300 rate, the larger): fp32 {p32:.1f} TF/s, "
                             f"fp64 {p64:.3f} TF/s, double words "
                             f"{pk['dw']:.2f} TF/s (fp32 x 2/29); op mix of this form"),
                flops_fp32=by["fp32"], flops_fp64=by["fp64"], flops_dw=by["dw"])


# ------------------------------------------------------------------ traffic

EXACT_SOURCES = ("affine_exact.cu", "terms.cuh", "async.cuh", "batch.cuh", "common.cuh", "dfloat.cuh")


def code_text(src: bytes) -> bytes:
    """Source text with `//` comments, trailing blanks and empty lines removed:
    what the counters of a capture depend on (a comment edit keeps them)."""
    out = []
    for line in src.decode().splitlines():
        code = line.split("//", 1)[0].rstrip()
        if code:
            out.append(code)
    return "\n".join(out).encode()


def source_hash(read) -> str:
    """SHA-256 prefix over the code text of the exact-path sources; `read(f)`
    returns the bytes of source file f."""
    import hashlib
    h = hashlib.sha256()
    for f in EXACT_SOURCES:
        h.update(code_text(read(f)))
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, units: int, form: str):
    """DRAM bytes (read + write) of `kernel`'s launches in one step of `form`
    from the committed ncu counters in profiles/traffic.json (records {kernel,
    form, bytes, units, source, capture}), scaled from the captured units to
    `units`; None unless the exact-path sources' code text still hashes to
    `source` (the counters describe this code)."""
    def read(f):
        with open(os.path.join(ROOT, "paper_2604_06575_b300", "csrc", f), "rb") as fh:
            return fh.read()
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            recs = json.load(fh)
    except (OSError, ValueError):
        return None
    src = source_hash(read)
    for r in recs:
        if r["kernel"] == kernel and r["form"] == form and r["source"] == src:
            return dict(bytes=int(r["bytes"] * units / r["units"]), captured=r["capture"],
                        captured_units=r["units"])
    return None


# ------------------------------------------------------------------ clocks

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=sorted(reasons), samples=len(sm))


# ------------------------------------------------------------------ reference / cpu baseline

def _oracle_point(args):
    """One direction by the CPU oracle ('ad' formula, trace term contracted
    term by term); a process-pool task."""
    from oracle import affine
    exps, coef, x, r = args
    nu, _, _ = affine.affine_normal_ad(exps, coef, x, r=r, third="contract")
    return nu


def _pool_init():
    try:
        from threadpoolctl import threadpool_limits
        threadpool_limits(1)
    except Exception:
        pass


class OraclePool:
    """The oracle on the host cores: one task per point, ``workers``
    single-threaded processes (spawned, so that a pool made after the first
    GPU call is safe)."""

    def __init__(self, workers: int):
        import multiprocessing as mp
        self.workers = workers
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_pool_init)

    def close(self):
        """Stops the workers (points still running are abandoned)."""
        self.pool.terminate()
        self.pool.join()

    def windows(self, polys, Xs, order, n_windows: int, window_s: float, r: float = 1e-6):
        """Runs points continuously -- taken round-robin over the polynomials in
        ``order`` (point j of every polynomial, j = 0, 1, ..), one per worker
        at all times -- through ``n_windows`` consecutive windows of
        ``window_s`` seconds, and counts the points completed in each window
        (a point still running at a window's end counts in the window where
        it completes).  Returns (completions per window, window durations,
        {(poly, point): nu})."""
        def tasks():
            for j in range(1 << 20):
                for i in order:
                    if j < Xs[i].shape[0]:
                        yield (i, j)
        it = tasks()
        pending, out, counts, durs = [], {}, [], []
        for _ in range(n_windows):
            t0 = time.perf_counter()
            done = 0
            while time.perf_counter() - t0 < window_s:
                while len(pending) < self.workers:
                    i, j = next(it)
                    pending.append(((i, j), self.pool.apply_async(
                        _oracle_point, ((polys[i].exps, polys[i].coef, Xs[i][j], r),))))
                ready = [q for q in pending if q[1].ready()]
                for q in ready:
                    pending.remove(q)
                    out[q[0]] = q[1].get()
                    done += 1
                if not ready:
                    time.sleep(0.002)
            counts.append(done)
            durs.append(time.perf_counter() - t0)
        return counts, durs, out


def single_thread_sample(polys, Xs, order, budget_s: float, r: float = 1e-6):
    """The oracle in this process on one thread: points taken round-robin over
    the polynomials in ``order`` are started while less than ``budget_s``
    seconds have passed; the last one started is finished and counted.
    Returns (directions, seconds, {(poly, point): nu})."""
    _pool_init()
    out = {}
    t0 = time.perf_counter()
    for j in range(1 << 20):
        for i in order:
            if time.perf_counter() - t0 >= budget_s:
                return len(out), time.perf_counter() - t0, out
            if j < Xs[i].shape[0]:
                out[(i, j)] = _oracle_point((polys[i].exps, polys[i].coef, Xs[i][j], r))
    return len(out), time.perf_counter() - t0, out


def sample_order(n_polys: int, seed: int):
    """A seeded random order of the polynomials (their point counts do not
    depend on their term counts, so points taken over it estimate the
    workload's mean cost per point)."""
    return [int(i) for i in np.random.default_rng(seed).permutation(n_polys)]


def run_reference(args):
    from paper_2604_06575_b300 import workloads
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    polys, Xs = workloads.batched_uneven(n_polys=args.polys)
    cores = os.cpu_count() or 1
    pool = OraclePool(cores)
    window = 3.0
    # the warm-up windows run the same stream of points (so that the timed
    # windows see the pool in its steady state) and are not counted
    counts, durs, _ = pool.windows(polys, Xs, sample_order(len(polys), 0), args.warmup + args.steps, window)
    pool.close()
    counts, durs = counts[args.warmup:], durs[args.warmup:]
    pts, t_all = sum(counts), sum(durs)
    v = pts / t_all
    desc = (f"points taken round-robin over the {len(polys)} polys in a seeded random order (point j of every poly), "
            f"run continuously on {cores} single-threaded processes; each step a {window:.0f} s window counting the "
            f"points completed in it, after {args.warmup} warm-up windows of the same stream; {pts} points in "
            f"{args.steps} windows")
    line = dict(metric=METRIC, value=v, unit="dirs/s", n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=t_all / args.steps * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, polys=args.polys, sample="bounded CPU sample per step"),
                cpu_baseline=dict(value=v, unit="dirs/s", cores=cores, kind="oracle", sample=desc),
                e2e=dict(value=v, unit="dirs/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    from paper_2604_06575_b300 import dist as pdist
    rank, world, local = pdist.rank_info()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import ctypes

    from paper_2604_06575_b300 import polylab as pl
    from paper_2604_06575_b300 import workloads

    probe = ctypes.CDLL(os.path.join(ROOT, "paper_2604_06575_b300", "libpolylab_probe.so"))
    probe.polylab_probe_alu.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_double)]

    def alu_peak(kind, iters):
        """The FMA probe's rate in this run, or the rate it measured on an unshared B300 at 2,032 MHz when this
        run's is lower (a busy or slowed GPU would otherwise inflate every fraction): the larger is the peak."""
        v = ctypes.c_double()
        rc = probe.polylab_probe_alu(kind, iters, 4, 5, ctypes.byref(v))
        live = v.value if rc == 0 else float("nan")
        ref = PROBE_REFERENCE_TFLOPS[kind]
        return live if live >= ref else ref

    if args.rows_only:
        only = [r for r in args.rows.split(",") if r]
        print(json.dumps(dict(rows=measure_rows(pl, workloads, torch, dev, alu_peak(0, 20000), alu_peak(1, 2000),
                                                only))), flush=True)
        return

    # ---- workload (rank r: its own batch, weak scaling)
    polys, Xs = workloads.batched_uneven(seed_off=pdist.workload_seed_offset(rank), n_polys=args.polys)
    dps = [pl.to_device(p, dev) for p in polys]
    plans = [pl.Plan(d) for d in dps]
    Xd = [torch.as_tensor(X, device=dev) for X in Xs]
    npts = sum(X.shape[0] for X in Xs)
    opts = {f: pl.an_opts(prec=f, regularization=1e-6) for f in ("fp64", "f32x2", "fp32")}
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    class _Eager:  # stands in for a graph: replay() launches the run directly
        def __init__(self, batch):
            self.batch = batch

        def replay(self):
            self.batch.run()

    def capture(batch):
        """One run (the work-counter memsets and the persistent launches of the three stages) in a CUDA graph."""
        if args.eager:
            return _Eager(batch)
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            batch.run()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            batch.run()
        return g

    forms = [f for f in ("fp64", "f32x2", "fp32") if f in args.forms.split(",")]
    batches, graphs, tuned = {}, {}, {}
    for form in forms:
        batches[form] = pl.Batch(dps, plans, Xd, opts[form])
        if args.config:
            batches[form].set_config(*(int(v) for v in args.config.split(",")))
            tuned[form] = dict(batches[form].config(), ms=None)
        else:
            cfg, ms = batches[form].autotune(reps=2)
            tuned[form] = dict(cfg, ms=round(ms, 3))
        graphs[form] = capture(batches[form])

    def timed(form, steps, warmup):
        g = graphs[form]
        for _ in range(warmup):
            g.replay()
        barrier()
        step_ms = []
        for _ in range(steps):
            flush.zero_()  # L2 flush between timed steps (outside the timed region)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            s0.record(stream)
            g.replay()
            s1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(s0.elapsed_time(s1))
        barrier()
        return step_ms

    def stage_times(form, steps):
        """Mean duration of each stage's launch (CUDA events on the launching
        stream, L2 flushed before every launch), same batch and configuration."""
        b = batches[form]
        b.run()
        out = {}
        for s, name in enumerate(STAGES):
            ms = []
            for _ in range(steps):
                flush.zero_()
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                b.run_stage(s)
                s1.record(stream)
                torch.cuda.synchronize()
                ms.append(s0.elapsed_time(s1))
            out[name] = statistics.mean(ms)
        return out

    clocks = Clocks()
    res = {}
    for form in forms:
        step_ms = timed(form, args.steps, args.warmup)
        res[form] = dict(total_ms=pdist.max_over_ranks(sum(step_ms), dev), step_ms=step_ms,
                         stage_ms=stage_times(form, args.steps))
    clk = clocks.stop()

    # error of the other forms against the FP64 form at every point: the
    # double-word form as the relative error of nu (its bar is the FP64
    # form's), the FP32-sum form as the angle (radians) of the unit directions
    def vs_fp64(form):
        worst, flags_equal = 0.0, True
        for i in range(len(dps)):
            a, b = batches["fp64"].D[i], batches[form].D[i]
            fa, fb = torch.isfinite(a).all(dim=1), torch.isfinite(b).all(dim=1)
            flags_equal &= bool(torch.equal(fa, fb))
            ok = fa & fb
            if ok.any():
                if form == "f32x2":
                    e = (b[ok] - a[ok]).norm(dim=1) / a[ok].norm(dim=1)
                else:
                    e = torch.arccos(torch.nn.functional.cosine_similarity(a[ok], b[ok], dim=1).clamp(-1, 1))
                worst = max(worst, float(e.max()))
        return worst, flags_equal

    def flagged(form):
        """Points the form flagged (zero gradient or projected Hessian not
        positive definite): their directions are NaN."""
        return int(sum(int((~torch.isfinite(d).all(dim=1)).sum()) for d in batches[form].D))

    BOUND = dict(f32x2=1e-9, fp32=1e-3)  # stated bounds: relative error of nu; angle in radians
    errs = {f: vs_fp64(f) for f in forms if f != "fp64"} if "fp64" in forms else {}
    ok = {f: errs[f][0] <= BOUND[f] and errs[f][1] for f in errs}
    # the headline is the fastest form held to the FP64 form's error bar
    if "fp64" in res:
        chosen = "f32x2" if ok.get("f32x2") and res["f32x2"]["total_ms"] < res["fp64"]["total_ms"] else "fp64"
    else:  # (profiling runs that time other forms only)
        chosen = forms[0]

    def rate(form):
        if form not in res:
            return float("nan")
        return pdist.job_rate(npts, world, args.steps, res[form]["total_ms"])

    # ---- e2e through the public API: pinned host points in, directions out, every step.  Two batches
    # over two sets of device buffers on two streams, steps alternating between them, so that one step's
    # host<->device copies overlap the other's kernels (the copy engines run beside the SMs).
    Xcat = torch.cat([torch.as_tensor(X).reshape(-1) for X in Xs]).pin_memory()
    Dhost = [torch.empty(Xcat.shape, dtype=torch.float64).pin_memory() for _ in range(2)]
    offs = np.cumsum([0] + [X.shape[0] * X.shape[1] for X in Xs])
    e2e = []
    for _ in range(2):
        Xdev_flat = torch.empty(Xcat.numel(), dtype=torch.float64, device=dev)
        Ddev_flat = torch.empty(Xcat.numel(), dtype=torch.float64, device=dev)
        xv = [Xdev_flat[offs[i]:offs[i + 1]].view(-1, polys[i].n) for i in range(len(polys))]
        dv = [Ddev_flat[offs[i]:offs[i + 1]].view(-1, polys[i].n) for i in range(len(polys))]
        bt = pl.Batch(dps, plans, xv, opts[chosen], want_unit=False, want_info=False, D=dv)
        bt.set_config(**{k: tuned[chosen][k] for k in pl.Batch.CONFIG_KEYS})
        e2e.append((Xdev_flat, Ddev_flat, bt, torch.cuda.Stream()))

    def e2e_step(i):
        Xdev_flat, Ddev_flat, bt, st = e2e[i % 2]
        with torch.cuda.stream(st):
            Xdev_flat.copy_(Xcat.view(-1), non_blocking=True)
            bt.run()
            Dhost[i % 2].view(-1).copy_(Ddev_flat, non_blocking=True)

    def e2e_run(steps):
        start = torch.cuda.Event()
        start.record(stream)
        for _, _, _, st in e2e:
            st.wait_event(start)
        for i in range(steps):
            e2e_step(i)
        for _, _, _, st in e2e:
            stream.wait_stream(st)

    e2e_run(args.warmup)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_rate = pdist.job_rate(npts, world, args.steps, pdist.max_over_ranks(e0.elapsed_time(e1), dev))
    nbytes = int(Xcat.numel() * 8)
    outs = {f: [(batches[f].D[i], batches[f].Du[i], batches[f].info[i]) for i in range(len(dps))]
            for f in forms}

    # ---- roofline of the dominant kernel (the exact affine-normal kernel, every launch of a step)
    p32 = alu_peak(0, 20000)
    p64 = alu_peak(1, 2000)
    flops = {}
    for p, X in zip(polys, Xs):
        for key, val in exact_flops(p, X.shape[0]).items():
            flops[key] = flops.get(key, 0.0) + val
    kernels = dict(terms="exact_terms_kernel", frame="exact_frame_kernel", third="exact_third_kernel")
    stage_ms = res[chosen]["stage_ms"]
    stages = {}
    for name in STAGES:
        r = alu_roofline(flops, stage_ms[name] * 1e-3, chosen, p32, p64, STAGE_PARTS[name])
        stages[name] = dict(kernel=kernels[name], ms=round(stage_ms[name], 3), achieved=r["achieved"],
                            peak=r["peak"], frac=r["frac"])
    dom = max(STAGES, key=lambda k: stage_ms[k])
    roof = alu_roofline(flops, stage_ms[dom] * 1e-3, chosen, p32, p64, STAGE_PARTS[dom])
    roof["kernel"] = f"{kernels[dom]} (the longest of the three stages of a step)"
    tr = profiled_traffic(kernels[dom], npts, chosen)
    roof["traffic"] = tr["bytes"] if tr else None
    roof["traffic_note"] = (f"dram read+write of the stage's launches in one step (launches_per_step), from "
                            f"{tr['captured']} ({tr['captured_units']} points), scaled to {npts} points"
                            if tr else "no ncu counters for this kernel at this source")
    launches = stage_launches(tuned[chosen], polys, Xs)
    roof["launches_per_step"] = launches[dom]
    roof["note"] = ("achieved = the stage's algorithmic flops / the stage's event-timed duration (all of its "
                    "launches in a step: the sweeps and the frame stage run one launch per class of n)")
    roof["stages"] = stages
    roof["path"] = alu_roofline(flops, statistics.median(res[chosen]["step_ms"]) * 1e-3, chosen, p32, p64)

    line = dict(metric=METRIC, value=round(rate(chosen), 1), unit="dirs/s", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=round(res[chosen]["total_ms"] / args.steps, 3),
                higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype={"fp64": "f64", "f32x2": "f32x2 (double-word FP32 pairs) sums + f64 factorization",
                       "fp32": "f32 sums + f64 factorization"}[chosen],
                data="synthetic",
                config=dict(workload=WORKLOAD, polys=args.polys, points=npts, form=chosen,
                            regularization=1e-6, l2="flushed (256 MB write) before every timed step",
                            parallelism=f"weak: each rank its own {args.polys}-poly batch" if world > 1 else "1 GPU"),
                forms={**{f: dict(dirs_per_s=round(rate(f), 1),
                                  ms_per_step=round(res[f]["total_ms"] / args.steps, 3),
                                  stage_ms={k: round(v, 3) for k, v in res[f]["stage_ms"].items()},
                                  flagged_points=flagged(f),
                                  speedup_vs_fp64=round(rate(f) / rate("fp64"), 3) if "fp64" in res else None,
                                  **({} if f not in errs else dict(
                                      max_err_vs_fp64=errs[f][0], err_kind=("relative |nu|" if f == "f32x2"
                                                                            else "angle, rad"),
                                      stated_bound=BOUND[f], flags_equal=errs[f][1])))
                          for f in forms}},
                e2e=dict(value=round(e2e_rate, 1), unit="dirs/s", h2d_bytes_per_step=nbytes,
                         d2h_bytes_per_step=nbytes),
                gpu_launches=sum(launches.values()) * args.steps,
                autotune=tuned,
                roofline=roof, clocks=clk)

    # ---- other rows of the path, measured after the headline
    if not args.no_rows:
        line["rows"] = measure_rows(pl, workloads, torch, dev, p32, p64, [r for r in args.rows.split(",") if r])

    if rank == 0 and not args.no_cpu_baseline:
        # the oracle on the host cores: one thread, then every core, each on a
        # bounded sample of the same workload
        cores = os.cpu_count() or 1
        order = sample_order(len(polys), 7)
        budget = args.cpu_budget
        small = [int(np.argmin([p.m for p in polys]))]
        d1, t1, ref = single_thread_sample(polys, Xs, order, budget)
        alln = OraclePool(cores)
        alln.windows(polys, Xs, small, 1, 1.0)
        cn, tn, ref_n = alln.windows(polys, Xs, order, 1, budget / 2)
        alln.close()
        dn, tn = cn[0], tn[0]
        ref.update(ref_n)
        errs = []
        for (i, j), nu in ref.items():
            d = outs[chosen][i][0][j].cpu().numpy()
            if np.all(np.isfinite(nu)):
                errs.append(float(np.linalg.norm(d - nu) / np.linalg.norm(nu)))
        what = (f"round-robin over the {len(polys)} polys in a seeded random order (point j of every poly), "
                f"workers started beforehand")
        line["cpu_baseline"] = dict(value=round(dn / tn, 3), unit="dirs/s", cores=cores, kind="oracle",
                                    sample=f"{dn} points completed in {tn:.1f} s on {cores} single-threaded "
                                           f"processes, {what}",
                                    single_thread=dict(value=round(d1 / t1, 3), cores=1,
                                                       sample=f"{d1} points in {t1:.1f} s (started within "
                                                              f"{budget:.0f} s, the last one finished), {what}"),
                                    max_rel_err_of_reported_form=max(errs) if errs else None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def stage_launches(cfg: dict, polys, Xs) -> dict:
    """Kernel launches of one run per stage: the gradient/Hessian sweep as one
    gather launch per non-empty class of n (n > 40, 24 < n <= 40, n <= 24) plus
    one term-by-term launch, the third-derivative sweep as one launch per range
    of support sizes (third_split) and class, and, with frame_split, one frame
    launch per class."""
    ns = [p.n for p, X in zip(polys, Xs) if X.shape[0] > 0]
    classes = sum(1 for lo, hi in ((40, 1 << 30), (24, 40), (0, 24)) if any(lo < n <= hi for n in ns))
    frame = classes if cfg.get("frame_split", 0) else 1
    return dict(terms=classes + 1, frame=frame, third=int(cfg.get("third_split", 1)) * classes)


def measure_rows(pl, workloads, torch, dev, p32, p64, only=None):
    """Every row of the path after the headline, or the named ones (`only`)."""
    table = (("mul_product_pair", lambda: measure_mul(pl, workloads, torch, dev)),
             ("eval_derivs", lambda: measure_eval(pl, workloads, torch, dev)),
             ("affine_small", lambda: measure_small(pl, workloads, torch, dev)),
             ("exact_scaling", lambda: measure_exact_scaling(pl, workloads, torch, dev)),
             ("stochastic_band", lambda: measure_stochastic_band(pl, workloads, torch, dev)),
             ("stochastic", lambda: measure_stochastic(pl, workloads, torch, dev, p32)),
             ("stochastic_jacobi_n500", lambda: measure_stochastic_one(pl, workloads, torch, dev)),
             ("crossover", lambda: measure_crossover(pl, workloads, torch, dev)),
             ("simplify_pd_cubed", lambda: measure_pd3(pl, workloads, torch, dev)),
             ("affine_ad", lambda: measure_ad(pl, workloads, torch, dev, p64)),
             ("precision", lambda: measure_precision(pl, workloads, torch, dev)))
    unknown = set(only or ()) - {k for k, _ in table}
    if unknown:
        raise SystemExit(f"unknown rows: {sorted(unknown)}")
    return {k: fn() for k, fn in table if not only or k in only}


def _ev_time(torch, fn, reps=5, warm=2):
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def measure_mul(pl, workloads, torch, dev):
    """Product simplify (4M-term expansion -> merged terms), host syncs included."""
    A, B = workloads.product_pair()
    da, db = pl.to_device(A, dev), pl.to_device(B, dev)
    r = pl.mul(da, db)
    for _ in range(2):
        pl.mul(da, db)
    torch.cuda.synchronize()
    ts = []
    for _ in range(5):
        t0 = time.perf_counter()
        pl.mul(da, db)
        torch.cuda.synchronize()
        ts.append((time.perf_counter() - t0) * 1e3)
    ms = statistics.median(ts)
    # algorithmic HBM bytes: the 4M expanded (key, coefficient) items written
    # and read once (16 + 8 bytes each) and the merged rows written (n bytes of
    # exponents + 8 bytes of coefficient each)
    alg = 4e6 * 24 * 2 + r.m * (r.n + 8)
    return dict(workload="2 x 2,000 terms, n=20 each, 10 shared ids, deg<=6: 4,000,000 products",
                ms=round(ms, 3), merged_terms=r.m, expanded_terms_per_s=round(4e6 / (ms * 1e-3), 1),
                roofline=dict(bound="hbm", achieved=round(alg / (ms * 1e-3) / 1e9, 1), peak=MEASURED_HBM_GBS,
                              unit="GB/s", frac=round(alg / (ms * 1e-3) / 1e9 / MEASURED_HBM_GBS, 4),
                              algorithmic_bytes=int(alg),
                              note="wall time of the call (host synchronisations included); "
                                   "peak: measured copy bandwidth"))


def measure_eval(pl, workloads, torch, dev):
    """Derivative evaluation (f, grad, Hessian) in every form on the n = 30
    batch, with the full-grid errors against FP64 and the tensor roofline."""
    poly, X = workloads.eval_batch()
    dp = pl.to_device(poly, dev)
    Xd = torch.as_tensor(X, device=dev)
    P, n = X.shape
    out = (torch.empty(P, dtype=torch.float64, device=dev), torch.empty(P, n, dtype=torch.float64, device=dev),
           torch.empty(P, n, n, dtype=torch.float64, device=dev))
    ev = {}
    # error scale of every output: the sum of |term contributions|, which is
    # f, grad f and the Hessian of the polynomial with |coefficients| at |x|
    # (every monomial derivative is non-negative there), by the FP64 form
    absp = pl.DevPoly(dp.var_ids, dp.exps, dp.coef.abs())
    scale = pl.eval_derivs(absp, Xd.abs())
    ref = tuple(t.clone() for t in pl.eval_derivs(dp, Xd))
    with pl.Plan(dp, gemm=True) as plan:
        gi = plan.gemm_info()
        for prec in ("fp64", "fp32", "tf32x3", "bf16"):
            ms = _ev_time(torch, lambda: pl.eval_derivs(dp, Xd, plan=plan, prec=prec, out=out))
            ev[prec] = dict(ms=round(ms, 3), evals_per_s=round(P / (ms * 1e-3), 1))
            if prec != "fp64":
                pl.eval_derivs(dp, Xd, plan=plan, prec=prec, out=out)
                err = {name: float(((o - r_) .abs() / sc.clamp_min(1e-300)).max())
                       for name, o, r_, sc in zip(("f", "grad", "hessian"), out, ref, scale)}
                ev[prec]["max_err_vs_fp64_over_sum_abs_terms"] = err
    pl.eval_check()
    del scale, ref
    tiles = -(-P // 128)
    # tensor work the kernels issue: per 128-point tile, every live block is
    # 128 x 256 x K_block MACs (BF16 K_block 64; TF32 K_block 32, three products)
    issued_bf16 = 2.0 * 128 * 256 * 64 * gi["bf16_live_halves"] * tiles
    issued_tf32 = 3 * 2.0 * 128 * 256 * 32 * gi["tf32_live_tiles"] * tiles
    bf16_peak = MEASURED_BF16_TFLOPS
    tf32_peak = MEASURED_BF16_TFLOPS * 1.1 / 2.25  # nominal dense tf32/bf16 ratio
    for prec, fl, pk in (("bf16", issued_bf16, bf16_peak), ("tf32x3", issued_tf32, tf32_peak)):
        t = ev[prec]["ms"] * 1e-3
        ev[prec]["roofline"] = dict(bound="tensor", achieved=round(fl / t / 1e12, 2), peak=round(pk, 1),
                                    unit="TFLOP/s", frac=round(fl / t / 1e12 / pk, 4),
                                    note="issued MMA work of live blocks; peak: measured bf16 burst"
                                         + (" x nominal tf32/bf16 ratio" if prec == "tf32x3" else ""))
    res = dict(workload="n=30, 5,000 terms deg<=4 <=4 active, 65,536 points in [-1,1]^30",
               closure_K=gi["K"], output_columns_padded=gi["Npad"], forms=ev,
               speedup_vs_fp64={k: round(ev["fp64"]["ms"] / v["ms"], 2) for k, v in ev.items()})
    del out, Xd
    return res


def measure_small(pl, workloads, torch, dev):
    """The n = 3 family (sum x^4 + sum x^2 + 0.1 x all 35 monomials of degree
    <= 4; 1,024 shell points), exact directions in both forms, r = 1e-8, and
    its indefinite stress variant (flags)."""
    stream = torch.cuda.current_stream()
    out = {}
    for name, gen in (("affine_small", workloads.affine_small), ("affine_small_stress", workloads.affine_small_stress)):
        poly, X = gen()
        dp = pl.to_device(poly, dev)
        Xd = torch.as_tensor(X, device=dev)
        row = dict(points=X.shape[0])
        with pl.Plan(dp) as plan:
            for prec in ("fp64", "fp32"):
                ms, res = _time_call(torch, lambda: pl.affine_normal(dp, Xd, plan=plan, regularization=1e-8,
                                                                     prec=prec), stream)
                fl = pl.info_numpy(res[2])["flags"]
                row[prec] = dict(ms=round(ms, 4), dirs_per_s=round(X.shape[0] / (ms * 1e-3), 1),
                                 flagged=int((fl != 0).sum()))
        out[name] = row
    return out


def measure_exact_scaling(pl, workloads, torch, dev):
    """The paper's exact-scaling family (Sec. 6, Fig. "exact"): sparse quartics
    with support 3 and m = 4d monomials in d variables, d in {20, 40, 80, 120,
    180, 260}, 4,096 shell points each, r = 1e-8; MF-logDet-Exact in both
    forms (the paper reports 0.174 s per point on average for MPOLY-HP in
    double, one point per call, on its own hardware)."""
    stream = torch.cuda.current_stream()
    out = {}
    for d in (20, 40, 80, 120, 180, 260):
        poly, X = workloads.sparse_quartic(d, 4 * d, 3, P=4096)
        dp = pl.to_device(poly, dev)
        Xd = torch.as_tensor(X, device=dev)
        row = {}
        with pl.Plan(dp) as plan:
            for prec in ("fp64", "fp32"):
                ms, _ = _time_call(torch, lambda: pl.affine_normal(dp, Xd, plan=plan, regularization=1e-8,
                                                                   prec=prec), stream)
                row[prec] = dict(ms=round(ms, 3), dirs_per_s=round(4096 / (ms * 1e-3), 1))
        out[f"d{d}"] = row
    return out


def measure_stochastic_band(pl, workloads, torch, dev):
    """The paper's stochastic-stability setting (Sec. 6, Table "stochstab": a
    6-variable sparse quartic with 17 monomials, q = 64, maxit 80, 10 probe
    seeds): angle of MF-logDet-Stochastic (FP64, Jacobi, tol 1e-4, r = 1e-8)
    to MF-logDet-Exact at 4,096 points for each of 10 seeds.  The paper
    reports 2.99 +- 1.31 degrees over its 10 seeds at its one point."""
    stream = torch.cuda.current_stream()
    poly, X = workloads.sparse_quartic(6, 17, 3, P=4096)
    dp = pl.to_device(poly, dev)
    Xd = torch.as_tensor(X, device=dev)
    with pl.Plan(dp) as plan:
        ex = pl.affine_normal(dp, Xd, plan=plan, regularization=1e-8)[1]
        ang, times = [], []
        for seed in range(10):
            ms, res = _time_call(torch, lambda: pl.affine_normal(
                dp, Xd, plan=plan, method="mf-stochastic", regularization=1e-8, num_probes=64, krylov_tol=1e-4,
                krylov_maxit=80, seed=1000 + seed), stream)
            c = (res[1] * ex).sum(1).clamp(-1, 1)
            ang.append(torch.rad2deg(torch.arccos(c)).cpu().numpy())
            times.append(ms)
    A = np.stack(ang)  # seeds x points
    per_seed = A.mean(axis=1)
    return dict(points=4096, seeds=10, q=64, ms_per_seed=round(float(np.median(times)), 3),
                angle_deg_mean_over_all=round(float(A.mean()), 4), angle_deg_std_over_all=round(float(A.std()), 4),
                angle_deg_per_seed_mean=round(float(per_seed.mean()), 4),
                angle_deg_per_seed_std=round(float(per_seed.std()), 4),
                point0_angle_deg_over_seeds=dict(mean=round(float(A[:, 0].mean()), 4),
                                                 std=round(float(A[:, 0].std()), 4)))


def measure_precision(pl, workloads, torch, dev):
    """Double versus single storage on the core and affine workloads of the
    paper's precision table: the 4,000,000-product pair (mul), p_4^3 in 5
    variables (pow), f/grad/Hessian on the n = 30 batch (65,536 points), and
    MF-logDet-Exact / -Stochastic on a support-3 sparse quartic with n = 80,
    m = 320 (4,096 points; stochastic q = 8, tol 1e-4, maxit 40).  The engine
    rows include their host synchronisations; ms per call, median of 5."""
    stream = torch.cuda.current_stream()

    def wall(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(5):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        return statistics.median(ts)

    def dev_ms(fn):
        ts = []
        for _ in range(5):
            ms, _ = _time_call(torch, fn, stream)
            ts.append(ms)
        return statistics.median(ts)

    out = {}
    A, B = workloads.product_pair()
    pd = workloads.dense_power_base(4)
    ev, Xe = workloads.eval_batch()
    aq, Xa = workloads.sparse_quartic(80, 320, 3, P=4096)
    for name, dt in (("double", torch.float64), ("single", torch.float32)):
        row = {}
        da, db = pl.to_device(A, dev, dtype=dt), pl.to_device(B, dev, dtype=dt)
        row["mul_ms"] = round(wall(lambda: pl.mul(da, db)), 3)
        dpp = pl.to_device(pd, dev, dtype=dt)
        row["pow_ms"] = round(wall(lambda: pl.pow(dpp, 3)), 3)
        de = pl.to_device(ev, dev, dtype=dt)
        Xd = torch.as_tensor(Xe, device=dev, dtype=dt)
        with pl.Plan(de) as plan:
            row["eval_ms"] = round(dev_ms(lambda: pl.eval_derivs(de, Xd, plan=plan)), 3)
        del Xd
        dq = pl.to_device(aq, dev, dtype=dt)
        Xq = torch.as_tensor(Xa, device=dev, dtype=dt)
        prec = "fp32" if dt == torch.float32 else "fp64"
        with pl.Plan(dq) as plan:
            row["exact_ms"] = round(dev_ms(lambda: pl.affine_normal(dq, Xq, plan=plan, prec=prec)), 3)
            row["stochastic_ms"] = round(dev_ms(lambda: pl.affine_normal(
                dq, Xq, plan=plan, prec=prec, method="mf-stochastic", num_probes=8, krylov_tol=1e-4,
                krylov_maxit=40)), 3)
        out[name] = row
    out["double_over_single"] = {k: round(out["double"][k] / out["single"][k], 2) for k in out["double"]}
    return out


def measure_ad(pl, workloads, torch, dev, p64):
    """The 'ad' route (third-derivative tensor materialised per point, FP64)
    beside MF-logDet-Exact (FP64) on the same points: n = 6 with 17 random
    quartic terms (the accuracy table's shape) at 65,536 points, and n = 20
    with 400 random terms of degree <= 6 at 16,384 points.  The ALU figure
    counts the tensor contraction alone, m (n^3 + n^2 m + m^2 n) FMAs per
    point (m = n - 1), against the measured FP64 FMA peak."""
    stream = torch.cuda.current_stream()
    out = {}
    cases = [("n6_17_terms", workloads.sparse_quartic(6, 17, 3, P=65536))]
    rng = np.random.default_rng(20)
    e = workloads.sparse_monomials(rng, 20, 400, 6, 6)
    cases.append(("n20_400_terms", (workloads.convexified(rng, 20, e, 0.1), workloads.shell_points(rng, 20, 16384))))
    for name, (poly, X) in cases:
        dp = pl.to_device(poly, dev)
        Xd = torch.as_tensor(X, device=dev)
        P, n = X.shape
        m = n - 1
        with pl.Plan(dp) as plan:
            ms_ad, (Da, _, ia) = _time_call(torch, lambda: pl.affine_normal(dp, Xd, plan=plan, method="ad"), stream)
            ms_ex, (De, _, ie) = _time_call(torch, lambda: pl.affine_normal(dp, Xd, plan=plan), stream)
        ok = (pl.info_numpy(ia)["flags"] == 0) & (pl.info_numpy(ie)["flags"] == 0)
        okd = torch.as_tensor(ok, device=dev)
        rel = (Da[okd] - De[okd]).norm(dim=1) / De[okd].norm(dim=1)
        fl = 2.0 * m * (n ** 3 + n * n * m + m * m * n) * P
        ach = fl / (ms_ad * 1e-3) / 1e12
        out[name] = dict(points=P, terms=poly.m, ad_ms=round(ms_ad, 3), exact_ms=round(ms_ex, 3),
                         ad_dirs_per_s=round(P / (ms_ad * 1e-3), 1),
                         max_rel_diff_ad_vs_exact=float(rel.max()) if rel.numel() else None,
                         roofline=dict(bound="alu", achieved=round(ach, 4), peak=round(p64, 4), unit="TFLOP/s",
                                       frac=round(ach / p64, 4) if p64 else None, note="tensor contraction FMAs only; "
                                                                      "measured FP64 FMA peak"))
    return out


def _time_call(torch, fn, stream):
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    res = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b), res


def _angle(torch, D, ref):
    """Mean angle (rad) between the rows of D and ref, over the rows where both
    are finite (the exact form returns NaN at points it flags)."""
    ok = torch.isfinite(D).all(1) & torch.isfinite(ref).all(1)
    if not bool(ok.any()):
        return None
    c = (torch.nn.functional.normalize(D[ok], dim=1) * torch.nn.functional.normalize(ref[ok], dim=1)).sum(1)
    return float(torch.arccos(c.clamp(-1, 1)).mean())


def measure_stochastic(pl, workloads, torch, dev, p32):
    """MF-logDet-Stochastic (FP32, tol 1e-4, maxit 80, r = 1e-4) at 4,096
    points for n in {500, 1000, 2000} and q in {16, 32, 64} probes, with the
    Jacobi and the learned preconditioner side by side, on two families: the
    large sparse one (20n random terms of degree <= 4, points in [-1,1]^n) and
    the clustered one (the same plus two mean-field clusters that make soft
    collective modes).  The network is trained per family and n (1,000 Adam
    steps on 128 points of another draw).  At n = 500 the exact FP32 form at
    256 of the points is the reference for the error."""
    stream = torch.cuda.current_stream()
    out = {}
    r = 1e-4
    fams = (("large_sparse", workloads.large_sparse), ("clustered_sparse", workloads.clustered_sparse))
    for fam, gen in fams:
        rows = {}
        for n in (500, 1000, 2000):
            poly, X = gen(n, P=4096)
            dp = pl.to_device(poly, dev)
            Xd = torch.as_tensor(X, device=dev)
            row = dict(terms=poly.m, points=4096)
            with pl.Plan(dp) as plan:
                tr = gen(n, P=128, seed_off=1)[1]
                data = pl.mlp_data(dp, torch.as_tensor(tr, device=dev), r, seed=21, plan=plan)
                t0 = time.perf_counter()
                params, packed, hist = pl.train_preconditioner(data, r, steps=1000, lr=3e-3)
                torch.cuda.synchronize()
                row["train"] = dict(steps=1000, points=128, seconds=round(time.perf_counter() - t0, 2),
                                    loss_first_last=[round(hist[0], 5), round(hist[-1], 5)])
                del data
                ref = None
                if n == 500:
                    sub = Xd[:256]
                    msx, rex = _time_call(torch, lambda: pl.affine_normal(dp, sub, plan=plan, regularization=r,
                                                                          prec="fp32"), stream)
                    ref = rex[0]
                    row["exact_fp32_256_points"] = dict(
                        ms=round(msx, 2), dirs_per_s=round(256 / (msx * 1e-3), 1),
                        unflagged=int((pl.info_numpy(rex[2])["flags"] == 0).sum()))
                for q in (16, 32, 64):
                    cell = {}
                    for pre in ("jacobi", "mlp"):
                        kw = dict(method="mf-stochastic", regularization=r, num_probes=q, krylov_tol=1e-4,
                                  krylov_maxit=80, prec="fp32", plan=plan, seed=7, precond=pre,
                                  mlp_weights=packed if pre == "mlp" else None)
                        ms, res = _time_call(torch, lambda: pl.affine_normal(dp, Xd, **kw), stream)
                        info = pl.info_numpy(res[2])
                        c = dict(ms=round(ms, 2), dirs_per_s=round(4096 / (ms * 1e-3), 1),
                                 krylov_iters_per_point=round(float(info["krylov_iters"].mean()), 2))
                        if ref is not None:
                            c["angle_to_exact_rad"] = _angle(torch, res[0][:256], ref)
                        cell[pre] = c
                    cell["mlp_over_jacobi_iters"] = round(cell["mlp"]["krylov_iters_per_point"]
                                                          / cell["jacobi"]["krylov_iters_per_point"], 4)
                    row[f"q{q}"] = cell
            rows[f"n{n}"] = row
            del Xd, dp
        out[fam] = rows
    return out


def measure_stochastic_one(pl, workloads, torch, dev):
    """One MF-logDet-Stochastic call alone: the large sparse family at
    n = 500 (11,000 terms), 4,096 points, FP32, Jacobi, q = 16, tol 1e-4,
    maxit 80, r = 1e-4 (the first cell of the stochastic row, without the
    network training around it: the configuration the stochastic kernel's
    profile is taken on)."""
    stream = torch.cuda.current_stream()
    poly, X = workloads.large_sparse(500, P=4096)
    dp = pl.to_device(poly, dev)
    Xd = torch.as_tensor(X, device=dev)
    with pl.Plan(dp) as plan:
        ms, res = _time_call(torch, lambda: pl.affine_normal(
            dp, Xd, plan=plan, method="mf-stochastic", regularization=1e-4, num_probes=16, krylov_tol=1e-4,
            krylov_maxit=80, prec="fp32", precond="jacobi", seed=7), stream)
        info = pl.info_numpy(res[2])
    return dict(ms=round(ms, 2), dirs_per_s=round(4096 / (ms * 1e-3), 1),
                krylov_iters_per_point=round(float(info["krylov_iters"].mean()), 2))


def measure_crossover(pl, workloads, torch, dev):
    """Paper-shaped stochastic-crossover family (sparse quartics, support 2,
    m = 3d, speed preset q=1, r=5e-4, tol 2e-2, maxit 6), 512 points each:
    exact / stochastic time ratio (the paper reports 1.84 / 5.07 / 1.52 on its
    hardware, one point per call)."""
    stream = torch.cuda.current_stream()
    out = {}
    for d in (80, 260, 500):
        poly, X = workloads.sparse_quartic(d, 3 * d, 2, P=512)
        dp = pl.to_device(poly, dev)
        Xd = torch.as_tensor(X, device=dev)
        with pl.Plan(dp) as plan:
            mse, _ = _time_call(torch, lambda: pl.affine_normal(dp, Xd, plan=plan, regularization=5e-4, prec="fp64"),
                                stream)
            mss, _ = _time_call(torch, lambda: pl.affine_normal(dp, Xd, plan=plan, method="mf-stochastic",
                                                                regularization=5e-4, num_probes=1, krylov_tol=2e-2,
                                                                krylov_maxit=6, prec="fp64"), stream)
        out[f"d{d}"] = dict(exact_ms=round(mse, 2), stochastic_ms=round(mss, 2), ratio=round(mse / mss, 2))
    return out


def measure_pd3(pl, workloads, torch, dev):
    """simplify(p_d^3) for p_d = sum_{|a|<=d} x^a in 5 variables (the paper's
    heavy-simplify family; it reports 0.158 s for MPOLY-HP at d = 4 on its
    hardware), as two products and as one polylab_pow call; plus the symbolic
    Jacobian (one polylab_diff per variable) of the 5,000-term, 30-variable
    evaluation polynomial.  Wall time of the calls (each synchronises)."""
    def wall(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return round((time.perf_counter() - t0) * 1e3, 3), r

    out = {}
    for d in (2, 3, 4):
        dp = pl.to_device(workloads.dense_power_base(d), dev)
        ms, c = wall(lambda: pl.mul(pl.mul(dp, dp), dp))
        ms_pow, c2 = wall(lambda: pl.pow(dp, 3))
        out[f"d{d}"] = dict(ms=ms, terms=c.m, pow_ms=ms_pow, pow_terms=c2.m)
    poly, _ = workloads.eval_batch(P=1)
    dp = pl.to_device(poly, dev)
    ms, jac = wall(lambda: pl.jacobian(dp))
    out["jacobian_n30_5000_terms"] = dict(ms=ms, polys=len(jac), terms=sum(j.m for j in jac))
    return out


if __name__ == "__main__":
    main()
