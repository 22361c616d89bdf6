"""Thin ctypes binding of libpolylab.so (the C ABI declared in include/polylab.h).

Argument marshalling only: torch tensors are passed as raw device pointers
together with the current torch stream; every computation runs in the
library's CUDA kernels.  Importing this module loads the in-tree library and
raises if it is missing -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpolylab.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"libpolylab.so not built ({LIB_PATH}); run __graft_entry__.build()")
_lib = C.CDLL(LIB_PATH)

OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "EXP_OVERFLOW", 3: "DUP_VAR_ID", 4: "OOM", 5: "CUDA", 6: "TIMEOUT",
          7: "UNSUPPORTED"}
PREC = {"fp64": 0, "tf32x3": 1, "bf16": 2, "fp32": 3, "f32x2": 4}
METHOD = {"mf-exact": 0, "mf-stochastic": 1, "ad": 2}
AD_MAX_N = 24
PRECOND = {"jacobi": 0, "none": 1, "mlp": 2}
FLAG_ZERO_GRAD, FLAG_NOT_PD, FLAG_KRYLOV_MAXIT = 1, 2, 4


class PolylabError(RuntimeError):
    def __init__(self, fn: str, status: int):
        msg = _lib.polylab_last_error().decode()
        super().__init__(f"{fn}: {STATUS.get(status, status)}" + (f" [{msg}]" if msg and status in (5, 6) else ""))
        self.status = status


class _Poly(C.Structure):
    _fields_ = [("n_vars", C.c_int32), ("var_ids", C.POINTER(C.c_uint64)), ("n_terms", C.c_int64),
                ("exps", C.c_void_p), ("coef", C.c_void_p)]


class _PolyOut(C.Structure):
    _fields_ = [("n_vars", C.c_int32), ("var_ids", C.POINTER(C.c_uint64)), ("n_terms", C.c_int64),
                ("exps", C.c_void_p), ("coef", C.c_void_p)]


class _AnOpts(C.Structure):
    _fields_ = [("method", C.c_int), ("regularization", C.c_double), ("num_probes", C.c_int32),
                ("krylov_tol", C.c_double), ("krylov_maxit", C.c_int32), ("assume_nonzero_x", C.c_int32),
                ("seed", C.c_uint64), ("prec", C.c_int), ("precond", C.c_int), ("mlp_weights", C.c_void_p)]


class _BatchConfig(C.Structure):
    _fields_ = [("threads", C.c_int32), ("ctas_per_sm", C.c_int32), ("order", C.c_int32),
                ("term_threads", C.c_int32), ("terms_ctas", C.c_int32), ("third_ctas", C.c_int32),
                ("frame_split", C.c_int32), ("third_threads", C.c_int32), ("third_split", C.c_int32)]


INFO_DTYPE = np.dtype([("grad_norm", "<f8"), ("logdet", "<f8"), ("flags", "<i4"), ("hv_evals", "<i4"),
                       ("third_evals", "<i4"), ("krylov_iters", "<i4")])
assert INFO_DTYPE.itemsize == 32

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)

_lib.polylab_status_string.restype = C.c_char_p
_lib.polylab_last_error.restype = C.c_char_p
_lib.polylab_plan_closure_size.restype = C.c_int64
_lib.polylab_plan_closure_size.argtypes = [C.c_void_p]
_lib.polylab_plan_create.argtypes = [C.POINTER(_Poly), C.c_uint32, C.c_void_p, C.POINTER(C.c_void_p)]
_lib.polylab_plan_destroy.argtypes = [C.c_void_p, C.c_void_p]
_lib.polylab_plan_gemm_info.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                        C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
_lib.polylab_eval_derivs.argtypes = [C.POINTER(_Poly), C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
_lib.polylab_affine_normal.argtypes = [C.POINTER(_Poly), C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(_AnOpts),
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
_lib.polylab_simplify.argtypes = [C.POINTER(_Poly), C.c_double, C.POINTER(_PolyOut), ALLOC_FN, C.c_void_p,
                                  C.c_void_p]
_lib.polylab_mul.argtypes = [C.POINTER(_Poly), C.POINTER(_Poly), C.c_double, C.POINTER(_PolyOut), ALLOC_FN,
                             C.c_void_p, C.c_void_p]
_lib.polylab_add.argtypes = _lib.polylab_mul.argtypes
_lib.polylab_sub.argtypes = _lib.polylab_mul.argtypes
_lib.polylab_pow.argtypes = [C.POINTER(_Poly), C.c_int32, C.c_double, C.POINTER(_PolyOut), ALLOC_FN, C.c_void_p,
                             C.c_void_p]
_lib.polylab_diff.argtypes = [C.POINTER(_Poly), C.c_uint64, C.c_double, C.POINTER(_PolyOut), ALLOC_FN, C.c_void_p,
                              C.c_void_p]
_lib.polylab_simplify_noalloc.argtypes = [C.POINTER(_Poly), C.c_double, C.POINTER(_PolyOut), C.c_int64, C.c_void_p]
_lib.polylab_an_opts_default.argtypes = [C.POINTER(_AnOpts)]
_lib.polylab_eval_check.argtypes = [C.c_void_p]
_PP = C.POINTER(C.c_void_p)
_lib.polylab_batch_create.argtypes = [C.c_int32, C.c_void_p, _PP, _PP, C.POINTER(C.c_int64), C.POINTER(_AnOpts),
                                      _PP, _PP, _PP, C.c_void_p, C.POINTER(C.c_void_p)]
_lib.polylab_batch_run.argtypes = [C.c_void_p, C.c_void_p]
_lib.polylab_batch_run_stage.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
_lib.polylab_batch_check.argtypes = [C.c_void_p, C.c_void_p]
_lib.polylab_batch_get_config.argtypes = [C.c_void_p, C.POINTER(_BatchConfig)]
_lib.polylab_batch_set_config.argtypes = [C.c_void_p, C.POINTER(_BatchConfig), C.c_void_p]
_lib.polylab_batch_autotune.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(_BatchConfig),
                                        C.POINTER(C.c_float)]
_lib.polylab_batch_destroy.argtypes = [C.c_void_p, C.c_void_p]
_lib.polylab_mlp_param_count.restype = C.c_int32
_lib.polylab_mlp_init.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p]
_lib.polylab_mlp_data.argtypes = [C.POINTER(_Poly), C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_uint64,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
_lib.polylab_mlp_loss_grad.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]
_lib.polylab_mlp_adam.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float,
                                  C.c_void_p]
_lib.polylab_mlp_pack.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
_lib.polylab_affine_normal_batched.argtypes = [C.c_int32, C.c_void_p, _PP, _PP, C.POINTER(C.c_int64),
                                               C.POINTER(_AnOpts), _PP, _PP, _PP, C.c_void_p]
# single-precision storage: the same structs with FP32 coefficient pointers
for _f in ("simplify", "mul", "add", "sub", "pow", "diff", "plan_create"):
    getattr(_lib, f"polylab_{_f}_f32").argtypes = getattr(_lib, f"polylab_{_f}").argtypes
_lib.polylab_eval_derivs_f32.argtypes = [C.POINTER(_Poly), C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p]
_lib.polylab_affine_normal_f32.argtypes = _lib.polylab_affine_normal.argtypes
F32_CALLS = ["polylab_simplify_f32", "polylab_mul_f32", "polylab_add_f32", "polylab_sub_f32", "polylab_pow_f32",
             "polylab_diff_f32", "polylab_plan_create_f32", "polylab_eval_derivs_f32", "polylab_affine_normal_f32"]
for _f in ("polylab_plan_create", "polylab_plan_destroy", "polylab_eval_derivs", "polylab_eval_check",
           "polylab_affine_normal",
           "polylab_simplify", "polylab_mul", "polylab_add", "polylab_sub", "polylab_pow", "polylab_diff",
           "polylab_simplify_noalloc", "polylab_batch_create",
           "polylab_batch_run", "polylab_batch_run_stage", "polylab_batch_check", "polylab_batch_get_config",
           "polylab_batch_set_config", "polylab_batch_autotune", "polylab_batch_destroy", "polylab_affine_normal_batched",
           "polylab_plan_gemm_info", "polylab_mlp_init",
           "polylab_mlp_data", "polylab_mlp_loss_grad", "polylab_mlp_adam", "polylab_mlp_pack", *F32_CALLS):
    getattr(_lib, _f).restype = C.c_int

EXPORTED = ["polylab_status_string", "polylab_last_error", "polylab_simplify", "polylab_mul", "polylab_add",
            "polylab_sub", "polylab_pow", "polylab_diff",
            "polylab_plan_create", "polylab_plan_destroy", "polylab_plan_closure_size", "polylab_eval_derivs",
            "polylab_eval_check",
            "polylab_an_opts_default", "polylab_affine_normal", "polylab_simplify_noalloc", "polylab_batch_create",
            "polylab_batch_run", "polylab_batch_run_stage", "polylab_batch_check", "polylab_batch_get_config",
            "polylab_batch_set_config",
            "polylab_batch_autotune", "polylab_batch_destroy", "polylab_affine_normal_batched", "polylab_plan_gemm_info",
            "polylab_mlp_param_count", "polylab_mlp_init", "polylab_mlp_data", "polylab_mlp_loss_grad",
            "polylab_mlp_adam", "polylab_mlp_pack", *F32_CALLS]


def lib():
    return _lib


def _check(fn: str, st: int):
    if st != OK:
        raise PolylabError(fn, st)


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous()
    return t.data_ptr()


@dataclass
class DevPoly:
    """A polynomial whose exponents and coefficients live on the device.
    float32 coefficients select the library's single-precision storage calls
    (the ``*_f32`` entry points) in every function below."""
    var_ids: np.ndarray   # uint64[n] (host)
    exps: torch.Tensor    # uint8 [m, n] cuda
    coef: torch.Tensor    # float64 or float32 [m] cuda

    @property
    def n(self) -> int:
        return int(self.var_ids.shape[0])

    @property
    def m(self) -> int:
        return int(self.coef.shape[0])

    @property
    def f32(self) -> bool:
        return self.coef.dtype == torch.float32

    def cstruct(self) -> _Poly:
        ids = np.ascontiguousarray(self.var_ids, dtype=np.uint64)
        self._ids_keep = ids
        return _Poly(self.n, ids.ctypes.data_as(C.POINTER(C.c_uint64)), self.m, _ptr(self.exps), _ptr(self.coef))


def to_device(poly, device="cuda", dtype=torch.float64) -> DevPoly:
    """From any object with var_ids / exps / coef arrays (e.g. workloads.Poly);
    dtype=torch.float32 stores the coefficients rounded to FP32."""
    npd = np.float32 if dtype == torch.float32 else np.float64
    return DevPoly(np.asarray(poly.var_ids, dtype=np.uint64),
                   torch.as_tensor(np.ascontiguousarray(poly.exps, dtype=np.uint8), device=device),
                   torch.as_tensor(np.ascontiguousarray(poly.coef, dtype=npd), device=device))


def _call(name: str, *polys: DevPoly):
    """(name, function) of the FP64 call or its single-precision namesake."""
    f32 = {p.f32 for p in polys}
    if len(f32) != 1:
        raise ValueError("operands mix FP64 and FP32 coefficient storage")
    name = name + "_f32" if f32.pop() else name
    return name, getattr(_lib, name)


class Plan:
    """Device-resident preprocessed polynomial (polylab_plan)."""

    def __init__(self, p: DevPoly, gemm: bool = False):
        self.p = p
        self.h = C.c_void_p()
        cp = p.cstruct()
        name, fn = _call("polylab_plan_create", p)
        _check(name, fn(C.byref(cp), 1 if gemm else 0, _stream(), C.byref(self.h)))

    @property
    def closure_size(self) -> int:
        return int(_lib.polylab_plan_closure_size(self.h))

    def gemm_info(self) -> dict:
        K, N, h16, t32 = C.c_int64(), C.c_int32(), C.c_int64(), C.c_int64()
        _check("polylab_plan_gemm_info", _lib.polylab_plan_gemm_info(self.h, C.byref(K), C.byref(N), C.byref(h16),
                                                                     C.byref(t32)))
        return dict(K=K.value, Npad=N.value, bf16_live_halves=h16.value, tf32_live_tiles=t32.value)

    def close(self):
        if self.h:
            _lib.polylab_plan_destroy(self.h, _stream())
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def eval_derivs(p: DevPoly, X: torch.Tensor, order: int = 2, prec: str | None = None, plan: Plan | None = None,
                out=None):
    """F[P], G[P,n], H[P,n,n] on the device, in X's dtype: float64 points with
    an FP64-storage polynomial (prec: fp64 default, fp32, tf32x3, bf16),
    float32 points with an FP32-storage one (prec fp32 only)."""
    P, n = X.shape
    dt = torch.float32 if p.f32 else torch.float64
    assert n == p.n and X.dtype == dt
    if prec is None:
        prec = "fp32" if p.f32 else "fp64"
    if p.f32 and prec != "fp32":
        raise ValueError("FP32-storage polynomials evaluate in the fp32 form only")
    if out is None:
        F = torch.empty(P, dtype=dt, device=X.device)
        G = torch.empty(P, n, dtype=dt, device=X.device) if order >= 1 else None
        H = torch.empty(P, n, n, dtype=dt, device=X.device) if order >= 2 else None
    else:
        F, G, H = out
    cp = p.cstruct()
    ph = plan.h if plan else None
    if p.f32:
        _check("polylab_eval_derivs_f32", _lib.polylab_eval_derivs_f32(C.byref(cp), ph, _ptr(X), P, order, _ptr(F),
                                                                       _ptr(G), _ptr(H), _stream()))
    else:
        _check("polylab_eval_derivs", _lib.polylab_eval_derivs(C.byref(cp), ph, _ptr(X), P, order, PREC[prec],
                                                               _ptr(F), _ptr(G), _ptr(H), _stream()))
    return F, G, H


def eval_check():
    """Synchronise the current stream and raise if a bounded wait of a
    tensor-core evaluation expired since the last check."""
    _check("polylab_eval_check", _lib.polylab_eval_check(_stream()))


def an_opts(method="mf-exact", regularization=1e-6, num_probes=8, krylov_tol=1e-4, krylov_maxit=40,
            assume_nonzero_x=False, seed=20260321, prec="fp64", precond="jacobi", mlp_weights=None) -> _AnOpts:
    o = _AnOpts()
    _lib.polylab_an_opts_default(C.byref(o))
    o.method = METHOD[method]
    o.regularization = regularization
    o.num_probes = num_probes
    o.krylov_tol = krylov_tol
    o.krylov_maxit = krylov_maxit
    o.assume_nonzero_x = int(bool(assume_nonzero_x))
    o.seed = seed
    o.prec = PREC[prec]
    o.precond = PRECOND[precond]
    o.mlp_weights = _ptr(mlp_weights)
    return o


def affine_normal(p: DevPoly, X: torch.Tensor, opts: _AnOpts | None = None, plan: Plan | None = None,
                  want_unit: bool = True, want_info: bool = True, out=None, **kw):
    """(D, Dunit, info_bytes) on the device; ``info_numpy`` decodes info.  An
    FP32-storage polynomial takes float32 points, returns float32 directions
    and runs the fp32 form (the default ``prec`` for it)."""
    P, n = X.shape
    dt = torch.float32 if p.f32 else torch.float64
    assert n == p.n and X.dtype == dt
    if opts is None:
        if p.f32:
            kw.setdefault("prec", "fp32")
        o = an_opts(**kw)
    else:
        o = opts
    if out is None:
        D = torch.empty(P, n, dtype=dt, device=X.device)
        Du = torch.empty(P, n, dtype=dt, device=X.device) if want_unit else None
        info = torch.empty(P, 32, dtype=torch.uint8, device=X.device) if want_info else None
    else:
        D, Du, info = out
    cp = p.cstruct()
    name, fn = _call("polylab_affine_normal", p)
    _check(name, fn(C.byref(cp), plan.h if plan else None, _ptr(X), P, C.byref(o), _ptr(D), _ptr(Du), _ptr(info),
                    _stream()))
    return D, Du, info


def info_numpy(info: torch.Tensor) -> np.ndarray:
    return info.cpu().numpy().view(INFO_DTYPE).reshape(-1)


class _Allocs:
    def __init__(self, device):
        self.keep = []
        self.device = device

        def fn(nbytes, ctx):
            t = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
            self.keep.append(t)
            return t.data_ptr()

        self.fn = ALLOC_FN(fn)


def _run_out(name, call, n_cap: int, device, dtype=torch.float64):
    ids = np.zeros(max(n_cap, 1), dtype=np.uint64)
    out = _PolyOut(0, ids.ctypes.data_as(C.POINTER(C.c_uint64)), 0, None, None)
    al = _Allocs(device)
    _check(name, call(C.byref(out), al.fn))
    n, m = out.n_vars, out.n_terms
    by_ptr = {t.data_ptr(): t for t in al.keep}
    if m > 0:
        exps = by_ptr[out.exps][: m * n].view(m, n)
        coef = by_ptr[out.coef][: m * dtype.itemsize].view(dtype)
    else:
        exps = torch.zeros(0, n, dtype=torch.uint8, device=device)
        coef = torch.zeros(0, dtype=dtype, device=device)
    return DevPoly(ids[:n].copy(), exps, coef)


def simplify(p: DevPoly, zeroprec: float = 0.0) -> DevPoly:
    cp = p.cstruct()
    name, fn = _call("polylab_simplify", p)
    return _run_out(name, lambda o, al: fn(C.byref(cp), zeroprec, o, al, None, _stream()), p.n, p.coef.device,
                    p.coef.dtype)


def _binary(base: str, a: DevPoly, b: DevPoly, zeroprec: float) -> DevPoly:
    ca, cb = a.cstruct(), b.cstruct()
    name, fn = _call(base, a, b)
    return _run_out(name, lambda o, al: fn(C.byref(ca), C.byref(cb), zeroprec, o, al, None, _stream()), a.n + b.n,
                    a.coef.device, a.coef.dtype)


def mul(a: DevPoly, b: DevPoly, zeroprec: float = 0.0) -> DevPoly:
    return _binary("polylab_mul", a, b, zeroprec)


def add(a: DevPoly, b: DevPoly, zeroprec: float = 0.0) -> DevPoly:
    return _binary("polylab_add", a, b, zeroprec)


def sub(a: DevPoly, b: DevPoly, zeroprec: float = 0.0) -> DevPoly:
    return _binary("polylab_sub", a, b, zeroprec)


def pow(p: DevPoly, k: int, zeroprec: float = 0.0) -> DevPoly:
    cp = p.cstruct()
    name, fn = _call("polylab_pow", p)
    return _run_out(name, lambda o, al: fn(C.byref(cp), k, zeroprec, o, al, None, _stream()), p.n, p.coef.device,
                    p.coef.dtype)


def diff(p: DevPoly, var_id: int, zeroprec: float = 0.0) -> DevPoly:
    cp = p.cstruct()
    name, fn = _call("polylab_diff", p)
    return _run_out(name, lambda o, al: fn(C.byref(cp), int(var_id), zeroprec, o, al, None, _stream()), p.n,
                    p.coef.device, p.coef.dtype)


def jacobian(p: DevPoly, zeroprec: float = 0.0) -> list:
    """The n partial derivatives of p (one polylab_diff per variable)."""
    return [diff(p, int(v), zeroprec) for v in p.var_ids]


def simplify_noalloc(p: DevPoly, exps_out: torch.Tensor, coef_out: torch.Tensor, zeroprec: float = 0.0) -> DevPoly:
    """polylab_simplify without device allocation inside the call: the result
    is written to the caller's uint8 [capacity, n] and float64 [capacity]
    buffers and returned as views of them."""
    assert exps_out.dtype == torch.uint8 and coef_out.dtype == torch.float64
    cap = int(coef_out.shape[0])
    assert exps_out.shape == (cap, p.n)
    ids = np.zeros(max(p.n, 1), dtype=np.uint64)
    out = _PolyOut(0, ids.ctypes.data_as(C.POINTER(C.c_uint64)), 0, _ptr(exps_out), _ptr(coef_out))
    cp = p.cstruct()
    st = _lib.polylab_simplify_noalloc(C.byref(cp), zeroprec, C.byref(out), cap, _stream())
    _check("polylab_simplify_noalloc", st)
    m = int(out.n_terms)
    return DevPoly(ids[: out.n_vars].copy(), exps_out[:m], coef_out[:m])


def _ptr_array(ts):
    return (C.c_void_p * len(ts))(*[_ptr(t) if t is not None else None for t in ts])


class Batch:
    """A polylab_batch: exact directions for many polynomials in one launch.
    Holds references to every tensor it writes or reads."""

    def __init__(self, polys, plans, Xs, opts, want_unit=True, want_info=True, D=None):
        self.polys, self.plans, self.Xs, self.opts = polys, plans, Xs, opts
        dev = Xs[0].device
        self.D = D if D is not None else [torch.empty(X.shape, dtype=torch.float64, device=dev) for X in Xs]
        self.Du = [torch.empty(X.shape, dtype=torch.float64, device=dev) for X in Xs] if want_unit else None
        self.info = [torch.empty(X.shape[0], 32, dtype=torch.uint8, device=dev) for X in Xs] if want_info else None
        n = len(polys)
        cps = (_Poly * n)(*[p.cstruct() for p in polys])
        plan_arr = (C.c_void_p * n)(*[pl.h.value if pl is not None else None for pl in plans])
        P = (C.c_int64 * n)(*[int(X.shape[0]) for X in Xs])
        self.h = C.c_void_p()
        _check("polylab_batch_create", _lib.polylab_batch_create(
            n, C.cast(cps, C.c_void_p), plan_arr, _ptr_array(Xs), P, C.byref(opts), _ptr_array(self.D),
            _ptr_array(self.Du) if self.Du else None, _ptr_array(self.info) if self.info else None, _stream(),
            C.byref(self.h)))

    def run(self):
        _check("polylab_batch_run", _lib.polylab_batch_run(self.h, _stream()))

    STAGES = ("terms", "frame", "third")

    def check(self):
        """Synchronise and raise if a bounded wait of any earlier run expired."""
        _check("polylab_batch_check", _lib.polylab_batch_check(self.h, _stream()))

    def run_stage(self, stage: int):
        _check("polylab_batch_run_stage", _lib.polylab_batch_run_stage(self.h, stage, _stream()))

    CONFIG_KEYS = ("threads", "ctas_per_sm", "order", "term_threads", "terms_ctas", "third_ctas", "frame_split",
                   "third_threads", "third_split")

    def config(self):
        c = _BatchConfig()
        _check("polylab_batch_get_config", _lib.polylab_batch_get_config(self.h, C.byref(c)))
        return {k: getattr(c, k) for k in self.CONFIG_KEYS}

    def set_config(self, threads, ctas_per_sm, order, term_threads=None, terms_ctas=None, third_ctas=None,
                   frame_split=None, third_threads=None, third_split=None):
        """Keys left as None keep their current value."""
        cur = self.config()
        given = dict(threads=threads, ctas_per_sm=ctas_per_sm, order=order, term_threads=term_threads,
                     terms_ctas=terms_ctas, third_ctas=third_ctas, frame_split=frame_split,
                     third_threads=third_threads, third_split=third_split)
        c = _BatchConfig(*[cur[k] if given[k] is None else given[k] for k in self.CONFIG_KEYS])
        _check("polylab_batch_set_config", _lib.polylab_batch_set_config(self.h, C.byref(c), _stream()))

    def autotune(self, reps=2):
        c, t = _BatchConfig(), C.c_float()
        _check("polylab_batch_autotune", _lib.polylab_batch_autotune(self.h, reps, _stream(), C.byref(c), C.byref(t)))
        return {k: getattr(c, k) for k in self.CONFIG_KEYS}, float(t.value)

    def close(self):
        if self.h:
            _lib.polylab_batch_destroy(self.h, _stream())
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_PARAMS = 355
MLP_FEATURES = 7
MLP_PROBES = 4


def mlp_data(p: DevPoly, X: torch.Tensor, regularization: float, seed: int, plan: Plan | None = None):
    """(feats, hdiag, e, Z, Y) float32 device tensors (polylab_mlp_data)."""
    P, n = X.shape
    dev = X.device
    feats = torch.empty(P, n, MLP_FEATURES, dtype=torch.float32, device=dev)
    hd = torch.empty(P, n, dtype=torch.float32, device=dev)
    e = torch.empty(P, n, dtype=torch.float32, device=dev)
    Z = torch.empty(P, n, MLP_PROBES, dtype=torch.float32, device=dev)
    Y = torch.empty(P, n, MLP_PROBES, dtype=torch.float32, device=dev)
    cp = p.cstruct()
    _check("polylab_mlp_data", _lib.polylab_mlp_data(C.byref(cp), plan.h if plan else None, _ptr(X), P, regularization,
                                                     seed, _ptr(feats), _ptr(hd), _ptr(e), _ptr(Z), _ptr(Y),
                                                     _stream()))
    return feats, hd, e, Z, Y


def mlp_loss_grad(params, data, regularization):
    feats, hd, e, Z, Y = data
    P, n = hd.shape
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=params.device)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    _check("polylab_mlp_loss_grad", _lib.polylab_mlp_loss_grad(_ptr(params), P, n, _ptr(feats), _ptr(hd), _ptr(e),
                                                               _ptr(Z), _ptr(Y), regularization, _ptr(grad),
                                                               _ptr(loss), _stream()))
    return loss, grad


def mlp_pack(params):
    """BF16 copy of FP32 network parameters (polylab_mlp_pack), the form
    opts.mlp_weights takes."""
    packed = torch.empty(MLP_PARAMS, dtype=torch.bfloat16, device=params.device)
    _check("polylab_mlp_pack", _lib.polylab_mlp_pack(_ptr(params), _ptr(packed), _stream()))
    return packed


def train_preconditioner(data, regularization, steps=200, lr=3e-3, seed=1, device="cuda"):
    """Adam on the library's loss/gradient kernels; returns (fp32 params,
    packed bf16 weights for opts.mlp_weights, loss history)."""
    params = torch.empty(MLP_PARAMS, dtype=torch.float32, device=device)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    _check("polylab_mlp_init", _lib.polylab_mlp_init(_ptr(params), seed, _stream()))
    hist = []
    for step in range(1, steps + 1):
        loss, grad = mlp_loss_grad(params, data, regularization)
        hist.append(loss)
        _check("polylab_mlp_adam", _lib.polylab_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), step, lr,
                                                         _stream()))
    final, _ = mlp_loss_grad(params, data, regularization)
    hist.append(final)
    return params, mlp_pack(params), [float(h) for h in torch.cat(hist).cpu()]
