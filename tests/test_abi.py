"""The C-ABI library loads and exports every function include/polylab.h
declares (no device needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(polylab_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_library_exports_every_declared_symbol():
    import __graft_entry__  # noqa: F401  (its build() compiles the in-tree .so)
    path = os.path.join(ROOT, "paper_2604_06575_b300", "libpolylab.so")
    if not os.path.exists(path):
        __graft_entry__.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert "polylab_affine_normal" in names and "polylab_simplify" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_declared_symbols():
    from paper_2604_06575_b300 import polylab
    for n in declared_functions():
        assert n in polylab.EXPORTED, n
    assert polylab.lib().polylab_status_string(7) == b"POLYLAB_ERR_UNSUPPORTED"


def test_default_options_match_paper_table():
    """Sec. 5 Table "affineopts": method mf-exact, regularization 1e-6,
    num_probes 8, krylov_tol 1e-4, krylov_maxit 40."""
    from paper_2604_06575_b300 import polylab
    o = polylab._AnOpts()
    polylab.lib().polylab_an_opts_default(ctypes.byref(o))
    assert (o.method, o.regularization, o.num_probes, o.krylov_tol, o.krylov_maxit) == (0, 1e-6, 8, 1e-4, 40)


def test_bench_counts_launches_per_step():
    """The bench's claim of kernel launches per step follows the configuration:
    the frame stage runs one launch per non-empty class of n when split."""
    import numpy as np

    import bench
    from paper_2604_06575_b300 import workloads
    rng = np.random.default_rng(0)
    polys = [workloads.convexified(rng, n, workloads.sparse_monomials(rng, n, 20, 3, 2), 0.1) for n in (5, 30, 50)]
    Xs = [np.zeros((4, p.n)) for p in polys]
    assert bench.stage_launches(dict(frame_split=1), polys, Xs) == dict(terms=4, frame=3, third=3)
    assert bench.stage_launches(dict(frame_split=1), polys[:1], Xs[:1]) == dict(terms=2, frame=1, third=1)
    assert bench.stage_launches(dict(frame_split=0), polys, Xs) == dict(terms=4, frame=1, third=3)
    assert bench.stage_launches(dict(frame_split=1, third_split=2), polys, Xs) == dict(terms=4, frame=3, third=6)


def test_header_is_plain_c(tmp_path):
    """include/polylab.h is a C interface: it compiles as strict C99 (and as
    C++), with every declared type usable from C."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "polylab.h"\n'
                   "int main(void) {\n"
                   "  polylab_an_opts o; polylab_an_opts_default(&o);\n"
                   "  polylab_poly p = {0}; polylab_poly_f32 q = {0}; polylab_batch_config c = {0};\n"
                   "  (void)p; (void)q; (void)c; return (int)o.method;\n"
                   "}\n")
    inc = os.path.join(ROOT, "include")
    for cmd in ([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, "-c", str(src),
                 "-o", str(tmp_path / "a.o")],
                [gcc, "-x", "c++", "-std=c++17", "-Wall", "-Werror", "-I", inc, "-c", str(src),
                 "-o", str(tmp_path / "b.o")]):
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
