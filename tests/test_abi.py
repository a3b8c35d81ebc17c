"""CPU checks of the C ABI: the library loads and exports every symbol that
include/eofa.h declares, with the struct layouts the binding assumes.  No
compute call is made (there may be no GPU)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eofa.h")


@pytest.fixture(scope="module")
def libeofa():
    from paper_1706_05843_gb300 import build
    build.build()
    from paper_1706_05843_gb300 import binding
    return binding.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eofa_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["eofa_create", "eofa_apply", "eofa_apply_dag", "eofa_apply_h", "eofa_solve",
              "eofa_apply_batched", "eofa_solve_batched", "eofa_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(libeofa):
    from paper_1706_05843_gb300 import binding
    for n in declared_functions():
        assert hasattr(libeofa, n), n
        assert n in binding.SIGNATURES, n
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (eofa_[a-z_]+)\b", out))
    assert set(declared_functions()) <= exported


def test_struct_layouts():
    from paper_1706_05843_gb300 import binding as B
    # sizes implied by include/eofa.h on LP64
    assert C.sizeof(B.eofa_params) == 4 * 4 + 4 + 4 + 7 * 8 + 4 + 4
    assert C.sizeof(B.eofa_solve_opts) == 8 + 4 + 4 + 8 + 6 * 4 + 8
    assert C.sizeof(B.eofa_solve_stats) == 4 * 4 + 5 * 8 + 8 + 2 * 4 + 8
    assert C.sizeof(B.eofa_train_opts) == 4 * 4 + 2 * 8 + 8      # holdout + tail padding
    assert C.sizeof(B.eofa_train_stats) == 3 * 4 + 4 + 3 * 8 + 4 + 4 + 2 * 8   # with alignment padding


def test_status_strings(libeofa):
    from paper_1706_05843_gb300 import binding as B
    assert B.eofa_status_string(0) == "ok"
    assert "converged" in B.eofa_status_string(4)


def test_status_strings_cover_every_code(libeofa):
    """Every code of the eofa_status enum in include/eofa.h has its own
    description; a value outside the enum gets the fallback."""
    from paper_1706_05843_gb300 import binding as B
    src = open(HEADER).read()
    enum = src[src.index("typedef enum"):src.index("} eofa_status;")]
    codes = [int(v) for v in re.findall(r"EOFA_[A-Z_]+\s*=\s*(\d+)", enum)]
    assert codes == list(range(len(codes))) and len(codes) == len(B.STATUS)
    texts = [B.eofa_status_string(c) for c in codes]
    assert len(set(texts)) == len(codes)
    fallback = B.eofa_status_string(len(codes))
    assert fallback not in texts
    assert B.eofa_status_string(-1) == fallback


def test_argument_errors_without_gpu(libeofa):
    """Invalid arguments are rejected before any device work."""
    from paper_1706_05843_gb300 import binding as B
    ctx = C.c_void_p()
    p = B.make_params((4, 4, 4, 3), 8)          # odd extent
    assert libeofa.eofa_create(C.byref(p), C.c_void_p(1), None, C.byref(ctx)) == 1
    p = B.make_params((4, 4, 4, 4), 8, pm=0)    # bad chirality
    assert libeofa.eofa_create(C.byref(p), C.c_void_p(1), None, C.byref(ctx)) == 1
    p = B.make_params((4, 4, 4, 4), 6)          # Ls outside the compiled set
    assert libeofa.eofa_create(C.byref(p), C.c_void_p(1), None, C.byref(ctx)) == 2
    assert libeofa.eofa_create(C.byref(p), None, None, C.byref(ctx)) == 1
    assert libeofa.eofa_apply(None, None, None, None) == 1
    assert libeofa.eofa_solve(None, None, None, None, None, None) == 1
    # G-parity: the direction mask must name 1..4 directions; the same
    # parameter checks as eofa_create
    p = B.make_params((4, 4, 4, 4), 8)
    for dirs in (0, 16, -1):
        assert libeofa.eofa_create_gparity(C.byref(p), C.c_void_p(1), dirs, None, C.byref(ctx)) == 1
    p = B.make_params((4, 4, 4, 3), 8)
    assert libeofa.eofa_create_gparity(C.byref(p), C.c_void_p(1), 1, None, C.byref(ctx)) == 1
    # host-buffer solve and the FMA probe: argument checks before any device work
    assert libeofa.eofa_solve_host(None, None, None, None, None, None) == 1
    out = C.c_double(0.0)
    assert libeofa.eofa_measure_fma(2, 3, C.byref(out), None) == 1   # FP16 has no FMA probe
    assert libeofa.eofa_measure_fma(0, 0, C.byref(out), None) == 1   # reps < 1
    assert libeofa.eofa_measure_fma(0, 3, None, None) == 1
    assert libeofa.eofa_dot(None, None, None, 0, None, None, None) == 1
    assert libeofa.eofa_force_norms(None, None, None, None, None) == 1
    # action calls without a context
    opts = B.make_opts(tol=1e-10)
    assert libeofa.eofa_set_system(None, 0.04, 1.0, 0.04, -1.0, 1) == 1
    assert libeofa.eofa_apply_meofa(None, 0.04, 1.0, None, None, C.byref(opts), None, None) == 1
    assert libeofa.eofa_force(None, 0.04, 1.0, None, None, C.byref(opts), None, None) == 1
    assert libeofa.eofa_heatbath(None, 0.04, 1.0, 0, None, None, None, 0, None, None, C.byref(opts), None,
                                 None) == 1


def test_empty_batches_are_no_ops(libeofa):
    """n = 0 returns EOFA_OK before touching any pointer or the device."""
    from paper_1706_05843_gb300 import binding as B
    opts = B.make_opts(tol=1e-10)
    assert libeofa.eofa_solve_batched(None, 0, None, None, C.byref(opts), None, None) == 0
    assert libeofa.eofa_solve_batched(None, 0, None, None, None, None, None) == 0
    assert libeofa.eofa_apply_batched(None, 0, None, None, 0, None) == 0
    assert libeofa.eofa_solve_batched(None, -1, None, None, None, None, None) == 1


def test_more_argument_errors_without_gpu(libeofa):
    """The remaining entry points reject missing arguments before any device
    work; the queries answer for a missing context without touching it."""
    from paper_1706_05843_gb300 import binding as B
    assert libeofa.eofa_apply_dag(None, None, None, None) == 1
    assert libeofa.eofa_apply_h(None, None, None, None) == 1
    p = B.make_params((4, 4, 4, 4), 8)
    assert libeofa.eofa_apply_noalloc(C.byref(p), None, None, None, None) == 1
    dims = (C.c_int * 4)(4, 4, 4, 4)
    assert libeofa.eofa_net_forward(None, dims, 1, None, None, None) == 1
    assert libeofa.eofa_net_forward(None, None, 1, None, None, None) == 1
    assert libeofa.eofa_net_backward(None, dims, 1, None, None, None, None, None) == 1
    assert libeofa.eofa_set_preconditioner(None, None) == 1
    assert libeofa.eofa_train_preconditioner(None, None, 0, None, None, None, None, None) == 1
    # a missing source among the sources (no context needed to reject it)
    w = (C.c_float * B.NET_WEIGHTS)()
    topts = B.make_train_opts()
    srcs = (C.c_void_p * 2)(1, None)
    assert libeofa.eofa_train_preconditioner(C.c_void_p(1), srcs, 2, w, C.byref(topts), w, None, None) == 1
    assert libeofa.eofa_last_error(None) == b""
    assert libeofa.eofa_tile_variant(None, 1, 0) == -1
    assert libeofa.eofa_tile_time(None, 1, 0, 0) == -1.0
    assert libeofa.eofa_hop_bytes(None, 1, 0) == 0.0
    libeofa.eofa_destroy(None)  # a no-op


def test_binding_checks_network_weight_count():
    """The library copies exactly NET_WEIGHTS weights from the host: the
    binding refuses any other count before calling it."""
    from paper_1706_05843_gb300 import binding as B
    for call in (lambda w: B.eofa_net_forward(w, (4, 4, 4, 4), None, None),
                 lambda w: B.eofa_net_backward(w, (4, 4, 4, 4), None, None),
                 lambda w: B.eofa_set_preconditioner(None, w)):
        with pytest.raises(ValueError):
            call(np.zeros(B.NET_WEIGHTS - 1, dtype=np.float32))


def test_binding_size_checks_without_gpu():
    """The Solver's size checks are host logic: a field of another size is
    refused before any library call."""
    from paper_1706_05843_gb300 import binding as B
    B._need(np.zeros(24, dtype=np.complex128), 24, "field")
    with pytest.raises(ValueError):
        B._need(np.zeros(23, dtype=np.complex128), 24, "field")
    with pytest.raises(ValueError):
        B.solve_batched([object(), object()], [None], tol=1e-10)   # one rhs for two solvers
    with pytest.raises(ValueError):
        B._net_rows((2, 2, 2, 2), np.zeros((1, 2, 2, 2, 2, 23), dtype=np.float32))
