"""The C-ABI library loads, exports every symbol include/rf.h declares, and
validates graphs on the host (no GPU work)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2003_12861_gb300 import _lib as L
from paper_2003_12861_gb300 import api
from paper_2003_12861_gb300 import workloads as W
from paper_2003_12861_gb300.workloads import Node

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            syms |= set(re.findall(r"\b(rf_[a-z0-9_]+)\s*\(", text))
    return syms


def test_library_exports_every_declared_symbol():
    lib = L.load()
    syms = declared_symbols()
    assert "rf_nll_grad" in syms and "rf_model_create" in syms
    missing = [s for s in sorted(syms) if not hasattr(lib, s)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(rf_[a-z0-9_]+)\b", out))
    assert syms <= exported, sorted(syms - exported)


def test_binding_covers_every_declared_symbol():
    assert declared_symbols() <= set(L.SIGNATURES)


def test_version():
    assert b"sm_103a" in L.load().rf_version()


@pytest.mark.parametrize("which", ["gauss_poly1_model", "decay_model", "prod3_model"])
def test_models_compile_on_host(which):
    spec = W.model_for(which)
    m = api.Model.from_spec(spec)
    assert m.n_free == spec.n_free and m.n_obs == spec.n_obs
    assert "free=%d" % spec.n_free in m.describe()


BASE = [Node("obs", (), 0, 0, 10), Node("param", (), 4.0, 0, 10, True), Node("param", (), 1.2, 0.1, 5, True),
        Node("gauss", (0, 1, 2))]


@pytest.mark.parametrize("nodes,root", [
    (BASE + [Node("prod", (3, 3))], 4),                                   # PROD over one observable twice
    (BASE + [Node("obs", (), 0, 0, 1), Node("poly", (4,)), Node("param", (), 0.5, 0, 1, True),
             Node("sum", (3, 5, 6))], 7),                                  # SUM over different observables
    (BASE + [Node("gauss", (0, 3, 2))], 4),                               # pdf where a parameter belongs
    (BASE, 1),                                                             # root is a parameter
    ([Node("obs", (), 0, 1, 1)] + BASE[1:3] + [Node("gauss", (0, 1, 2))], 3),  # empty range
    (BASE[:3] + [Node("gauss", (0, 1))], 3),                              # arity
    (BASE + [Node("sum", (3, 5, 1)), Node("sum", (3, 4, 1))], 4),         # cycle through two SUMs
])
def test_invalid_graphs_rejected(nodes, root):
    with pytest.raises(L.RFError) as e:
        api.Model(nodes, root)
    assert e.value.status == L.RF_E_INVALID


def test_too_many_free_parameters_rejected():
    nodes = [Node("obs", (), 0, 0, 1)]
    for i in range(17):
        nodes.append(Node("param", (), 0.0, -1, 1, True))
    nodes.append(Node("poly", (0, 1, 2, 3, 4, 5, 6, 7)))
    with pytest.raises(L.RFError):
        api.Model(nodes, len(nodes) - 1)


def test_null_arguments_are_errors_not_crashes():
    lib = L.load()
    assert lib.rf_model_create(None, 0, 0, None) == L.RF_E_INVALID
    h = C.c_void_p()
    assert lib.rf_model_create(None, 3, 0, C.byref(h)) == L.RF_E_INVALID
    assert lib.rf_last_error()


# ----------------------------------------------- allocation-free pass: host side

# The documented limits of rf_nll_grad_noalloc's 16 MiB static scratch
# (include/rf.h): about 2e8 events for the float-float shapes with 6
# gradient slots, 1.4e8 with 12, about 5e8 for the generic kernel.
@pytest.mark.parametrize("which,lo,hi", [("decay_model", 1.9e8, 2.2e8), ("prod3_model", 1.35e8, 1.55e8),
                                         ("decay_generic_model", 4.5e8, 5.5e8)])
def test_noalloc_limit_matches_documented_figures(which, lo, hi):
    m = api.Model.from_spec(W.model_for(which))
    n_max = api.noalloc_max_events(m)
    assert lo <= n_max <= hi, n_max
    assert n_max % 4096 == 0


@pytest.mark.parametrize("which", ["decay_model", "prod3_model", "decay_generic_model"])
def test_noalloc_rejects_one_chunk_beyond_the_limit(which):
    # Through the C ABI; the size is checked before any device call, so
    # nothing is read from the (dummy) column pointers.
    m = api.Model.from_spec(W.model_for(which))
    n_max = api.noalloc_max_events(m)
    lib = L.load()
    ptrs = (C.c_void_p * m.n_obs)(*([0x1000] * m.n_obs))
    st = lib.rf_nll_grad_noalloc(m._h, ptrs, None, n_max + 1, C.c_void_p(0x1000), C.c_void_p(0x1000),
                                 C.c_void_p(0x1000), None)
    assert st == L.RF_E_INVALID
    assert b"static array" in lib.rf_last_error()


class _FakeTensor:
    """Duck-typed stand-in for a tensor: enough for the argument checks of
    nll_grad_noalloc, which must reject it before the C call."""

    def __init__(self, dtype, numel, is_cuda=True, contiguous=True):
        self.dtype, self._n, self.is_cuda, self._c = dtype, numel, is_cuda, contiguous

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c

    def data_ptr(self):  # never reached: the checks fail first
        raise AssertionError("the C entry point must not be called")


def test_noalloc_wrapper_rejects_bad_buffers_on_the_host():
    import torch

    m = api.Model.from_spec(W.decay_model())
    P = m.n_free
    good = dict(cols=[_FakeTensor(torch.float64, 100)], d_theta=_FakeTensor(torch.float64, P),
                d_out=_FakeTensor(torch.float64, 1 + P), d_flags=_FakeTensor(torch.int32, 1))
    bad_cases = [
        dict(cols=[]),                                                       # column count
        dict(cols=[_FakeTensor(torch.float64, 100)] * 2),
        dict(cols=[_FakeTensor(torch.float64, 100, is_cuda=False)]),         # host tensor
        dict(cols=[_FakeTensor(torch.float64, 100, contiguous=False)]),
        dict(cols=[_FakeTensor(torch.float16, 100)]),                        # dtype
        dict(cols=[_FakeTensor(torch.int32, 100)]),
        dict(d_theta=_FakeTensor(torch.float32, P)),
        dict(d_theta=_FakeTensor(torch.float64, P - 1)),
        dict(d_theta=_FakeTensor(torch.float64, P + 1)),
        dict(d_out=_FakeTensor(torch.float64, P)),
        dict(d_out=_FakeTensor(torch.float32, 1 + P)),
        dict(d_flags=_FakeTensor(torch.int64, 1)),
        dict(d_flags=_FakeTensor(torch.int32, 0)),
        dict(d_flags=_FakeTensor(torch.int32, 1, is_cuda=False)),
    ]
    for case in bad_cases:
        args = dict(good, **case)
        with pytest.raises(ValueError):
            api.nll_grad_noalloc(m, args["cols"], args["d_theta"], args["d_out"], args["d_flags"])
    # columns of unequal length (a two-observable model)
    m3 = api.Model.from_spec(W.prod3_model())
    P3 = m3.n_free
    with pytest.raises(ValueError):
        api.nll_grad_noalloc(m3, [_FakeTensor(torch.float32, 10), _FakeTensor(torch.float32, 10),
                                  _FakeTensor(torch.float32, 11)], _FakeTensor(torch.float64, P3),
                             _FakeTensor(torch.float64, 1 + P3), _FakeTensor(torch.int32, 1))


def test_fp64_switch_selects_the_interpreter():
    m = api.Model.from_spec(W.prod3_model())
    assert "kernel=ff_prod3" in m.describe()
    m.set_fp64(True)
    assert "kernel=generic_fp64" in m.describe()
    m.set_fp64(False)
    assert "kernel=ff_prod3" in m.describe()
    assert L.load().rf_model_set_fp64(m._h, 2) == L.RF_E_INVALID


def test_expr_models_compile_and_bad_programs_are_rejected():
    m = api.Model.from_spec(W.expr_mix_model())
    assert "EXPR" in m.describe() and "kernel=generic_fp64" in m.describe()
    lib = L.load()
    nodes = [Node("obs", (), 0.0, 0.0, 1.0), Node("param", (), 0.5, 0.0, 1.0, True),
             Node("expr", (0, 1), prog=W.expr_program("x p0 *"))]
    arr = api.make_nodes(nodes)
    h = C.c_void_p()
    # an EXPR node without a program
    assert lib.rf_model_create(arr, 3, 2, C.byref(h)) == L.RF_E_INVALID
    bad = ["x +", "x x", "p1", "c0", " ".join(["x"] * 17) + " +" * 16, " ".join(["x exp"] * 33)]
    for text in bad:
        ops = W.expr_program(text)
        o = (C.c_int32 * len(ops))(*ops)
        ex = (L.rf_expr * 1)()
        ex[0].node, ex[0].n_ops, ex[0].ops, ex[0].n_consts = 2, len(ops), o, 0
        assert lib.rf_model_create_expr(arr, 3, 2, ex, 1, C.byref(h)) == L.RF_E_INVALID, text
    # a program for a node that is not EXPR
    ops = W.expr_program("x")
    o = (C.c_int32 * 1)(*ops)
    ex = (L.rf_expr * 1)()
    ex[0].node, ex[0].n_ops, ex[0].ops, ex[0].n_consts = 1, 1, o, 0
    assert lib.rf_model_create_expr(arr, 3, 2, ex, 1, C.byref(h)) == L.RF_E_INVALID


def test_launch_shape_is_128_threads_with_tunable_blocks_per_sm():
    m = api.Model.from_spec(W.decay_model())
    m.set_launch(128, 4)
    m.set_launch(0, 0)
    for t in (64, 256, 512):
        with pytest.raises(L.RFError):
            m.set_launch(t, 4)
    with pytest.raises(L.RFError):
        m.set_launch(128, 33)


def test_fit_options_layout_matches_the_header():
    """rf_fit_opts as include/rf.h lays it out: tol_edm, max_evals,
    want_cov, no_graph, host_steps (the binding's ctypes struct is what the
    library reads)."""
    src = open(os.path.join(ROOT, "include", "rf.h")).read()
    body = src[src.index("typedef struct {", src.index("/* ------------------------------------------------------------------- fits */")):]
    body = body[: body.index("} rf_fit_opts;")]
    fields = [ln.split(";")[0].split()[-1] for ln in body.splitlines() if ";" in ln and ln.strip().split()[0] in ("double", "int32_t")]
    assert fields == ["tol_edm", "max_evals", "want_cov", "no_graph", "host_steps"], fields
    assert [f[0] for f in L.rf_fit_opts._fields_] == fields
    assert C.sizeof(L.rf_fit_opts) == 24
    assert L.rf_fit_opts.host_steps.offset == 20
