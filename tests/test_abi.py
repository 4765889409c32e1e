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
