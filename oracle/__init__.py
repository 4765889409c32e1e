"""CPU oracle for the batched unbinned-likelihood hot path (test infrastructure).

Only the tests, the package's smoke check and the benchmark's CPU-baseline leg
may import this package.  It loads ``liboracle.so`` built from ``oracle.cpp``
(plain single-threaded C++17, compiled with ``-ffp-contract=off``) and the
numpy MLP reference in ``mlp.py``.  It imports nothing from the CUDA package;
models arrive as plain node lists (objects with ``kind``, ``inputs``, ``value``,
``lo``, ``hi``, ``free`` attributes; an ``expr`` node also carries ``prog`` and
``consts``, its postfix program) and data as numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

# The oracle's own numbering of node kinds (independent of the CUDA library's).
_KIND = {"obs": 0, "param": 1, "gauss": 2, "exp": 3, "gaussexp": 4, "cheb": 5, "poly": 6, "sum": 7, "prod": 8,
         "poisson": 9, "extend": 10, "expr": 11}


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (g++, C++17, no fp contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp, ip, vp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p
        L.orc_model_new.restype = vp
        L.orc_model_new.argtypes = [C.c_int, ip, ip, ip, dp, dp, dp, ip, C.c_int]
        L.orc_model_free.argtypes = [vp]
        L.orc_model_set_expr.argtypes = [vp, C.c_int, C.c_int, ip, C.c_int, dp]
        L.orc_n_free.argtypes = [vp]
        L.orc_n_obs.argtypes = [vp]
        L.orc_last_error.restype = C.c_char_p
        L.orc_leaf_norm.argtypes = [vp, C.c_int, dp, dp, dp]
        L.orc_leaf_shape.restype = C.c_double
        L.orc_leaf_shape.argtypes = [vp, C.c_int, dp, C.c_double]
        L.orc_pdf.argtypes = [vp, C.c_int, dp, C.POINTER(dp), C.c_int64, dp, dp]
        L.orc_nll.argtypes = [vp, dp, C.POINTER(dp), C.c_int64, dp, dp, dp, dp]
        L.orc_fit.argtypes = [vp, C.POINTER(dp), C.c_int64, dp, C.c_double, C.c_int, dp, dp, dp, ip]
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        L.orc_poisson.restype = C.c_int64
        L.orc_poisson.argtypes = [C.c_uint64, C.c_uint32, C.c_double]
        L.orc_gen_bounds.argtypes = [vp, dp, dp, C.c_int]
        L.orc_generate.argtypes = [vp, dp, dp, C.c_uint64, C.c_uint32, C.c_int64, C.c_int64, C.POINTER(dp)]
        L.orc_hist64.argtypes = [dp, C.c_int64, C.c_double, C.c_double, C.POINTER(C.c_float)]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Model:
    """An oracle model built from a node list and the index of its top pdf."""

    def __init__(self, nodes, root: int):
        L = lib()
        n = len(nodes)
        kinds = np.array([_KIND[nd.kind] for nd in nodes], dtype=np.int32)
        nin = np.array([len(nd.inputs) for nd in nodes], dtype=np.int32)
        ins = np.zeros((n, 8), dtype=np.int32)
        for i, nd in enumerate(nodes):
            if len(nd.inputs) > 8:
                raise ValueError("at most 8 inputs per node")
            ins[i, : len(nd.inputs)] = nd.inputs
        vals = np.array([nd.value for nd in nodes], dtype=np.float64)
        los = np.array([nd.lo for nd in nodes], dtype=np.float64)
        his = np.array([nd.hi for nd in nodes], dtype=np.float64)
        free = np.array([1 if nd.free else 0 for nd in nodes], dtype=np.int32)
        ip = C.POINTER(C.c_int)
        h = L.orc_model_new(n, kinds.ctypes.data_as(ip), nin.ctypes.data_as(ip), ins.ctypes.data_as(ip),
                            _dp(vals), _dp(los), _dp(his), free.ctypes.data_as(ip), root)
        if not h:
            raise ValueError("oracle rejected the model: " + L.orc_last_error().decode())
        self._h = h
        for i, nd in enumerate(nodes):
            if nd.kind == "expr":
                ops = np.ascontiguousarray(getattr(nd, "prog", ()), dtype=np.int32)
                cst = np.ascontiguousarray(getattr(nd, "consts", ()), dtype=np.float64)
                if L.orc_model_set_expr(h, i, len(ops), ops.ctypes.data_as(ip), len(cst),
                                        _dp(cst) if len(cst) else None) != 0:
                    raise ValueError("oracle rejected the program: " + L.orc_last_error().decode())
        self.nodes = list(nodes)
        self.root = root
        self.n_free = L.orc_n_free(h)
        self.n_obs = L.orc_n_obs(h)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_model_free(self._h)
            self._h = None

    def _cols(self, cols):
        cols = [_f64(c) for c in cols]
        if len(cols) != self.n_obs:
            raise ValueError(f"expected {self.n_obs} columns")
        arr = (C.POINTER(C.c_double) * len(cols))(*[_dp(c) for c in cols])
        return cols, arr, (len(cols[0]) if cols else 0)

    def leaf_norm(self, node: int, theta):
        theta = _f64(theta)
        I = C.c_double()
        dI = np.zeros(max(self.n_free, 1))
        rc = lib().orc_leaf_norm(self._h, node, _dp(theta), C.byref(I), _dp(dI))
        if rc != 0:
            raise ValueError(f"leaf_norm failed ({rc})")
        return I.value, dI[: self.n_free]

    def leaf_shape(self, node: int, theta, x: float) -> float:
        theta = _f64(theta)
        return lib().orc_leaf_shape(self._h, node, _dp(theta), float(x))

    def pdf(self, theta, cols, node: int | None = None, grad: bool = False):
        theta = _f64(theta)
        keep, arr, N = self._cols(cols)
        p = np.zeros(N)
        g = np.zeros((N, self.n_free)) if grad else None
        rc = lib().orc_pdf(self._h, self.root if node is None else node, _dp(theta), arr, N, _dp(p),
                           _dp(g) if grad else None)
        if rc != 0:
            raise ValueError(f"pdf failed ({rc})")
        return (p, g) if grad else p

    def nll(self, theta, cols):
        """(nll, grad, sum|log p|, sum|dlog p/dtheta|, status)."""
        theta = _f64(theta)
        keep, arr, N = self._cols(cols)
        nll = C.c_double()
        g = np.zeros(max(self.n_free, 1))
        ag = np.zeros(max(self.n_free, 1))
        al = C.c_double()
        rc = lib().orc_nll(self._h, _dp(theta), arr, N, C.byref(nll), _dp(g), C.byref(al), _dp(ag))
        return nll.value, g[: self.n_free].copy(), al.value, ag[: self.n_free].copy(), rc

    def fit(self, cols, theta0=None, tol_edm=1e-10, max_evals=2000, cov=True):
        keep, arr, N = self._cols(cols)
        th0 = None if theta0 is None else _f64(theta0)
        th = np.zeros(self.n_free)
        nll = C.c_double()
        cv = np.zeros((self.n_free, self.n_free)) if cov else None
        ne = C.c_int()
        rc = lib().orc_fit(self._h, arr, N, _dp(th0) if th0 is not None else None, tol_edm, max_evals, _dp(th),
                           C.byref(nll), _dp(cv) if cov else None, C.byref(ne))
        return dict(theta=th, nll=nll.value, cov=cv, n_evals=ne.value, status=rc)

    def gen_bounds(self, theta, max_factors=8):
        theta = _f64(theta)
        b = np.zeros(max_factors)
        n = lib().orc_gen_bounds(self._h, _dp(theta), _dp(b), max_factors)
        if n < 0:
            raise ValueError("cannot generate from this model")
        return b[:n]

    def generate(self, theta, seed: int, set_index: int, i0: int, i1: int, bounds=None):
        """Events [i0, i1) of set `set_index`; returns a list of float64 columns."""
        theta = _f64(theta)
        bnd = _f64(self.gen_bounds(theta) if bounds is None else bounds)
        cols = [np.zeros(i1 - i0) for _ in range(self.n_obs)]
        arr = (C.POINTER(C.c_double) * self.n_obs)(*[_dp(c) for c in cols])
        rc = lib().orc_generate(self._h, _dp(theta), _dp(bnd), seed, set_index, i0, i1, arr)
        if rc != 0:
            raise RuntimeError("generation failed")
        return cols


def philox4x32_10(ctr, key):
    a = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(a, k, o)
    return list(o)


def poisson(seed: int, set_index: int, mu: float) -> int:
    return int(lib().orc_poisson(seed, set_index, mu))


def hist64(x, lo: float, hi: float):
    x = _f64(x)
    out = np.zeros(64, dtype=np.float32)
    lib().orc_hist64(_dp(x), len(x), lo, hi, out.ctypes.data_as(C.POINTER(C.c_float)))
    return out
